"""Householder QR + solve on the GPU against the oracle (Sec. 2 Eqs. 2-3).

Tolerances (relative image error ||x - x_ref|| / ||x_ref||): FP64 path 1e-10,
plain FP32 path 1e-4.  Factors are compared through R (LAPACK sign
convention on both sides) and through invariants, since blockings differ."""
import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth


def _case(O, ns, nv, nb, sl, k, noisy, seed0=1234):
    g = O.Geometry(ns, nv, nb, sqrt_lambda=sl)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(ns, k, 8 if ns <= 32 else 10, seed0)
    P = O.forward(csr, X)
    B = synth.poisson_sinogram(P, ns, 1e4, seed=seed0) if noisy else P
    return g, csr, X, B


def _gpu_solve(torch, ct, g, B, precision, **kw):
    storage = "fp64" if precision == "fp64" else "fp32"
    sysg = ct.System(ct.make_geometry(g.n_side, g.n_views, g.n_bins, g.sqrt_lambda), storage)
    F = sysg.factor(precision, **kw)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda()
    X = F.solve(Bt, allow_noconv=True)
    return sysg, F, X.double().cpu().numpy().T


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_c1_noiseless_matches_oracle(oracle_mod, precision, tol):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, 32, 60, 46, 0.0, 3, False)
    Xo, VR, tau = O.qr_solve(g, O.dense_system(g, csr), B)
    sysg, F, Xg = _gpu_solve(torch, ct, g, B, precision)
    assert rel_err_cols(Xg, Xo).max() <= tol
    assert rel_err_cols(Xg, X).max() <= tol  # exact recovery from consistent data
    if precision == "fp64":
        VRg, taug = F.export()
        n = g.n
        Ro, Rg = np.triu(VR[:n]), np.triu(VRg[:n])
        np.testing.assert_allclose(Rg, Ro, rtol=0, atol=1e-11 * np.abs(Ro).max())
        np.testing.assert_allclose(taug, tau, rtol=0, atol=1e-11)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
@pytest.mark.parametrize("ns,nv,nb,sl", [(19, 31, 29, 0.05), (24, 40, 36, 0.05), (20, 37, 30, 0.0)])
def test_ragged_noisy_matches_oracle(oracle_mod, precision, tol, ns, nv, nb, sl):
    """Sizes that are not multiples of any tile or block (n = 361, 576, 400;
    M' = 1260, 2016, 1110), noisy data, with and without regularisation."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, ns, nv, nb, sl, 5, True)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    for nb_outer in (0, 64):
        _, _, Xg = _gpu_solve(torch, ct, g, B, precision, nb_outer=nb_outer)
        assert rel_err_cols(Xg, Xo).max() <= tol


@pytest.mark.gpu
def test_tf32_direct_solve_is_tf32_accurate(oracle_mod):
    """The TF32 tensor-core factorisation without refinement: error of the
    order of kappa * 2^-10, far above FP32 and far below 1."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, 32, 60, 46, 0.0, 3, False)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    sysg = ct.System(ct.make_geometry(32, 60, 46), "fp32")
    F = sysg.factor("tf32")
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xg = F.solve(Bt, max_iter=-1, allow_noconv=True).cpu().numpy().T
    err = rel_err_cols(Xg, Xo).max()
    print("tf32 direct error", err)
    assert err < 0.5


@pytest.mark.gpu
def test_adjoint_identity_fp64(oracle_mod):
    """<solve(b), y> = <b, adjoint(y)> (the adjoint is Q [R^-T y; 0] restricted
    to the ray rows)."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    sysg = ct.System(ct.make_geometry(24, 40, 36, 0.05), "fp64")
    F = sysg.factor("fp64")
    rng = np.random.default_rng(1)
    b = torch.from_numpy(rng.standard_normal((3, sysg.m))).cuda()
    y = torch.from_numpy(rng.standard_normal((3, sysg.n))).cuda()
    x = F.solve(b)
    gb = F.adjoint(y)
    lhs = (x * y).sum(1)
    rhs = (b * gb).sum(1)
    np.testing.assert_allclose(lhs.cpu().numpy(), rhs.cpu().numpy(), rtol=1e-12)


@pytest.mark.gpu
def test_adjoint_matches_oracle_gradient(oracle_mod):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(24, 40, 36, sqrt_lambda=0.05)
    VR, tau = O.householder_qr(O.dense_system(g))
    rng = np.random.default_rng(2)
    y = rng.standard_normal((g.n, 2))
    z = O.forwardsolve_rt(VR, y)
    full = np.zeros((g.rows, 2), order="F")
    full[: g.n] = z
    want = O.apply_q(VR, tau, full)[: g.m]
    sysg = ct.System(ct.make_geometry(24, 40, 36, 0.05), "fp64")
    F = sysg.factor("fp64")
    gb = F.adjoint(torch.from_numpy(np.ascontiguousarray(y.T)).cuda()).cpu().numpy().T
    np.testing.assert_allclose(gb, want, rtol=0, atol=1e-10 * np.abs(want).max())


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32", "bf16", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("ns,nv,nb,sl,noisy", [(32, 60, 46, 0.0, False), (24, 40, 36, 0.05, True),
                                               (19, 31, 29, 0.05, True)])
def test_refined_reaches_1e6(oracle_mod, precision, ns, nv, nb, sl, noisy):
    """TF32, BF16 or split-precision tensor-core factors + FP64 refinement:
    relative image error <= 1e-6 against the FP64 oracle solution."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, ns, nv, nb, sl, 4, noisy)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    sysg = ct.System(ct.make_geometry(ns, nv, nb, sl), "fp32")
    # small blocks so the BF16 trailing-update GEMMs run at these sizes
    F = sysg.factor(precision, nb_outer=64 if precision != "tf32" else 0)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xg = F.solve(Bt, max_iter=30, tol=1e-9).cpu().numpy().T
    print("refine info", F.last_info)
    assert rel_err_cols(Xg, Xo).max() <= 1e-6


@pytest.mark.gpu
def test_split_precision_widens_refinement(oracle_mod):
    """An ill-conditioned system (32x32 image from 30 views, no
    regularisation: condition number about 3e4, so TF32 or BF16 factors are
    poor preconditioners): the split-precision factors refine to the oracle
    solution in a few FP64 steps with a handful of inner steps, where the
    single-pass TF32 factor needs many times more inner steps."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, 32, 30, 46, 0.0, 3, False)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    info = {}
    for precision in ("tf32", "tf32x3", "bf16x3"):
        sysg = ct.System(ct.make_geometry(32, 30, 46, 0.0), "fp32")
        F = sysg.factor(precision, nb_outer=64)
        Xg = F.solve(Bt, max_iter=10, tol=1e-12, allow_noconv=True).cpu().numpy().T
        info[precision] = F.last_info
        print(precision, rel_err_cols(Xg, Xo).max(), F.last_info)
        if precision != "tf32":
            assert rel_err_cols(Xg, Xo).max() <= 1e-10
            assert F.last_info["iterations"] <= 6
    for precision in ("tf32x3", "bf16x3"):
        assert 5 * info[precision]["inner_iterations"] <= info["tf32"]["inner_iterations"]


@pytest.mark.gpu
def test_graph_replay_matches_eager(oracle_mod):
    """Repeated solves replay captured CUDA graphs (warm-up, capture, replay):
    the results equal the eager launches bit for bit."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, 24, 40, 36, 0.05, 5, True)
    sysg = ct.System(ct.make_geometry(24, 40, 36, 0.05), "fp32")
    F = sysg.factor("tf32")
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    F.graphs = False
    ref = F.solve(Bt, max_iter=12, tol=1e-12, allow_noconv=True).clone()
    F.graphs = True
    outs = [F.solve(Bt, max_iter=12, tol=1e-12, allow_noconv=True).clone() for _ in range(4)]
    for o in outs:
        assert torch.equal(o, ref)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32", "fp64"])
def test_factor_checkpoint_roundtrip(oracle_mod, tmp_path, precision):
    """A factor written to a file and read back (for a freshly built system of
    the same geometry) solves to the same bits; a corrupted file or another
    geometry is refused."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, 19, 31, 29, 0.05, 3, True)
    storage = "fp64" if precision == "fp64" else "fp32"
    geom = ct.make_geometry(19, 31, 29, 0.05)
    s1 = ct.System(geom, storage)
    F1 = s1.factor(precision)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    x1 = F1.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).clone()
    path = str(tmp_path / "factor.ctqr")
    F1.save(path)
    s2 = ct.System(geom, storage)
    F2 = ct.Factor.load(s2, path)
    assert F2.precision == precision
    x2 = F2.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True)
    assert torch.equal(x1, x2)
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0xFF
    open(path + ".bad", "wb").write(bytes(raw))
    with pytest.raises(ct.CTQRError):
        ct.Factor.load(s2, path + ".bad")
    s3 = ct.System(ct.make_geometry(19, 31, 30, 0.05), storage)
    with pytest.raises(ct.CTQRError):
        ct.Factor.load(s3, path)
    # tampered headers: block sizes the factorisation never makes are refused
    # before any data is read; any other header change fails the checksum,
    # which covers the header too
    import struct
    good = open(path, "rb").read()
    for off, val, why in ((40, 0, "block sizes"), (48, 0, "block sizes"),
                          (56, struct.unpack_from("<q", good, 56)[0] - 1, "block sizes"),
                          (48, 33, "block sizes")):
        raw = bytearray(good)
        struct.pack_into("<q", raw, off, val)
        open(path + ".hdr", "wb").write(bytes(raw))
        with pytest.raises(ct.CTQRError) as e:
            ct.Factor.load(s2, path + ".hdr")
        assert e.value.status == 1 and why in str(e.value), (off, str(e.value))
    import ctypes
    rjj_min_at = 64 + ctypes.sizeof(ct.Geometry)  # magic .. nblocks, then the geometry
    raw = bytearray(good)
    struct.pack_into("<d", raw, rjj_min_at, 123.0)
    open(path + ".hdr", "wb").write(bytes(raw))
    with pytest.raises(ct.CTQRError) as e:
        ct.Factor.load(s2, path + ".hdr")
    assert e.value.status == 1


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("tf32", 1e-6)])
def test_fan_beam_solve_matches_oracle(oracle_mod, precision, tol):
    """The whole path on a fan-beam system (24x24 image, 60 sources over 360
    degrees, 40 detectors over 30 degrees, source at 50 pixels, sqrt(lambda)
    = 0.05): GPU solve against the oracle's Householder QR solve."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    ns, nv, nd, fan, sid, sl = 24, 60, 40, 30.0, 50.0, 0.05
    g = O.Geometry(ns, nv, nd, arc_deg=360.0, sqrt_lambda=sl, kind="fan", source_dist=sid, fan_deg=fan)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(ns, 3, 8, 1234)
    B = synth.poisson_sinogram(O.forward(csr, X), ns, 1e4, seed=1234)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    storage = "fp64" if precision == "fp64" else "fp32"
    sysg = ct.System(ct.make_geometry(ns, nv, nd, sl, kind="fan", source_dist=sid, fan_deg=fan), storage)
    F = sysg.factor(precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda()
    Xg = F.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).double().cpu().numpy().T
    err = rel_err_cols(Xg, Xo)
    print(precision, "fan-beam max rel err", err.max(), F.last_info)
    assert err.max() <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("tf32", 1e-6)])
def test_joseph_solve_matches_oracle(oracle_mod, precision, tol):
    """The whole path on a Joseph-projector system (24x24, 40 views x 36
    bins, sqrt(lambda) = 0.05)."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    ns, nv, nb, sl = 24, 40, 36, 0.05
    g = O.Geometry(ns, nv, nb, sqrt_lambda=sl, projector="joseph")
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(ns, 3, 8, 1234)
    B = synth.poisson_sinogram(O.forward(csr, X), ns, 1e4, seed=1234)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    storage = "fp64" if precision == "fp64" else "fp32"
    sysg = ct.System(ct.make_geometry(ns, nv, nb, sl, projector="joseph"), storage)
    F = sysg.factor(precision)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xg = F.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).cpu().numpy().T
    err = rel_err_cols(Xg, Xo)
    print(precision, "joseph max rel err", err.max(), F.last_info)
    assert err.max() <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("tf32", 1e-6), ("bf16", 1e-6)])
@pytest.mark.parametrize("ns,nv,nb,sl,noisy", [(24, 40, 36, 0.05, True), (32, 60, 46, 0.0, False),
                                               (40, 70, 58, 0.05, True)])
def test_gram_panel_matches_column_panel(oracle_mod, precision, tol, ns, nv, nb, sl, noisy):
    """FP32 panels factored from their Gram matrices (CholeskyQR twice, then
    the Householder reflectors reconstructed) solve to the oracle's accuracy,
    like the column-by-column sweep; the factors agree with the sweep's to
    FP32 rounding (R up to the sign of each row), so the reconstruction gives
    the same reflectors."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, ns, nv, nb, sl, 3, noisy)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda()
    out = {}
    for column in (False, True):
        sysg = ct.System(ct.make_geometry(ns, nv, nb, sl), "fp32")
        F = sysg.factor(precision, nb_outer=64, column_panel=column)
        VR, tau = F.export()
        Xg = F.solve(Bt, max_iter=20, tol=1e-9, allow_noconv=True).double().cpu().numpy().T
        assert rel_err_cols(Xg, Xo).max() <= tol
        out[column] = (VR, tau)
    (VRg, taug), (VRc, tauc) = out[False], out[True]
    n = ns * ns
    Rg, Rc = np.triu(VRg[:n]), np.triu(VRc[:n])
    sg = np.sign(np.diag(Rg)) * np.sign(np.diag(Rc))
    scale = np.abs(Rc).max()
    # a few roundings of the trailing updates' operand type: TF32 (2^-11) and
    # FP32 panels within 2e-3 of the largest entry, BF16 (2^-8) within 8e-3
    r_tol = 8e-3 if precision == "bf16" else 2e-3
    assert np.abs(sg[:, None] * Rg - Rc).max() <= r_tol * scale
    assert not np.array_equal(VRg, VRc)  # a different kernel ran


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_fallback_panels_refine(oracle_mod, precision):
    """Panels too ill-conditioned for the Gram route (32x32 image, 30 views,
    no regularisation: condition number about 3e4) fall back to the
    column-by-column sweep, which then also builds the panel's T and the top
    of its V; the refined solve reaches the oracle solution as with the
    sweep alone."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B = _case(O, 32, 30, 46, 0.0, 3, False)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    for column in (False, True):
        sysg = ct.System(ct.make_geometry(32, 30, 46, 0.0), "fp32")
        F = sysg.factor(precision, nb_outer=64, column_panel=column)
        Xg = F.solve(Bt, max_iter=12, tol=1e-12, allow_noconv=True).cpu().numpy().T
        print(precision, column, rel_err_cols(Xg, Xo).max(), F.last_info)
        assert rel_err_cols(Xg, Xo).max() <= 1e-8
