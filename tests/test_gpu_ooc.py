"""Out-of-core path (host-resident dense matrix, left-looking superpanels
under a device budget): the host build equals the in-core build bit for
bit, and the out-of-core factorisation solves to the same accuracy as the
in-core one against the FP64 oracle, with budgets small enough to force
several superpanels and streamed V blocks."""
import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth

NS, NV, NBINS, SL = 24, 40, 36, 0.05


def _case(O, k=3):
    g = O.Geometry(NS, NV, NBINS, sqrt_lambda=SL)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(NS, k, 8, 1234)
    B = synth.poisson_sinogram(O.forward(csr, X), NS, 1e4, seed=1234)
    return g, csr, B


def _budget(sysg, es, nb_outer, width):
    """Device bytes for two staging buffers of one outer block plus `width` columns."""
    stage = es * (-(-sysg.rows // 32) * 32) * nb_outer
    return 2 * stage + es * sysg.lda * width


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_host_build_equals_device_build(storage):
    need_cuda()
    import paper_2412_07631_b300 as ct
    geom = ct.make_geometry(NS, NV, NBINS, SL)
    dev = ct.System(geom, storage)
    es = 8 if storage == "fp64" else 4
    host = ct.System(geom, storage, host_budget=es * dev.lda * 100)  # 6 slabs of 100 columns
    a, b = dev.export_dense(), host.export_dense()
    assert a.dtype == b.dtype
    np.testing.assert_array_equal(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("tf32", 1e-6),
                                           ("bf16", 1e-6)])
def test_ooc_factor_matches_oracle(oracle_mod, precision, tol):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, B = _case(O)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    storage = "fp64" if precision == "fp64" else "fp32"
    es = 8 if storage == "fp64" else 4
    geom = ct.make_geometry(NS, NV, NBINS, SL)
    probe = ct.System(geom, storage)
    budget = _budget(probe, es, 64, 128)  # superpanels of 128 columns: 5 of them
    probe.free()
    sysg = ct.System(geom, storage, host_budget=budget)
    F = sysg.factor_ooc(precision, device_budget=budget, nb_outer=64)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda()
    Xg = F.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).double().cpu().numpy().T
    err = rel_err_cols(Xg, Xo)
    print(precision, "ooc max rel err", err.max(), F.last_info)
    assert err.max() <= tol


@pytest.mark.gpu
def test_ooc_fp64_factor_equals_in_core():
    """Same blocks, same reflectors: the out-of-core FP64 factors (V below
    the diagonal, R above) agree with the in-core ones to rounding."""
    need_cuda()
    import paper_2412_07631_b300 as ct
    geom = ct.make_geometry(NS, NV, NBINS, SL)
    incore = ct.System(geom, "fp64")
    Fi = incore.factor("fp64", nb_outer=64)
    VRi, taui = Fi.export()
    budget = _budget(incore, 8, 64, 192)
    host = ct.System(geom, "fp64", host_budget=budget)
    Fo = host.factor_ooc("fp64", device_budget=budget, nb_outer=64)
    VRo, tauo = Fo.export()
    scale = np.abs(VRi).max()
    assert np.abs(VRo - VRi).max() <= 1e-12 * scale
    assert np.abs(tauo - taui).max() <= 1e-12


@pytest.mark.gpu
def test_ooc_budget_too_small_is_refused():
    need_cuda()
    import paper_2412_07631_b300 as ct
    geom = ct.make_geometry(NS, NV, NBINS, SL)
    host = ct.System(geom, "fp32", host_budget=1 << 20)
    with pytest.raises(ct.CTQRError):
        host.factor_ooc("tf32", device_budget=1 << 16, nb_outer=64)
    # the system keeps its host matrix after the refusal
    F = host.factor_ooc("tf32", device_budget=64 << 20, nb_outer=64)
    assert F.n == NS * NS


@pytest.mark.gpu
def test_ooc_factor_checkpoint_loads_in_core(oracle_mod, tmp_path):
    """An out-of-core factor written with save() loads as an in-core factor
    of a device-built system and solves to the same bits."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, B = _case(O)
    geom = ct.make_geometry(NS, NV, NBINS, SL)
    probe = ct.System(geom, "fp64")
    budget = _budget(probe, 8, 64, 128)
    probe.free()
    host = ct.System(geom, "fp64", host_budget=budget)
    Fo = host.factor_ooc("fp64", device_budget=budget, nb_outer=64)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    x1 = Fo.solve(Bt).clone()
    path = str(tmp_path / "ooc.ctqr")
    Fo.save(path)
    dev = ct.System(geom, "fp64")
    Fi = ct.Factor.load(dev, path)
    x2 = Fi.solve(Bt)
    assert torch.allclose(x1, x2, rtol=0, atol=1e-12 * float(x1.abs().max()))
