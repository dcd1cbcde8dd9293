"""Edge cases of the path against the oracle: empty batches, all-zero
sinograms (exactly zero images, also inside a noisy batch), single slices
and slice counts that are not multiples of the vector width (the scalar
sparse-product kernels), and degenerate geometries down to one pixel."""
import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth

PREC = [("fp64", 1e-10), ("fp32", 1e-4), ("tf32", 1e-6), ("bf16", 1e-6)]


def _system(ct, O, ns, nv, nb, sl, precision):
    g = O.Geometry(ns, nv, nb, sqrt_lambda=sl)
    storage = "fp64" if precision == "fp64" else "fp32"
    sysg = ct.System(ct.make_geometry(ns, nv, nb, sl), storage)
    return g, sysg, sysg.factor(precision)


def _dtype(torch, precision):
    return torch.float32 if precision == "fp32" else torch.float64


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_zero_slices(oracle_mod, precision):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    g, sysg, F = _system(ct, oracle_mod, 12, 18, 18, 0.05, precision)
    dt = _dtype(torch, precision)
    X = F.solve(torch.empty((0, sysg.m), dtype=dt, device="cuda"))
    assert tuple(X.shape) == (0, sysg.n)
    gB = F.adjoint(torch.empty((0, sysg.n), dtype=dt, device="cuda"))
    assert tuple(gB.shape) == (0, sysg.m)
    Xh = F.solve_host(torch.empty((0, sysg.m), dtype=dt))
    assert tuple(Xh.shape) == (0, sysg.n)
    P = sysg.forward(torch.empty((0, sysg.n), dtype=torch.float64, device="cuda"))
    assert tuple(P.shape) == (0, sysg.m)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", PREC)
def test_zero_sinograms_give_zero_images(oracle_mod, precision, tol):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, sysg, F = _system(ct, O, 16, 24, 24, 0.05, precision)
    dt = _dtype(torch, precision)
    X = F.solve(torch.zeros((3, sysg.m), dtype=dt, device="cuda"))
    assert torch.count_nonzero(X).item() == 0
    # one zero sinogram inside a noisy batch: its image stays exactly zero,
    # the others match the oracle
    csr = O.siddon_csr(g)
    B = synth.poisson_sinogram(O.forward(csr, synth.phantom_batch(16, 4, 8, 77)), 16, 1e4, seed=77)
    B[:, 2] = 0.0
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    Xg = F.solve(torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda(), max_iter=20, tol=1e-10,
                 allow_noconv=True).double().cpu().numpy().T
    assert np.count_nonzero(Xg[:, 2]) == 0
    keep = [0, 1, 3]
    assert rel_err_cols(Xg[:, keep], Xo[:, keep]).max() <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", PREC)
@pytest.mark.parametrize("k", [1, 7])
def test_odd_slice_counts(oracle_mod, precision, tol, k):
    """k = 1 and k = 7: not multiples of the 16-byte vector width, so the
    sparse products of the refinement take their scalar kernels."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, sysg, F = _system(ct, O, 19, 31, 29, 0.05, precision)
    csr = O.siddon_csr(g)
    B = synth.poisson_sinogram(O.forward(csr, synth.phantom_batch(19, k, 8, 91)), 19, 1e4, seed=91)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(_dtype(torch, precision)).cuda()
    Xg = F.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).double().cpu().numpy().T
    assert rel_err_cols(Xg, Xo).max() <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", PREC)
@pytest.mark.parametrize("ns,nv,nb,sl", [(1, 3, 4, 0.0), (1, 3, 4, 0.05), (2, 3, 4, 0.05), (3, 5, 6, 0.0),
                                         (5, 7, 8, 0.05)])
def test_degenerate_geometries(oracle_mod, precision, tol, ns, nv, nb, sl):
    """Images of 1 to 25 pixels: one panel narrower than a warp, the whole
    factor inside one tile, the triangular solve inside one diagonal block."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, sysg, F = _system(ct, O, ns, nv, nb, sl, precision)
    csr = O.siddon_csr(g)
    rng = np.random.default_rng(ns * 100 + nv)
    X = rng.uniform(0.0, 1.0, (g.n, 3))
    B = O.forward(csr, X) + 0.01 * rng.standard_normal((g.m, 3))
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(_dtype(torch, precision)).cuda()
    Xg = F.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).double().cpu().numpy().T
    assert np.all(np.isfinite(Xg))
    assert rel_err_cols(Xg, Xo).max() <= tol
