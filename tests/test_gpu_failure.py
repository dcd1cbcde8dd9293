"""Failure detection on the GPU without a fault.

* A device-side wait that cannot complete (the panel kernels' grid meet on a
  grid missing a CTA) gives up after its time limit, the library reports
  CT_ERR_TIMEOUT with the site at the next synchronisation point, and the
  context stays usable: the status word is clear and the next factorisation
  and solve match the oracle.
* A numerically rank-deficient system (one view of a 4 x 4 image: rank 4 of
  16, R with exact zeros on its diagonal) is reported as CT_ERR_RANK by the
  |R_jj| >= n u max|R_jj| test, with the factor kept for inspection.
* Refinement stopped short of its tolerance returns CT_ERR_NOCONV with the
  best iterate written and its stopping measure reported.  The same factor
  then solves normally.
* Non-finite data is reported, not turned into a silently wrong image: a NaN
  written into A~ (through the system's device pointer) before the
  factorisation gives CT_ERR_NONFINITE from ct_qr_factor, and a NaN in a
  sinogram (or in the gradient fed to the adjoint) gives CT_ERR_NONFINITE
  from the direct FP64/FP32 solves and from the refining ones.  The NaNs are
  written from the host; nothing faults."""
import time

import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth


@pytest.mark.gpu
def test_stalled_wait_surfaces_as_timeout(oracle_mod):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert ct.selftest_wait_timeout() == "CT_ERR_TIMEOUT"
    waited = time.perf_counter() - t0
    assert 3.5 <= waited <= 60.0, waited
    assert "site 90" in ct.lib().ct_last_error().decode()

    g = O.Geometry(16, 24, 24, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    B = synth.poisson_sinogram(O.forward(csr, synth.phantom_batch(16, 3, 8, 5)), 16, 1e4, seed=5)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    sysg = ct.System(ct.make_geometry(16, 24, 24, 0.05), "fp32")
    F = sysg.factor("tf32")
    Xg = F.solve(torch.from_numpy(np.ascontiguousarray(B.T)).cuda(), max_iter=20,
                 tol=1e-10).cpu().numpy().T
    assert rel_err_cols(Xg, Xo).max() <= 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("storage,precision", [("fp64", "fp64"), ("fp32", "fp32"), ("fp32", "tf32")])
def test_rank_deficient_system_is_reported(storage, precision):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    # one view at 0 degrees, 20 bins: the rays through the four pixel columns
    # each cover one column of the image, so A has four distinct rows
    sysg = ct.System(ct.make_geometry(4, 1, 20), storage)
    with pytest.raises(ct.CTQRError) as ei:
        sysg.factor(precision)
    assert ei.value.name == "CT_ERR_RANK", str(ei.value)
    assert "rank deficient" in str(ei.value)
    assert ei.value.factor.h
    ei.value.factor.free()
    sysg.free()
    # the context is unaffected: a full-rank system factors and solves
    sysg = ct.System(ct.make_geometry(4, 6, 8, 0.05), storage)
    F = sysg.factor(precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    X = F.solve(torch.ones((1, sysg.m), dtype=dt, device="cuda"), max_iter=20, tol=1e-10,
                allow_noconv=True)
    assert torch.isfinite(X).all()


@pytest.mark.gpu
def test_refinement_short_of_tolerance_reports_noconv(oracle_mod):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(12, 20, 18, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    B = synth.poisson_sinogram(O.forward(csr, synth.phantom_batch(12, 2, 6, 9)), 12, 1e4, seed=9)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    sysg = ct.System(ct.make_geometry(12, 20, 18, 0.05), "fp32")
    F = sysg.factor("tf32")
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    with pytest.raises(ct.CTQRError) as ei:
        F.solve(Bt, max_iter=1, tol=1e-300)
    assert ei.value.name == "CT_ERR_NOCONV"
    X1 = F.solve(Bt, max_iter=1, tol=1e-300, allow_noconv=True)
    assert F.last_info["iterations"] == 1
    assert 1e-300 < F.last_info["stop_measure"] < 1.0
    assert torch.isfinite(X1).all()
    gX = torch.from_numpy(np.random.default_rng(2).standard_normal((2, sysg.n))).cuda()
    with pytest.raises(ct.CTQRError) as ei:
        F.adjoint(gX, max_iter=1, tol=1e-300)
    assert ei.value.name == "CT_ERR_NOCONV"
    # the factor and the context are intact
    Xg = F.solve(Bt, max_iter=20, tol=1e-10).cpu().numpy().T
    assert rel_err_cols(Xg, Xo).max() <= 1e-6


class _DeviceView:
    """One element of device memory at a raw address, as a torch tensor (CUDA
    array interface), so a test can write into library-owned storage."""

    def __init__(self, ptr, typestr):
        self.__cuda_array_interface__ = {"shape": (1,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


@pytest.mark.gpu
@pytest.mark.parametrize("storage,precision", [("fp64", "fp64"), ("fp32", "fp32"), ("fp32", "tf32"),
                                               ("fp32", "bf16")])
def test_nonfinite_matrix_is_reported(storage, precision):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    sysg = ct.System(ct.make_geometry(12, 20, 18, 0.05), storage)
    es, ts = (8, "<f8") if storage == "fp64" else (4, "<f4")
    ptr = ct.system_device_ptrs(sysg)["dense"] + es * (40 + 70 * sysg.lda)  # row 40 of column 70
    torch.as_tensor(_DeviceView(ptr, ts), device="cuda").fill_(float("nan"))
    torch.cuda.synchronize()
    with pytest.raises(ct.CTQRError) as ei:
        sysg.factor(precision)
    assert ei.value.name == "CT_ERR_NONFINITE", str(ei.value)
    sysg.free()
    # the context is unaffected
    sysg = ct.System(ct.make_geometry(12, 20, 18, 0.05), storage)
    F = sysg.factor(precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    assert torch.isfinite(F.solve(torch.ones((1, sysg.m), dtype=dt, device="cuda"), max_iter=20,
                                  tol=1e-10, allow_noconv=True)).all()


@pytest.mark.gpu
@pytest.mark.parametrize("storage,precision", [("fp64", "fp64"), ("fp32", "fp32"), ("fp32", "tf32")])
def test_nonfinite_sinogram_or_gradient_is_reported(oracle_mod, storage, precision):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(12, 20, 18, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    B = synth.poisson_sinogram(O.forward(csr, synth.phantom_batch(12, 3, 6, 9)), 12, 1e4, seed=9)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    sysg = ct.System(ct.make_geometry(12, 20, 18, 0.05), storage)
    F = sysg.factor(precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda()
    Bn = Bt.clone()
    Bn[1, 5] = float("nan")
    with pytest.raises(ct.CTQRError) as ei:
        F.solve(Bn, max_iter=20, tol=1e-10)
    assert ei.value.name == "CT_ERR_NONFINITE", str(ei.value)
    Bn[1, 5] = float("inf")
    with pytest.raises(ct.CTQRError) as ei:
        F.solve(Bn, max_iter=20, tol=1e-10, allow_noconv=True)
    assert ei.value.name == "CT_ERR_NONFINITE"
    gX = torch.zeros((2, sysg.n), dtype=dt, device="cuda")
    gX[0, 7] = float("nan")
    with pytest.raises(ct.CTQRError) as ei:
        F.adjoint(gX, max_iter=20, tol=1e-10)
    assert ei.value.name == "CT_ERR_NONFINITE"
    # the factor and the context are intact
    tol = {"fp64": 1e-10, "fp32": 1e-4, "tf32": 1e-6}[precision]
    Xg = F.solve(Bt, max_iter=20, tol=1e-10).cpu().numpy().T
    assert rel_err_cols(Xg, Xo).max() <= tol
