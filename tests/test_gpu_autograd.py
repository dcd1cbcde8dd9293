"""Differentiation through the reconstruction (not in the paper; the solve
used as a layer of a trained model): the solve as a torch.autograd.Function
whose backward pass is the hand-written adjoint grad_b = [Q R^-T grad_x]_{0:m},
refined in FP64 for the TF32 factors.  Loss = mean squared error to the
phantom.  Checks: central finite differences (h = 1e-3, FP64; the loss is
quadratic in b, so the central difference is exact up to rounding) <= 1e-4
relative; an FP64 reference gradient from the oracle (Q R^-T applied by the
plain Householder route) <= 1e-6; the adjoint identity
<solve(b), y> = <b, adjoint(y)>."""
import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth


def _setup(O, ns, nv, nb, sl, k, torch, ct, precision="tf32"):
    g = O.Geometry(ns, nv, nb, sqrt_lambda=sl)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(ns, k, 8)
    B = synth.poisson_sinogram(O.forward(csr, X), ns, 1e4, seed=17)
    sysg = ct.System(ct.make_geometry(ns, nv, nb, sl), "fp64" if precision == "fp64" else "fp32")
    F = sysg.factor(precision)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    return g, csr, X, B, sysg, F, Bt, Xt


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32", "fp64"])
def test_gradient_matches_oracle_and_finite_differences(oracle_mod, precision):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, X, B, sysg, F, Bt, Xt = _setup(O, 24, 40, 36, 0.05, 3, torch, ct, precision)
    it, tol = 60, 1e-11
    Bv = Bt.clone().requires_grad_(True)
    Xr = ct.CTSolve.apply(Bv, F, it, tol)
    loss = ((Xr - Xt) ** 2).mean()
    loss.backward()
    grad = Bv.grad.cpu().numpy().T  # (m x k)
    # FP64 reference: dL/dx = 2 (x - x_phantom) / (n k); grad_b = [Q R^-T dL/dx]_{0:m}
    Xo, VR, tau = O.qr_solve(g, O.dense_system(g, csr), B)
    gx = 2.0 * (Xo - X) / Xo.size
    z = O.forwardsolve_rt(VR, gx)
    full = np.zeros((g.rows, gx.shape[1]), order="F")
    full[: g.n] = z
    ref = O.apply_q(VR, tau, full)[: g.m]
    rel = np.linalg.norm(grad - ref) / np.linalg.norm(ref)
    print(precision, "gradient vs oracle", rel, F.last_info)
    assert rel <= 1e-6
    # central finite differences along random unit directions
    rng = np.random.default_rng(5)
    with torch.no_grad():
        for _ in range(4):
            d = rng.standard_normal(B.T.shape)
            d /= np.linalg.norm(d)
            dt = torch.from_numpy(d).cuda()
            h = 1e-3
            lp = ((F.solve(Bt + h * dt, max_iter=it, tol=tol) - Xt) ** 2).mean().item()
            lm = ((F.solve(Bt - h * dt, max_iter=it, tol=tol) - Xt) ** 2).mean().item()
            fd = (lp - lm) / (2 * h)
            an = float(np.sum(grad.T * d))
            assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-12), (fd, an)


@pytest.mark.gpu
def test_adjoint_identity_refined_tf32(oracle_mod):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    sysg = ct.System(ct.make_geometry(24, 40, 36, 0.05), "fp32")
    F = sysg.factor("tf32")
    rng = np.random.default_rng(1)
    b = torch.from_numpy(rng.standard_normal((3, sysg.m))).cuda()
    y = torch.from_numpy(rng.standard_normal((3, sysg.n))).cuda()
    x = F.solve(b, max_iter=60, tol=1e-11)
    gb = F.adjoint(y, max_iter=60, tol=1e-11)
    lhs = (x * y).sum(1).cpu().numpy()
    rhs = (b * gb).sum(1).cpu().numpy()
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9)


def _c4_inputs(O):
    ns, nv, nb, sl, k = 128, 180, 182, 0.05, 256
    g = O.Geometry(ns, nv, nb, sqrt_lambda=sl)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(ns, k, 10)
    B = synth.poisson_sinogram(O.forward(csr, X), ns, 1e4, seed=23)
    return g, csr, X, B


@pytest.mark.gpu
def test_c4_workload_gradient_matches_oracle(oracle_mod):
    """128 x 128 geometry (the differentiation config), 256 noisy sinograms
    through the autograd layer with TF32 factors and FP64 refinement.  On
    the sampled slices the images must equal the oracle's least-squares
    solution and grad_b the oracle's FP64 gradient (LAPACK route: dgeqrf,
    then R^-T and Q applied in reverse order of the forward solve, stored in
    tests/golden/c4_grad.npz by make_c4_gradient.py) within 1e-6 relative per
    slice; the refined backward pass must reach its certified stop; and
    <grad_b, d> must match central finite differences of the loss along two
    random directions."""
    import hashlib
    import os
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "c4_grad.npz"))
    g, csr, X, B = _c4_inputs(O)
    assert hashlib.sha256(np.ascontiguousarray(B).tobytes()).hexdigest() == str(ref["b_sha256"])
    sysg = ct.System(ct.make_geometry(128, 180, 182, 0.05), "fp32")
    F = sysg.factor("tf32")
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    it, tol = 60, 1e-9
    Bv = Bt.clone().requires_grad_(True)
    Xr = ct.CTSolve.apply(Bv, F, it, tol)
    loss = ((Xr - Xt) ** 2).mean()
    loss.backward()
    print("c4 backward info", F.last_info)
    grad = Bv.grad
    assert F.last_info["stop_measure"] <= tol
    S = [int(v) for v in ref["slices"]]
    x_err = rel_err_cols(Xr.detach()[S].cpu().numpy().T, ref["xref"])
    g_err = rel_err_cols(grad[S].cpu().numpy().T, ref["grad_b"])
    print("c4 image error", x_err, "gradient error", g_err)
    assert np.all(x_err <= 1e-6)
    assert np.all(g_err <= 1e-6)
    rng = np.random.default_rng(9)
    with torch.no_grad():
        for _ in range(2):
            d = torch.from_numpy(rng.standard_normal(Bt.shape)).cuda()
            d /= d.norm()
            h = 1e-3
            lp = ((F.solve(Bt + h * d, max_iter=it, tol=tol) - Xt) ** 2).mean().item()
            lm = ((F.solve(Bt - h * d, max_iter=it, tol=tol) - Xt) ** 2).mean().item()
            fd = (lp - lm) / (2 * h)
            an = float((grad * d).sum())
            assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-12), (fd, an)
