"""The solve plan: the blocking of the batched solve (superblock rows of the
triangular solve, least split-K depth of the solve's GEMMs), chosen by the
caller or by autotune.solve_plan.  Every plan must give the same solution up
to the factor's rounding, and refined solves are certified against the exact
least-squares solution."""
import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth



@pytest.mark.gpu
def test_solve_plans_agree_and_certify(oracle_mod):
    """The solve plan (superblock rows of the triangular solve, least split-K
    depth of the solve's GEMMs) changes only the blocking: on a 64x64 image
    (4,096 unknowns, so several superblocks) with TF32 factors, every plan's
    direct (unrefined) solve is as close to the certified least-squares
    solution as the default plan's, up to the TF32 rounding of a different
    summation order (a wrong block would be off by O(1)), and every plan's
    refined solve is certified against the exact least-squares solution (the
    oracle's long-double bound) to 1e-6.  Invalid plans are refused."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(64, 90, 92, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    B = synth.poisson_sinogram(O.forward(csr, synth.phantom_batch(64, 16, 10)), 64, 1e4, seed=3)
    sysg = ct.System(ct.make_geometry(64, 90, 92, 0.05), "fp32")
    F = sysg.factor("tf32")
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    F.solve_plan = (0, 0)
    Xref = F.solve(Bt, max_iter=30, tol=1e-9).cpu().numpy().T
    assert O.certificate(g, csr, B, Xref).max() <= 1e-8
    e0 = rel_err_cols(F.solve(Bt, max_iter=-1).cpu().numpy().T, Xref).max()
    for plan in [(512, 256), (1024, 64), (4096, 1024), (128, 32), (0, 0)]:
        F.solve_plan = plan
        Xd = F.solve(Bt, max_iter=-1).cpu().numpy().T
        e = rel_err_cols(Xd, Xref).max()
        print(plan, "direct error", e, "default", e0)
        assert e <= 3 * e0 + 1e-3, (plan, e, e0)
        Xr = F.solve(Bt, max_iter=30, tol=1e-9).cpu().numpy().T
        cert = O.certificate(g, csr, B, Xr)
        assert cert.max() <= 1e-6, (plan, cert.max())
    for bad in [(100, 0), (384, 0), (0, 33), (32768, 0)]:
        F.solve_plan = bad
        with pytest.raises(ct.CTQRError) as ei:
            F.solve(Bt, max_iter=-1)
        assert ei.value.name == "CT_ERR_ARG", bad

