"""The 256x256 workload at full size, in the benchmark's launch
configuration: 360 views x 364 bins + sqrt(lambda) = 0.05 I rows
(M' = 196,576, n = 65,536), 512 noisy sinograms in one batch, BF16 trailing
updates, FP64 refinement; with the library's default blocking and with the
blockings the benchmark's tuner chooses among (outer blocks of 2560 and
3072, triangular-solve superblocks of 4096 rows, split-K depth >= 1024).

A dense FP64 oracle solve of this size does not fit on the host, so the
result is checked on sampled slices through facts that hold at any size,
computed by the oracle alone from its own Siddon matrix:
  * the forward projections that make the sinograms equal the oracle's;
  * the certified bound ||x - x*|| / ||x|| <= ||A~^T (b~ - A~ x)|| / (lambda ||x||)
    (every singular value of A~ is >= sqrt(lambda)), with the residual
    accumulated in long double, is <= 1e-6 for every sampled slice, and no
    larger than the stopping measure the library reported for the batch.
"""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2412_07631_b300 import synth

NS, NV, NB, SL, K, I0, NE = 256, 360, 364, 0.05, 512, 5e3, 10
PICK = [0, 1, 170, 341, 511]


@pytest.fixture(scope="module")
def full_size_inputs(oracle_mod):
    """The oracle's Siddon matrix, the phantoms, and the sinograms from the
    library's forward projection (checked against the oracle's on the
    sampled slices)."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(NS, NV, NB, sqrt_lambda=SL)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(NS, K, NE, synth.BASE_SEED)  # (n, k)
    sysg = ct.System(ct.make_geometry(NS, NV, NB, SL), "fp32")
    Pg = sysg.forward(torch.from_numpy(np.ascontiguousarray(X.T)).cuda()).cpu().numpy().T  # (m, k)
    sysg.free()
    Po = O.forward(csr, X[:, PICK])
    np.testing.assert_allclose(Pg[:, PICK], Po, rtol=1e-13, atol=1e-11)
    B = synth.poisson_sinogram(Pg, NS, I0, seed=synth.BASE_SEED)  # (m, k)
    return g, csr, B


@pytest.mark.gpu
@pytest.mark.parametrize("nb_outer,plan", [(0, (0, 0)), (2560, (4096, 1024)), (3072, (4096, 1024))])
def test_256_bf16_batch_is_certified_by_the_oracle(oracle_mod, full_size_inputs, nb_outer, plan):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, B = full_size_inputs
    sysg = ct.System(ct.make_geometry(NS, NV, NB, SL), "fp32")
    F = sysg.factor("bf16", nb_outer=nb_outer)
    F.solve_plan = plan
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xg = F.solve(Bt, max_iter=10, tol=1e-7).cpu().numpy()  # (k, n)
    info = F.last_info
    F.free()
    sysg.free()

    cert = O.certificate(g, csr, np.asfortranarray(B[:, PICK]), np.asfortranarray(Xg[PICK].T))
    print(nb_outer, plan, "iterations", info, "oracle certificate on sampled slices", cert)
    assert np.all(np.isfinite(Xg))
    assert cert.max() <= 1e-6
    assert info["stop_measure"] <= 1e-7
    # the library's FP64 stopping measure is the max over the batch of the
    # same bound: the oracle's value for any slice cannot exceed it (beyond
    # the rounding of an FP64 against a long-double residual)
    assert cert.max() <= info["stop_measure"] * (1 + 1e-3) + 1e-12
