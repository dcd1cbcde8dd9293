"""Failure detection on the GPU without a fault: a device-side wait that
cannot complete (the panel kernels' grid meet on a grid missing a CTA) gives
up after its time limit, the library reports CT_ERR_TIMEOUT with the site at
the next synchronisation point, and the context stays usable: the status
word is clear and the next factorisation and solve match the oracle."""
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
