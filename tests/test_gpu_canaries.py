"""Sanitizer substitute: guard bands past the capacity of every library
scratch buffer (ct_debug_canaries).  The whole path runs at ragged sizes in
every precision with the bands on -- build, in-core and out-of-core
factorisation, refined and direct solves, adjoints, the GEMM engine with
every kind and transposition -- and no band may change: no kernel writes
past the end of its scratch.  The check itself is shown to fire on a band
overwritten from the host (inside the buffer's allocation; nothing faults)."""
import numpy as np
import pytest

from gpu_util import need_cuda


@pytest.mark.gpu
def test_no_kernel_writes_past_its_scratch():
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    ct.debug_canaries(True)
    seen = [0, 0]

    def check():  # the bands of every live buffer, while the factors exist
        checked, corrupted = ct.debug_check_canaries()
        seen[0] += checked
        seen[1] += corrupted

    try:
        rng = np.random.default_rng(4)
        for ns, nv, nb, sl in ((13, 21, 19, 0.05), (24, 40, 36, 0.05), (9, 30, 14, 0.0)):
            for storage, prec in (("fp64", "fp64"), ("fp32", "fp32"), ("fp32", "tf32"), ("fp32", "bf16"),
                                  ("fp32", "bf16x3")):
                geom = ct.make_geometry(ns, nv, nb, sl)
                sysg = ct.System(geom, storage)
                F = sysg.factor(prec, nb_outer=64)
                dt = torch.float32 if prec == "fp32" else torch.float64
                B = torch.from_numpy(rng.standard_normal((5, sysg.m))).to(dt).cuda()
                X = F.solve(B, max_iter=8, tol=1e-9, allow_noconv=True)
                F.adjoint(torch.ones_like(X), max_iter=8, tol=1e-9, allow_noconv=True)
                check()
                F.free()
                sysg.free()
            hs = ct.System(ct.make_geometry(ns, nv, nb, sl), "fp32", host_budget=1 << 22)
            Fo = hs.factor_ooc("bf16", device_budget=1 << 22, nb_outer=64)
            Fo.solve(torch.ones((3, hs.m), dtype=torch.float64, device="cuda"), max_iter=8, tol=1e-9,
                     allow_noconv=True)
            check()
            Fo.free()
            hs.free()
        for kind in ("fp64", "fp32", "tf32", "bf16", "tf32x3", "bf16x3"):
            dt = torch.float64 if kind == "fp64" else torch.float32
            for ta in "NT":
                for tb in "NT":
                    M, N, K = 133, 301, 517
                    ra, ca = (K, M) if ta == "T" else (M, K)
                    rb, cb = (N, K) if tb == "T" else (K, N)
                    lda, ldb = -(-ra // 32) * 32, -(-rb // 32) * 32
                    A = torch.rand((ca, lda), dtype=dt, device="cuda")
                    Bm = torch.rand((cb, ldb), dtype=dt, device="cuda")
                    Cm = torch.rand((N, M), dtype=dt, device="cuda")
                    ct.gemm(kind, ta, tb, M, N, K, 1.0, A, lda, Bm, ldb, 0.5, Cm, M)
        check()
        # every case held several banded buffers (GEMM copies, workspaces)
        assert seen[0] >= 30 and seen[1] == 0, seen
        # the check fires on a band overwritten from the host
        checked, corrupted = ct.debug_check_canaries(corrupt_first=True)
        assert corrupted == 1, (checked, corrupted)
    finally:
        ct.debug_canaries(False)
