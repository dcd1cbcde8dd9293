"""ct_gemm_noalloc -- the GEMM engine for callers that cannot allocate device
memory (their device memory is all in their own pool, or they must not
allocate at run time) -- gives the results of ct_gemm on the same operands.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.  Passes alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import need_cuda

CASES = [  # kind, ta, tb, M, N, K: split-K partials in the array; K-major copies in the array
    ("tf32", "T", "N", 64, 96, 40000),
    ("tf32", "N", "N", 300, 520, 1000),
    ("fp32", "T", "N", 48, 40, 30000),
    # ct_gemm's plan splits K ten ways (40 MiB of partials): the depth is cut to
    # what fits in the 16 MiB array
    ("tf32", "T", "N", 1024, 1024, 16384),
]


def _operands(rng, kind, ta, tb, M, N, K):
    """Column-major storage (torch row = matrix column) and the logical
    op(A) (M x K), op(B) (K x N) in float64."""
    ra, ca = (K, M) if ta == "T" else (M, K)
    rb, cb = (N, K) if tb == "T" else (K, N)
    lda, ldb, ldc = -(-ra // 4) * 4, -(-rb // 4) * 4, M
    A = rng.uniform(-1, 1, (ca, lda)).astype(np.float32)
    B = rng.uniform(-1, 1, (cb, ldb)).astype(np.float32)
    C = rng.uniform(-1, 1, (N, ldc)).astype(np.float32)
    if kind == "tf32":
        A = (A.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
        B = (B.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    Amat = A[:, :ra].T.astype(np.float64)
    Bmat = B[:, :rb].T.astype(np.float64)
    opA = Amat.T if ta == "T" else Amat
    opB = Bmat.T if tb == "T" else Bmat
    return A, B, C, lda, ldb, ldc, opA, opB


@pytest.mark.gpu
def test_noalloc_gemm_matches_ct_gemm_twice_in_a_row():
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    rng = np.random.default_rng(11)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    alpha, beta = 0.75, -0.5
    for rep in range(2):
        for kind, ta, tb, M, N, K in CASES:
            A, B, C, lda, ldb, ldc, opA, opB = _operands(rng, kind, ta, tb, M, N, K)
            dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            c_ref, c_new = torch.from_numpy(C).cuda(), torch.from_numpy(C).cuda()
            args = (ct.GEMM_KINDS[kind], ta.encode(), tb.encode(), M, N, K, alpha,
                    ctypes.c_void_p(dA.data_ptr()), lda, ctypes.c_void_p(dB.data_ptr()), ldb, beta)
            assert L.ct_gemm(*args, ctypes.c_void_p(c_ref.data_ptr()), ldc, stream) == 0
            st = L.ct_gemm_noalloc(*args, ctypes.c_void_p(c_new.data_ptr()), ldc, stream)
            assert st == 0, L.ct_last_error()
            torch.cuda.synchronize()
            got_ref = c_ref.cpu().numpy()[:, :M].T.astype(np.float64)
            got_new = c_new.cpu().numpy()[:, :M].T.astype(np.float64)
            c0 = C[:, :M].T.astype(np.float64)
            exact = alpha * opA @ opB + beta * c0
            scale = abs(alpha) * np.abs(opA) @ np.abs(opB) + abs(beta) * np.abs(c0)
            tol = 4 * (K + 2) * 2.0 ** -23 * scale
            assert np.all(np.abs(got_ref - exact) <= tol)
            assert np.all(np.abs(got_new - exact) <= tol), (rep, kind, ta, tb)
            assert np.all(np.abs(got_new - got_ref) <= 2 * tol)


@pytest.mark.gpu
def test_noalloc_gemm_allocates_no_device_memory():
    """Free device memory (cudaMemGetInfo) does not move across calls of the
    allocation-free entry point.  Around the first call on the device it may
    drop by the fixed array itself, which the driver places when it first
    loads the array's module; nothing beyond that."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(3)
    ops = []
    for kind, ta, tb, M, N, K in CASES:
        A, B, C, lda, ldb, ldc, _, _ = _operands(rng, kind, ta, tb, M, N, K)
        dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
        args = (ct.GEMM_KINDS[kind], ta.encode(), tb.encode(), M, N, K, 1.0,
                ctypes.c_void_p(dA.data_ptr()), lda, ctypes.c_void_p(dB.data_ptr()), ldb, 0.5,
                ctypes.c_void_p(dC.data_ptr()), ldc, stream)
        ops.append((args, dA, dB, dC))
        assert L.ct_gemm(*args) == 0  # loads every kernel the products use
    torch.cuda.synchronize()

    def free_bytes():
        torch.cuda.synchronize()
        return torch.cuda.mem_get_info()[0]

    f0 = free_bytes()
    assert L.ct_gemm_noalloc(*ops[0][0]) == 0, L.ct_last_error()
    f1 = free_bytes()
    assert 0 <= f0 - f1 <= (16 << 20) + (4 << 20), (f0, f1)
    for _ in range(2):
        for args, *_ in ops:
            assert L.ct_gemm_noalloc(*args) == 0, L.ct_last_error()
    assert free_bytes() == f1


@pytest.mark.gpu
def test_noalloc_refuses_bf16_and_split_kinds():
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    d = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kind in ("bf16", "tf32x3", "bf16x3"):
        st = L.ct_gemm_noalloc(ct.GEMM_KINDS[kind], b"T", b"N", 64, 64, 64, 1.0, p, 64, p, 64, 0.0,
                               p, 64, stream)
        assert st == 1, kind


@pytest.mark.gpu
def test_noalloc_refuses_oversized_copies_with_a_clear_error():
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    M, N, K = 8192, 256, 1024  # an 'N' operand of 8192 x 1024 floats needs 32 MiB of copies
    dA = torch.zeros((K, M), dtype=torch.float32, device="cuda")
    dB = torch.zeros((N, K), dtype=torch.float32, device="cuda")
    dC = torch.zeros((N, M), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.ct_gemm_noalloc(ct.GEMM_KINDS["tf32"], b"N", b"N", M, N, K, 1.0,
                           ctypes.c_void_p(dA.data_ptr()), M, ctypes.c_void_p(dB.data_ptr()), K,
                           0.0, ctypes.c_void_p(dC.data_ptr()), M, stream)
    assert st == 1
    assert b"fixed limit" in L.ct_last_error()
