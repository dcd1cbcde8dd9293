"""GEMM engine behind the WY updates and the Q^T application (tcgen05 TF32
and BF16 tensor cores; CUDA-core FP32/FP64) against a float64 matmul of the
same operands.  Tensor-core operands are pre-rounded to TF32 (truncation, as
the hardware reads FP32) or BF16 (nearest even, as the engine converts), so
the products are exact and only FP32 accumulation error remains.  beta = 0
and beta = 1 select the TMA store and reduce-add epilogues when C is 16-byte
aligned; other values the thread epilogue."""
import numpy as np
import pytest

from gpu_util import need_cuda

SHAPES = [(128, 256, 64), (300, 520, 1000), (64, 96, 40000), (1, 1, 1), (513, 257, 33),
          (256, 512, 4096)]


def tf32_round(a):
    b = a.astype(np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def bf16_round(a):
    u = a.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


CASES = ([(k, b) for k in ("tf32", "bf16") for b in (-0.5, 0.0, 1.0)] +
         [("fp32", -0.5), ("fp64", -0.5)])


@pytest.mark.gpu
@pytest.mark.parametrize("kind,beta", CASES)
@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_matches_float64(kind, beta, ta, tb, M, N, K):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    dt = np.float64 if kind == "fp64" else np.float32
    pad = 4
    # logical op(A) is M x K, op(B) is K x N; storage is column-major
    ra, ca = (K, M) if ta == "T" else (M, K)
    rb, cb = (N, K) if tb == "T" else (K, N)
    lda, ldb, ldc = -(-ra // 4) * 4 + pad, -(-rb // 4) * 4 + pad, M + pad
    A = rng.uniform(-1, 1, (ca, lda)).astype(dt)   # torch row (ca, lda) = col-major (lda x ca)
    B = rng.uniform(-1, 1, (cb, ldb)).astype(dt)
    Cm = rng.uniform(-1, 1, (N, ldc)).astype(dt)
    if kind == "tf32":
        A, B = tf32_round(A), tf32_round(B)
    elif kind == "bf16":
        A, B = bf16_round(A), bf16_round(B)
    Amat = A[:, :ra].T.astype(np.float64)  # stored matrix ra x ca
    Bmat = B[:, :rb].T.astype(np.float64)
    opA = Amat.T if ta == "T" else Amat
    opB = Bmat.T if tb == "T" else Bmat
    alpha = 0.75
    ref = alpha * opA @ opB + beta * Cm[:, :M].T.astype(np.float64)
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, Cm))
    ct.gemm(kind, ta, tb, M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()[:, :M].T.astype(np.float64)
    scale = np.abs(opA) @ np.abs(opB) * abs(alpha) + abs(beta) * np.abs(Cm[:, :M].T)
    eps = 2.0 ** -52 if kind == "fp64" else 2.0 ** -23
    tol = 4 * (K + 2) * eps * scale + 1e-300
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])
    # padding rows of C untouched
    np.testing.assert_array_equal(dC.cpu().numpy()[:, M:], Cm[:, M:])


PAIR_SHAPES = [(4000, 3000, 300), (1024, 1024, 8192), (2000, 2600, 1500)]


@pytest.mark.gpu
@pytest.mark.parametrize("kind,beta", [(k, b) for k in ("tf32", "bf16") for b in (-0.5, 0.0, 1.0)])
@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "T")])
@pytest.mark.parametrize("M,N,K", PAIR_SHAPES)
def test_gemm_pairs_match_float64(kind, beta, ta, tb, M, N, K):
    """Products with enough 256 x 256 tiles run on SM pairs (2-CTA
    clusters); ragged edges in both dimensions and a split-K case."""
    test_gemm_matches_float64(kind, beta, ta, tb, M, N, K)


def tf32_nearest(a):
    """Nearest TF32 value, ties away from zero (the split copies' rounding)."""
    u = a.astype(np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x1000) & 0xFFFFE000).astype(np.uint32)).view(np.float32)


def split3(a, kind):
    """(hi, lo) of the split-precision operand copies, as float64."""
    rnd = tf32_nearest if kind == "tf32x3" else bf16_round
    a32 = a.astype(np.float32)
    hi = rnd(a32)
    lo = rnd((a32 - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


SPLIT_SHAPES = [(128, 256, 64), (300, 520, 1000), (513, 257, 33), (64, 96, 20000), (2000, 2600, 1500)]


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("beta", [0.0, 1.0, -0.5])
@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("M,N,K", SPLIT_SHAPES)
def test_split_gemm_three_term_products(kind, beta, ta, tb, M, N, K):
    """Split-precision products equal A_hi B_hi + A_hi B_lo + A_lo B_hi of
    the rounded halves up to FP32 accumulation over 3K terms, and land far
    closer to the unrounded FP32 product than one TF32 or BF16 pass."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    rng = np.random.default_rng(M * 5 + N * 11 + K)
    ra, ca = (K, M) if ta == "T" else (M, K)
    rb, cb = (N, K) if tb == "T" else (K, N)
    lda, ldb, ldc = -(-ra // 4) * 4 + 4, -(-rb // 4) * 4 + 4, M + 4
    A = rng.uniform(-1, 1, (ca, lda)).astype(np.float32)
    B = rng.uniform(-1, 1, (cb, ldb)).astype(np.float32)
    Cm = rng.uniform(-1, 1, (N, ldc)).astype(np.float32)
    Amat, Bmat = A[:, :ra].T, B[:, :rb].T
    Ah, Al = split3(Amat, kind)
    Bh, Bl = split3(Bmat, kind)
    op = (lambda X, t: X.T if t == "T" else X)
    alpha = 0.75
    C0 = beta * Cm[:, :M].T.astype(np.float64)
    ref = alpha * (op(Ah, ta) @ op(Bh, tb) + op(Ah, ta) @ op(Bl, tb) + op(Al, ta) @ op(Bh, tb)) + C0
    exact = alpha * op(Amat.astype(np.float64), ta) @ op(Bmat.astype(np.float64), tb) + C0
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, Cm))
    ct.gemm(kind, ta, tb, M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()[:, :M].T.astype(np.float64)
    scale = np.abs(op(Amat, ta)).astype(np.float64) @ np.abs(op(Bmat, tb)).astype(np.float64) * alpha \
        + abs(beta) * np.abs(Cm[:, :M].T)
    acc = 4 * (3 * K + 2) * 2.0 ** -23 * scale
    assert (np.abs(got - ref) <= acc + 1e-300).all()
    # the dropped lo*lo term and the halves' rounding: 2^-20 (TF32x3), 2^-14 (BF16x3)
    drop = (2.0 ** -20 if kind == "tf32x3" else 2.0 ** -14) * scale
    assert (np.abs(got - exact) <= acc + drop).all()
    np.testing.assert_array_equal(dC.cpu().numpy()[:, M:], Cm[:, M:])
