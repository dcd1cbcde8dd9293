// gemm_simt.cu -- CUDA-core GEMM for the FP64 and FP32 paths, and the
// split-K reduction shared with the tensor-core engine.
//
// C = alpha * op(A) * op(B) + beta * C, column-major.  Block tile BM x BN
// (simt_tile.cuh); split-K over blockIdx.z.  FP64 on B300 runs at roughly 1/64 of the
// FP32 rate, so the FP64 instance is bound by the DFMA pipe, not by memory.
#include "common.cuh"
#include "kernels.cuh"
#include "simt_tile.cuh"

#include <algorithm>

namespace ctqr {

namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_simt_kernel(bool ta, bool tb, int64_t M, int64_t N,
                                                        int64_t K, int64_t kchunk, T alpha,
                                                        const T *__restrict__ A, int64_t lda,
                                                        const T *__restrict__ B, int64_t ldb,
                                                        T beta, T *C, int64_t ldc,
                                                        int64_t split_stride) {
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    simt_tile<T, BM, BN, BK, TM, TN>(ta, tb, M, N, kb, min(K, kb + kchunk), alpha, A, lda, B, ldb, beta,
                                     C + (int64_t)blockIdx.z * split_stride, ldc, (int64_t)blockIdx.x * BM,
                                     (int64_t)blockIdx.y * BN);
}

template <typename T>
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int splits, const T *P, T alpha, T beta,
                                     T *C, int64_t ldc) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    int64_t i = idx % M, j = idx / M;
    // the partials are summed in split order; loads are issued eight at a
    // time so that deep splits are not a chain of dependent loads
    const int64_t MN = M * N;
    const T *p = P + idx;
    T acc = T(0);
    int z = 0;
    for (; z + 8 <= splits; z += 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p[(int64_t)(z + u) * MN];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; z < splits; ++z) acc += p[(int64_t)z * MN];
    T *c = C + i + j * ldc;
    T v = alpha * acc;
    if (beta != T(0)) v += beta * *c;
    *c = v;
}

}  // namespace

ct_status gemm_simt_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                           cudaStream_t s) {
    const double es = g.kind == GEMM_F64 ? 8.0 : 4.0;
    ProfScope prof(PROF_SIMT_GEMM, s, 2.0 * g.M * g.N * g.K,
                   es * ((double)g.M * g.K + (double)g.K * g.N + (double)g.M * g.N * splits),
                   g.M, g.N, g.K, splits);
    if (g.kind == GEMM_F64) {
        constexpr int BM = 64, BN = 64;
        dim3 grid((unsigned)ceil_div(g.M, BM), (unsigned)ceil_div(g.N, BN), (unsigned)splits);
        gemm_simt_kernel<double, BM, BN, 16, 4, 4><<<grid, 256, 0, s>>>(
            g.ta, g.tb, g.M, g.N, g.K, kchunk, g.alpha, (const double *)g.A, g.lda,
            (const double *)g.B, g.ldb, g.beta, (double *)g.C, g.ldc, split_stride);
        count_launch();
    } else {
        constexpr int BM = 128, BN = 128;
        dim3 grid((unsigned)ceil_div(g.M, BM), (unsigned)ceil_div(g.N, BN), (unsigned)splits);
        gemm_simt_kernel<float, BM, BN, 8, 8, 8><<<grid, 256, 0, s>>>(
            g.ta, g.tb, g.M, g.N, g.K, kchunk, (float)g.alpha, (const float *)g.A, g.lda,
            (const float *)g.B, g.ldb, (float)g.beta, (float *)g.C, g.ldc, split_stride);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status splitk_reduce(bool fp64, int64_t M, int64_t N, int splits, const void *P, double alpha,
                        double beta, void *C, int64_t ldc, cudaStream_t s) {
    const int64_t total = M * N;
    if (total == 0) return CT_OK;
    const double es = fp64 ? 8.0 : 4.0;
    ProfScope prof(PROF_OTHER, s, (double)splits * total, es * (double)total * (splits + (beta != 0.0 ? 2 : 1)), M, N,
                   splits, 0);
    const unsigned blocks = (unsigned)ceil_div(total, 256);
    if (fp64) {
        splitk_reduce_kernel<double><<<blocks, 256, 0, s>>>(M, N, splits, (const double *)P, alpha,
                                                            beta, (double *)C, ldc);
        count_launch();
    }
    else {
        splitk_reduce_kernel<float><<<blocks, 256, 0, s>>>(M, N, splits, (const float *)P,
                                                           (float)alpha, (float)beta, (float *)C,
                                                           ldc);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Split-K depth for a tile grid (enough CTAs to cover the machine about
// twice, each split at least min_chunk deep, chunks multiples of align).
// All scratch of one engine call (K-major operand copies for the tensor
// cores, then split-K partial products) lives in the caller's `ws`; nothing
// process-wide is used, so a captured graph that replays such a call
// references only its caller's buffers.
void plan_splits(int64_t tiles, int64_t K, int64_t min_chunk, int64_t align,
                        int64_t *splits_out, int64_t *kchunk_out) {
    const int64_t target = 2 * (int64_t)num_sms();
    int64_t splits = 1;
    if (tiles < target) splits = std::min(ceil_div(target, tiles), std::max<int64_t>(1, K / min_chunk));
    splits = std::min<int64_t>(splits, 64);
    int64_t kchunk = K;
    if (splits > 1) {
        kchunk = round_up(ceil_div(K, splits), align);
        splits = ceil_div(K, kchunk);
    }
    *splits_out = splits;
    *kchunk_out = kchunk;
}

// Tensor-core products through K-major operand copies in `ws`:
//   BF16: both operands rounded (to nearest even) to BF16;
//   BF16X3 / TF32X3: both operands split into hi + lo of the narrow type and
//     laid out as [hi, hi, lo] and [hi, lo, hi] along a K three times as
//     deep, so one product sums A_hi B_hi + A_hi B_lo + A_lo B_hi;
// then multiplied with FP32 accumulation.  A product whose B copy would
// exceed kChunkBytes is done in column slabs of C, reusing the A copy.
static ct_status gemm_copied(const GemmArgs &g, Scratch &ws, cudaStream_t s) {
    constexpr size_t kChunkBytes = (size_t)4 << 30;
    const bool split = g.kind == GEMM_BF16X3 || g.kind == GEMM_TF32X3;
    const bool b16 = g.kind == GEMM_BF16 || g.kind == GEMM_BF16X3;
    const int64_t es = b16 ? 2 : 4;
    const int64_t Kc = split ? 3 * g.K : g.K;  // depth of the product of the copies
    const int64_t ldt = round_up(Kc, 64);
    const bool pre_a = g.kind == GEMM_BF16 && g.A16 != nullptr;  // A already converted by the caller
    const bool pre_b = g.kind == GEMM_BF16 && g.B16 != nullptr;  // B likewise: no copy, one slab
    const size_t abytes = pre_a ? 0 : (size_t)round_up(es * ldt * g.M, 256);
    int64_t nslab = g.N;
    if (!pre_b && (size_t)(es * ldt) * (size_t)g.N > kChunkBytes)
        nslab = std::max<int64_t>(256, (int64_t)(kChunkBytes / (size_t)(es * ldt)) / 256 * 256);
    const size_t bbytes = pre_b ? 0 : (size_t)round_up(es * ldt * nslab, 256);
    const int64_t tiles = ceil_div(g.M, 128) * ceil_div(nslab, 256);
    int64_t splits, kchunk;
    plan_splits(tiles, Kc, 2048, 64, &splits, &kchunk);
    // the last, narrower slab may split K further: size the partials for both
    const int64_t nlast = g.N - (g.N - 1) / nslab * nslab;
    int64_t sp_last, kc_last;
    plan_splits(ceil_div(g.M, 128) * ceil_div(nlast, 256), Kc, 2048, 64, &sp_last, &kc_last);
    const size_t pbytes = std::max(splits > 1 ? 4 * (size_t)(g.M * nslab * splits) : (size_t)0,
                                   sp_last > 1 ? 4 * (size_t)(g.M * nlast * sp_last) : (size_t)0);
    CT_TRY(ws.ensure(abytes + bbytes + pbytes));
    void *Ab = pre_a ? const_cast<void *>(g.A16) : ws.ptr, *Bb = (char *)ws.ptr + abytes,
         *part = (char *)ws.ptr + abytes + bbytes;
    const int64_t lda_b = pre_a ? g.lda16 : ldt;
    const int split_kind = b16 ? 2 : 3;
    if (pre_a) {
        // nothing to convert
    } else if (split) CT_TRY(split3_copy((const float *)g.A, g.lda, g.ta, split_kind, false, Ab, ldt, g.K, g.M, s));
    else if (g.ta) CT_TRY(copy_convert_2d(0, g.A, g.lda, 2, Ab, ldt, g.K, g.M, s));
    else CT_TRY(transpose_any(0, g.A, g.lda, 2, Ab, ldt, g.M, g.K, s));
    for (int64_t n0 = 0; n0 < g.N; n0 += nslab) {
        const int64_t nn = std::min(nslab, g.N - n0);
        const size_t fs = 4;  // FP32 operands and C
        const float *Bs = (const float *)((const char *)g.B + fs * (size_t)(g.tb ? n0 : n0 * g.ldb));
        if (pre_b) {
            // nothing to convert
        } else if (split) CT_TRY(split3_copy(Bs, g.ldb, !g.tb, split_kind, true, Bb, ldt, g.K, nn, s));
        else if (!g.tb) CT_TRY(copy_convert_2d(0, Bs, g.ldb, 2, Bb, ldt, g.K, nn, s));
        else CT_TRY(transpose_any(0, Bs, g.ldb, 2, Bb, ldt, nn, g.K, s));
        GemmArgs b = g;
        b.kind = b16 ? GEMM_BF16 : GEMM_TF32;
        b.K = Kc;
        b.ta = true;
        b.tb = false;
        b.A = Ab;
        b.lda = lda_b;
        b.B = pre_b ? (const void *)((const char *)g.B16 + 2 * (size_t)(n0 * g.ldb16)) : (const void *)Bb;
        b.ldb = pre_b ? g.ldb16 : ldt;
        b.N = nn;
        b.C = (char *)g.C + fs * (size_t)(n0 * g.ldc);
        int64_t sp = splits, kc = kchunk;
        if (nn != nslab) {
            sp = sp_last;
            kc = kc_last;
        }
        if (sp <= 1) {
            CT_TRY(gemm_tc_launch(b, 1, Kc, 0, s));
            continue;
        }
        GemmArgs p = b;
        p.alpha = 1.0;
        p.beta = 0.0;
        p.C = part;
        p.ldc = g.M;
        CT_TRY(gemm_tc_launch(p, (int)sp, kc, g.M * nn, s));
        CT_TRY(splitk_reduce(false, g.M, nn, (int)sp, part, g.alpha, g.beta, b.C, g.ldc, s));
    }
    return CT_OK;
}

ct_status gemm(const GemmArgs &g0, Scratch &ws, cudaStream_t s) {
    if (g0.M < 0 || g0.N < 0 || g0.K < 0) return CT_ERR_ARG;
    if (g0.M == 0 || g0.N == 0) return CT_OK;
    const bool copied = g0.kind == GEMM_BF16 || g0.kind == GEMM_BF16X3 || g0.kind == GEMM_TF32X3;
    if (g0.splits_out) *g0.splits_out = 0;
    if (copied && g0.K > 0) return gemm_copied(g0, ws, s);
    GemmArgs g = g0;
    const bool fp64 = g.kind == GEMM_F64;
    if (copied) g.kind = GEMM_F32;  // only reached with K == 0
    bool tc = g.kind == GEMM_TF32;
    if (tc && (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15) || (g.lda & 3) || (g.ldb & 3))) {
        // A TMA tile must start on a 16-byte boundary; ragged sub-blocks that
        // do not (only at the edges of odd-sized problems) use the FP32 SIMT path.
        g.kind = GEMM_F32;
        tc = false;
    }
    if (g.K == 0) {
        // C = beta * C
        if (g.beta == 1.0) return CT_OK;
        return splitk_reduce(fp64, g.M, g.N, 0, nullptr, 0.0, g.beta, g.C, g.ldc, s);
    }
    // The tensor cores take TF32 operands K-major only (each output row's K
    // values contiguous; the MN-major form is not available for 32-bit
    // operands).  An operand stored the other way round is transposed into a
    // K-major copy first.
    const bool tra = tc && !g.ta, trb = tc && g.tb;
    const int64_t ldt = round_up(g.K, 32);
    const size_t abytes = tra ? (size_t)round_up((int64_t)(sizeof(float) * ldt * g.M), 256) : 0;
    const size_t bbytes = trb ? (size_t)round_up((int64_t)(sizeof(float) * ldt * g.N), 256) : 0;
    const int64_t BM = tc ? 128 : (fp64 ? 64 : 128);
    const int64_t BN = tc ? 256 : (fp64 ? 64 : 128);
    const int64_t tiles = ceil_div(g.M, BM) * ceil_div(g.N, BN);
    int64_t splits, kchunk;
    plan_splits(tiles, g.K, g.min_chunk > 0 ? g.min_chunk : (tc ? 256 : 128), tc ? 32 : 16, &splits, &kchunk);
    const size_t esz = fp64 ? 8 : 4;
    const size_t pbytes = splits > 1 ? esz * (size_t)(g.M * g.N * splits) : 0;
    if (abytes + bbytes + pbytes > 0) CT_TRY(ws.ensure(abytes + bbytes + pbytes));
    if (tra) {
        CT_TRY(transpose_any(0, g.A, g.lda, 0, ws.ptr, ldt, g.M, g.K, s));  // A (M x K) -> K x M
        g.A = ws.ptr;
        g.lda = ldt;
        g.ta = true;
    }
    if (trb) {
        void *bt = (char *)ws.ptr + abytes;
        CT_TRY(transpose_any(0, g.B, g.ldb, 0, bt, ldt, g.N, g.K, s));  // B (N x K) -> K x N
        g.B = bt;
        g.ldb = ldt;
        g.tb = false;
    }
    if (splits <= 1) {
        return tc ? gemm_tc_launch(g, 1, g.K, 0, s) : gemm_simt_launch(g, 1, g.K, 0, s);
    }
    void *part = (char *)ws.ptr + abytes + bbytes;
    GemmArgs p = g;
    p.alpha = 1.0;
    p.beta = 0.0;
    p.C = part;
    p.ldc = g.M;
    CT_TRY(tc ? gemm_tc_launch(p, (int)splits, kchunk, g.M * g.N, s)
              : gemm_simt_launch(p, (int)splits, kchunk, g.M * g.N, s));
    if (g.partials_out != nullptr && g.splits_out != nullptr) {  // the caller reduces
        *g.partials_out = part;
        *g.splits_out = (int)splits;
        return CT_OK;
    }
    return splitk_reduce(fp64, g.M, g.N, (int)splits, part, g.alpha, g.beta, g.C, g.ldc, s);
}

}  // namespace ctqr
