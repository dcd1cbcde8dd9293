// simt_tile.cuh -- one output tile of a CUDA-core GEMM, shared by the GEMM
// engine's SIMT kernel and the batched triangular-inverse doubling.
//
// C[m0:m0+BM, n0:n0+BN] = alpha * sum_{k in [kb, ke)} op(A)(m, k) op(B)(k, n)
//                         + beta * C   (column-major; op = N or T)
// 256 threads, each owning a TM x TN register tile; op(A)/op(B) tiles staged
// in shared memory with the M (resp. N) index fastest so the inner product
// loop reads contiguous vectors.  k runs in ascending order from kb.
#pragma once

#include <stdint.h>

namespace ctqr {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void simt_tile(bool ta, bool tb, int64_t M, int64_t N, int64_t kb,
                                          int64_t ke, T alpha, const T *__restrict__ A, int64_t lda,
                                          const T *__restrict__ B, int64_t ldb, T beta, T *C,
                                          int64_t ldc, int64_t m0, int64_t n0) {
    static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        // op(A) tile: element (i, kk) = A(m0+i, k0+kk) or A(k0+kk, m0+i).
        for (int idx = tid; idx < BM * BK; idx += 256) {
            int i, kk;
            if (!ta) { i = idx % BM; kk = idx / BM; }
            else { kk = idx % BK; i = idx / BK; }
            int64_t gm = m0 + i, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < ke) v = ta ? A[gk + gm * lda] : A[gm + gk * lda];
            As[kk][i] = v;
        }
        // op(B) tile: element (kk, j) = B(k0+kk, n0+j) or B(n0+j, k0+kk).
        for (int idx = tid; idx < BN * BK; idx += 256) {
            int j, kk;
            if (!tb) { kk = idx % BK; j = idx / BK; }
            else { j = idx % BN; kk = idx / BN; }
            int64_t gn = n0 + j, gk = k0 + kk;
            T v = T(0);
            if (gn < N && gk < ke) v = tb ? B[gn + gk * ldb] : B[gk + gn * ldb];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        int64_t gn = n0 + tx * TN + j;
        if (gn >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int64_t gm = m0 + ty * TM + i;
            if (gm >= M) continue;
            T *c = C + gm + gn * ldc;
            T v = alpha * acc[i][j];
            if (beta != T(0)) v += beta * *c;
            *c = v;
        }
    }
}

}  // namespace ctqr
