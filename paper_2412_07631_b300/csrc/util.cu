// util.cu -- layout/precision copies and small reductions used around the
// factorisation and the solve.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

#include <cuda_bf16.h>

namespace ctqr {

namespace {

template <typename D> __device__ __forceinline__ D cvt(float v) { return (D)v; }
template <typename D> __device__ __forceinline__ D cvt(double v) { return (D)v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

template <typename S, typename D>
__global__ void copy_convert_kernel(const S *src, int64_t lds, D *dst, int64_t ldd, int64_t rows,
                                    int64_t cols) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    int64_t i = idx % rows, j = idx / rows;
    dst[i + j * ldd] = cvt<D>(src[i + j * lds]);
}

// FP32 -> BF16 (round to nearest even) in both layouts at once, from one read
// of the source (rows x cols, column-major, ld lds): colm(r, c) at
// r + c * ldc (the same layout) and rowm(r, c) at c + r * ldr (transposed).
// 32 x 32 tiles, block (32, 8); the transposed writes go through shared
// memory so both stores are contiguous along a warp.
__global__ void to_bf16_dual_kernel(const float *src, int64_t lds, int64_t rows, int64_t cols,
                                    __nv_bfloat16 *colm, int64_t ldc, __nv_bfloat16 *rowm, int64_t ldr) {
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t r = r0 + tx, c = c0 + ty + 8 * q;
        float v = 0.0f;
        if (r < rows && c < cols) {
            v = src[r + c * lds];
            if (colm) colm[r + c * ldc] = __float2bfloat16_rn(v);
        }
        t[ty + 8 * q][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t r = r0 + ty + 8 * q, c = c0 + tx;
        if (r < rows && c < cols) rowm[c + r * ldr] = __float2bfloat16_rn(t[tx][ty + 8 * q]);
    }
}

// The same conversion over 64 x 64 tiles: each thread reads 16 values and
// writes the transposed copy as pairs (4-byte stores, 128 bytes per warp).
// Needs rowm 4-byte aligned and ldr even.
__global__ void __launch_bounds__(256) to_bf16_dual64_kernel(const float *src, int64_t lds, int64_t rows,
                                                             int64_t cols, __nv_bfloat16 *colm, int64_t ldc,
                                                             __nv_bfloat16 *rowm, int64_t ldr) {
    __shared__ __align__(16) float t[64][66];  // t[row][col] of the tile
    const int64_t r0 = (int64_t)blockIdx.x * 64, c0 = (int64_t)blockIdx.y * 64;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lr = tx + 32 * h, lc = ty + 8 * q;
            const int64_t r = r0 + lr, c = c0 + lc;
            float v = 0.0f;
            if (r < rows && c < cols) {
                v = src[r + c * lds];
                if (colm) colm[r + c * ldc] = __float2bfloat16_rn(v);
            }
            t[lr][lc] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int lr = ty + 8 * q, lc = 2 * tx;
        const int64_t r = r0 + lr, c = c0 + lc;
        if (r < rows && c < cols) {
            const float2 p = *reinterpret_cast<const float2 *>(&t[lr][lc]);
            if (c + 1 < cols)
                *reinterpret_cast<__nv_bfloat162 *>(rowm + c + r * ldr) = __floats2bfloat162_rn(p.x, p.y);
            else
                rowm[c + r * ldr] = __float2bfloat16_rn(p.x);
        }
    }
}

// FP32 -> BF16 (round to nearest even), column by column: blockIdx.y strides
// over columns, each thread converts 4 consecutive rows.
__global__ void to_bf16_kernel(const float *src, int64_t lds, __nv_bfloat16 *dst, int64_t ldd,
                               int64_t rows, int64_t cols) {
    const int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= rows) return;
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y) {
        const float *sp = src + j * lds + i;
        __nv_bfloat16 *dp = dst + j * ldd + i;
        if (i + 4 <= rows) {
            const float a = sp[0], b = sp[1], c = sp[2], d = sp[3];
            dp[0] = __float2bfloat16_rn(a);
            dp[1] = __float2bfloat16_rn(b);
            dp[2] = __float2bfloat16_rn(c);
            dp[3] = __float2bfloat16_rn(d);
        } else {
            for (int64_t r = i; r < rows; ++r) dst[j * ldd + r] = __float2bfloat16_rn(src[j * lds + r]);
        }
    }
}

// As to_bf16_kernel with 16-byte accesses: each thread converts 8
// consecutive rows (two float4 loads, one 16-byte store).  Needs src, dst,
// lds * 4 and ldd * 2 bytes to be multiples of 16.
__global__ void to_bf16_vec_kernel(const float *src, int64_t lds, __nv_bfloat16 *dst, int64_t ldd,
                                   int64_t rows, int64_t cols) {
    const int64_t i = 8 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= rows) return;
    for (int64_t j = blockIdx.y; j < cols; j += gridDim.y) {
        const float *sp = src + j * lds + i;
        __nv_bfloat16 *dp = dst + j * ldd + i;
        if (i + 8 <= rows) {
            const float4 a = __ldcs(reinterpret_cast<const float4 *>(sp));
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(sp + 4));
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
            uint4 o;
            o.x = *reinterpret_cast<const uint32_t *>(&p0);
            o.y = *reinterpret_cast<const uint32_t *>(&p1);
            o.z = *reinterpret_cast<const uint32_t *>(&p2);
            o.w = *reinterpret_cast<const uint32_t *>(&p3);
            *reinterpret_cast<uint4 *>(dp) = o;
        } else {
            for (int64_t r = i; r < rows; ++r) dst[j * ldd + r] = __float2bfloat16_rn(src[j * lds + r]);
        }
    }
}

template <typename T>
__global__ void fill_zero_kernel(T *dst, int64_t ld, int64_t rows, int64_t cols) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    int64_t i = idx % rows, j = idx / rows;
    dst[i + j * ld] = T(0);
}

// Raises DEV_NONFINITE (site `where`) if any element of the rows x cols
// column-major block is NaN or Inf.  Grid-stride; one status write at most
// per warp that meets one.
template <typename T>
__global__ void scan_finite_kernel(const T *A, int64_t ld, int64_t rows, int64_t cols, int where,
                                   DevStatus *st) {
    const int64_t total = rows * cols;
    bool bad = false;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx % rows, j = idx / rows;
        if (!isfinite(A[i + j * ld])) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(st, DEV_NONFINITE, where, 0);
}

template <typename T>
__global__ void rdiag_minmax_kernel(const T *A, int64_t lda, int64_t n, double *out,
                                    DevStatus *st) {
    __shared__ double smin[256], smax[256];
    double mn = INFINITY, mx = 0.0;
    bool bad = false;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double v = fabs((double)A[j + j * lda]);
        if (!isfinite(v)) bad = true;
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
    if (bad) raise_status(st, DEV_NONFINITE, 30, 0);
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smin[0];
        out[1] = smax[0];
    }
}

// dst[j + i*ldd] = src[i + j*lds] for i < rows, j < cols (32 x 32 smem tiles).
template <typename S, typename D>
__global__ void transpose_kernel(const S *src, int64_t lds, D *dst, int64_t ldd, int64_t rows,
                                 int64_t cols) {
    __shared__ D tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int64_t i = i0 + threadIdx.x, j = j0 + r;
        if (i < rows && j < cols) tile[r][threadIdx.x] = cvt<D>(src[i + j * lds]);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int64_t j = j0 + threadIdx.x, i = i0 + r;
        if (i < rows && j < cols) dst[j + i * ldd] = tile[threadIdx.x][r];
    }
}

// Round to the nearest TF32 value (10 explicit mantissa bits), ties away
// from zero, kept in FP32 format with the 13 low bits cleared.  Finite
// inputs only (the factorisation stops on non-finite values elsewhere).
__device__ __forceinline__ float round_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <typename D> struct Split;
template <> struct Split<__nv_bfloat16> {
    static __device__ __forceinline__ void run(float x, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
        *hi = __float2bfloat16_rn(x);
        *lo = __float2bfloat16_rn(x - __bfloat162float(*hi));
    }
};
template <> struct Split<float> {  // TF32 values in FP32 words
    static __device__ __forceinline__ void run(float x, float *hi, float *lo) {
        *hi = round_tf32(x);
        *lo = round_tf32(x - *hi);
    }
};

// One 32 x 32 tile of op(src) (k0.., j0..) through shared memory, so both
// the read (either layout) and the three K-runs of the write are coalesced.
template <typename D, bool KMAJOR>
__global__ void split3_kernel(const float *src, int64_t lds, D *dst, int64_t ldt, int64_t K, int64_t MN,
                              bool second) {
    __shared__ float tile[32][33];  // [j][k]
    const int64_t k0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        if (KMAJOR) {
            const int64_t k = k0 + threadIdx.x, j = j0 + r;
            if (k < K && j < MN) tile[r][threadIdx.x] = src[k + j * lds];
        } else {
            const int64_t j = j0 + threadIdx.x, k = k0 + r;
            if (k < K && j < MN) tile[threadIdx.x][r] = src[j + k * lds];
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t k = k0 + threadIdx.x, j = j0 + r;
        if (k < K && j < MN) {
            D hi, lo;
            Split<D>::run(tile[r][threadIdx.x], &hi, &lo);
            D *d = dst + j * ldt;
            d[k] = hi;
            d[K + k] = second ? lo : hi;
            d[2 * K + k] = second ? hi : lo;
        }
    }
}

}  // namespace

ct_status split3_copy(const float *src, int64_t lds, bool src_kmajor, int dst_kind, bool second_operand,
                      void *dst, int64_t ldt, int64_t K, int64_t MN, cudaStream_t s) {
    if (K == 0 || MN == 0) return CT_OK;
    if ((dst_kind != 2 && dst_kind != 3) || ldt < 3 * K) return CT_ERR_ARG;
    const dim3 block(32, 8);
    for (int64_t c0 = 0; c0 < MN; c0 += 32 * 65535LL) {  // grid.y limit
        const int64_t cc = std::min<int64_t>(MN - c0, 32 * 65535LL);
        const float *sp = src + (src_kmajor ? c0 * lds : c0);
        const dim3 grid((unsigned)ceil_div(K, 32), (unsigned)ceil_div(cc, 32));
        if (dst_kind == 2) {
            __nv_bfloat16 *dp = (__nv_bfloat16 *)dst + c0 * ldt;
            if (src_kmajor) split3_kernel<__nv_bfloat16, true><<<grid, block, 0, s>>>(sp, lds, dp, ldt, K, cc, second_operand);
            else split3_kernel<__nv_bfloat16, false><<<grid, block, 0, s>>>(sp, lds, dp, ldt, K, cc, second_operand);
        } else {
            float *dp = (float *)dst + c0 * ldt;
            if (src_kmajor) split3_kernel<float, true><<<grid, block, 0, s>>>(sp, lds, dp, ldt, K, cc, second_operand);
            else split3_kernel<float, false><<<grid, block, 0, s>>>(sp, lds, dp, ldt, K, cc, second_operand);
        }
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Bytes of one element of a buffer kind: 0 float, 1 double, 2 bf16.
static inline double kind_bytes(int kind) { return kind == 1 ? 8.0 : (kind == 2 ? 2.0 : 4.0); }

ct_status transpose_any(int src_kind, const void *src, int64_t lds, int dst_kind, void *dst,
                        int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s) {
    if (rows == 0 || cols == 0) return CT_OK;
    ProfScope prof(PROF_COPY, s, 0.0, (kind_bytes(src_kind) + kind_bytes(dst_kind)) * (double)rows * cols, rows,
                   cols, src_kind, dst_kind);
    dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32)), block(32, 8);
    if (dst_kind == 2) {  // FP32 -> BF16
        if (src_kind != 0) return CT_ERR_ARG;
        for (int64_t c0 = 0; c0 < cols; c0 += 32 * 65535LL) {  // grid.y limit
            const int64_t cc = std::min<int64_t>(cols - c0, 32 * 65535LL);
            dim3 g2((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cc, 32));
            transpose_kernel<float, __nv_bfloat16><<<g2, block, 0, s>>>(
                (const float *)src + c0 * lds, lds, (__nv_bfloat16 *)dst + c0, ldd, rows, cc);
            count_launch();
        }
    }
    else if (src_kind == 1 && dst_kind == 1) {
        transpose_kernel<double, double><<<grid, block, 0, s>>>((const double *)src, lds, (double *)dst, ldd, rows, cols);
        count_launch();
    }
    else if (src_kind == 1 && dst_kind == 0) {
        transpose_kernel<double, float><<<grid, block, 0, s>>>((const double *)src, lds, (float *)dst, ldd, rows, cols);
        count_launch();
    }
    else if (src_kind == 0 && dst_kind == 1) {
        transpose_kernel<float, double><<<grid, block, 0, s>>>((const float *)src, lds, (double *)dst, ldd, rows, cols);
        count_launch();
    }
    else {
        transpose_kernel<float, float><<<grid, block, 0, s>>>((const float *)src, lds, (float *)dst, ldd, rows, cols);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status transpose_d(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t rows,
                      int64_t cols, cudaStream_t s) {
    return transpose_any(1, src, lds, 1, dst, ldd, rows, cols, s);
}

ct_status convert_bf16_dual(const float *src, int64_t lds, int64_t rows, int64_t cols, void *colm, int64_t ldc,
                            void *rowm, int64_t ldr, cudaStream_t s) {
    if (rows == 0 || cols == 0) return CT_OK;
    ProfScope prof(PROF_COPY, s, 0.0, (colm ? 8.0 : 6.0) * (double)rows * cols, rows, cols, 0, colm ? 4 : 5);
    const bool wide = (ldr & 1) == 0 && ((uintptr_t)rowm & 3) == 0;  // pairs of the transposed copy
    const int64_t tile = wide ? 64 : 32;
    for (int64_t c0 = 0; c0 < cols; c0 += tile * 65535LL) {  // grid.y limit
        const int64_t cc = std::min<int64_t>(cols - c0, tile * 65535LL);
        dim3 grid((unsigned)ceil_div(rows, tile), (unsigned)ceil_div(cc, tile)), block(32, 8);
        __nv_bfloat16 *cm = colm ? (__nv_bfloat16 *)colm + c0 * ldc : nullptr;
        if (wide)
            to_bf16_dual64_kernel<<<grid, block, 0, s>>>(src + c0 * lds, lds, rows, cc, cm, ldc,
                                                         (__nv_bfloat16 *)rowm + c0, ldr);
        else
            to_bf16_dual_kernel<<<grid, block, 0, s>>>(src + c0 * lds, lds, rows, cc, cm, ldc,
                                                       (__nv_bfloat16 *)rowm + c0, ldr);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status copy_convert_2d(int src_kind, const void *src, int64_t lds, int dst_kind, void *dst,
                          int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s) {
    const int64_t total = rows * cols;
    if (total == 0) return CT_OK;
    ProfScope prof(PROF_COPY, s, 0.0, (kind_bytes(src_kind) + kind_bytes(dst_kind)) * (double)total, rows, cols,
                   src_kind, dst_kind);
    const unsigned b = (unsigned)ceil_div(total, 256);
    if (dst_kind == 2) {  // FP32 -> BF16
        if (src_kind != 0) return CT_ERR_ARG;
        const bool vec = ((uintptr_t)src & 15) == 0 && ((uintptr_t)dst & 15) == 0 && (lds & 3) == 0 &&
                         (ldd & 7) == 0;
        if (vec) {
            dim3 g2((unsigned)ceil_div(ceil_div(rows, 8), 256), (unsigned)std::min<int64_t>(cols, 32768));
            to_bf16_vec_kernel<<<g2, 256, 0, s>>>((const float *)src, lds, (__nv_bfloat16 *)dst, ldd, rows, cols);
        } else {
            dim3 g2((unsigned)ceil_div(ceil_div(rows, 4), 256), (unsigned)std::min<int64_t>(cols, 32768));
            to_bf16_kernel<<<g2, 256, 0, s>>>((const float *)src, lds, (__nv_bfloat16 *)dst, ldd, rows, cols);
        }
        count_launch();
    }
    else if (src_kind == 0 && dst_kind == 0) {
        copy_convert_kernel<float, float><<<b, 256, 0, s>>>((const float *)src, lds, (float *)dst, ldd, rows, cols);
        count_launch();
    }
    else if (src_kind == 0 && dst_kind == 1) {
        copy_convert_kernel<float, double><<<b, 256, 0, s>>>((const float *)src, lds, (double *)dst, ldd, rows, cols);
        count_launch();
    }
    else if (src_kind == 1 && dst_kind == 0) {
        copy_convert_kernel<double, float><<<b, 256, 0, s>>>((const double *)src, lds, (float *)dst, ldd, rows, cols);
        count_launch();
    }
    else {
        copy_convert_kernel<double, double><<<b, 256, 0, s>>>((const double *)src, lds, (double *)dst, ldd, rows, cols);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status fill_zero_2d(bool fp64, void *dst, int64_t ld, int64_t rows, int64_t cols,
                       cudaStream_t s) {
    const int64_t total = rows * cols;
    if (total == 0) return CT_OK;
    const unsigned b = (unsigned)ceil_div(total, 256);
    if (fp64) fill_zero_kernel<double><<<b, 256, 0, s>>>((double *)dst, ld, rows, cols);
    else fill_zero_kernel<float><<<b, 256, 0, s>>>((float *)dst, ld, rows, cols);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status scan_finite(int kind, const void *A, int64_t ld, int64_t rows, int64_t cols, int where,
                      cudaStream_t s) {
    const int64_t total = rows * cols;
    if (total == 0) return CT_OK;
    const unsigned b = (unsigned)std::min<int64_t>(ceil_div(total, 256), 8 * (int64_t)num_sms());
    if (kind == 1) scan_finite_kernel<double><<<b, 256, 0, s>>>((const double *)A, ld, rows, cols, where, device_status());
    else scan_finite_kernel<float><<<b, 256, 0, s>>>((const float *)A, ld, rows, cols, where, device_status());
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status rdiag_minmax(bool fp64, const void *A, int64_t lda, int64_t n, double *out,
                       cudaStream_t s) {
    if (fp64) rdiag_minmax_kernel<double><<<1, 256, 0, s>>>((const double *)A, lda, n, out, device_status());
    else rdiag_minmax_kernel<float><<<1, 256, 0, s>>>((const float *)A, lda, n, out, device_status());
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ctqr
