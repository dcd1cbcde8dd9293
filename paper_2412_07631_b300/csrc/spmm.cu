// spmm.cu -- sparse products with the Siddon matrix for k images at once:
// the forward projection A X, the regularised residual b~ - A~ X and the
// back-projection A~^T R.  The refinement computes its residuals here, in
// FP64, from the exact sparse A rather than from the low-precision dense
// copy; its inner correction solves use the same kernels in FP32.
//
// Operands are row-major with the slice index fastest (element (i, s) at
// Y[i*k + s]) so that the k values a nonzero multiplies are one contiguous,
// coalesced run.  One warp per matrix row; lanes stride over the slices.
#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

// out[i, :] = alpha*Y[i, :] + beta * sum_q val[q] * X[col[q], :]   (ray rows)
// and for the sqrt(lambda) rows i = m + j:  (A~ X)[m+j, :] = sl * X[j, :].
template <typename T>
__global__ void spmm_ax_kernel(int64_t m, int64_t n, int64_t k, T sl, const int64_t *row_ptr,
                               const int32_t *col, const T *val, const T *X, T alpha,
                               const T *Y, T beta, T *out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    const int64_t rows = m + (sl > T(0) ? n : 0);
    if (row >= rows) return;
    for (int64_t s0 = 0; s0 < k; s0 += 32 * 4) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        if (row < m) {
            for (int64_t q = row_ptr[row]; q < row_ptr[row + 1]; ++q) {
                const T a = val[q];
                const T *xr = X + (int64_t)col[q] * k;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t s = s0 + lane + 32 * u;
                    if (s < k) acc[u] += a * xr[s];
                }
            }
        } else {
            const T *xr = X + (row - m) * k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t s = s0 + lane + 32 * u;
                if (s < k) acc[u] = sl * xr[s];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t s = s0 + lane + 32 * u;
            if (s < k) {
                T v = beta * acc[u];
                if (alpha != T(0)) v += alpha * Y[row * k + s];
                out[row * k + s] = v;
            }
        }
    }
}

// out[j, :] = alpha*Y[j, :] + beta * (sum_{q in col j} csc_val[q] * R[csc_row[q], :]
//                                     + sl * R[m + j, :])
template <typename T>
__global__ void spmm_atr_kernel(int64_t m, int64_t n, int64_t k, T sl, const int64_t *col_ptr,
                                const int32_t *csc_row, const T *csc_val, const T *R,
                                T alpha, const T *Y, T beta, T *out) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (j >= n) return;
    for (int64_t s0 = 0; s0 < k; s0 += 32 * 4) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int64_t q = col_ptr[j]; q < col_ptr[j + 1]; ++q) {
            const T a = csc_val[q];
            const T *rr = R + (int64_t)csc_row[q] * k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t s = s0 + lane + 32 * u;
                if (s < k) acc[u] += a * rr[s];
            }
        }
        if (sl > T(0)) {
            const T *rr = R + (m + j) * k;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t s = s0 + lane + 32 * u;
                if (s < k) acc[u] += sl * rr[s];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t s = s0 + lane + 32 * u;
            if (s < k) {
                T v = beta * acc[u];
                if (alpha != T(0)) v += alpha * Y[j * k + s];
                out[j * k + s] = v;
            }
        }
    }
}

// Variants with 16-byte accesses, for k a multiple of the vector width (4
// floats, 2 doubles): one warp per row (column), each lane keeping NV
// vector accumulators, i.e. 512 slices per pass over the row's nonzeros (one
// pass for k <= 512), so the row's indices are read once per 512 slices and
// each nonzero gathers its image row with 16-byte loads.  Same FMAs in the
// same order as the scalar kernels above.
template <typename T> struct Vec;
template <> struct Vec<float> {
    using V = float4;
    static constexpr int W = 4, NV = 4;
    static __device__ __forceinline__ V fma1(float a, V x, V c) {
        return make_float4(fmaf(a, x.x, c.x), fmaf(a, x.y, c.y), fmaf(a, x.z, c.z), fmaf(a, x.w, c.w));
    }
    static __device__ __forceinline__ V zero() { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
    static __device__ __forceinline__ V axpby(float b, V acc, float a, V y) {
        return make_float4(b * acc.x + a * y.x, b * acc.y + a * y.y, b * acc.z + a * y.z, b * acc.w + a * y.w);
    }
    static __device__ __forceinline__ V scale(float b, V acc) {
        return make_float4(b * acc.x, b * acc.y, b * acc.z, b * acc.w);
    }
};
template <> struct Vec<double> {
    using V = double2;
    static constexpr int W = 2, NV = 8;
    static __device__ __forceinline__ V fma1(double a, V x, V c) { return make_double2(fma(a, x.x, c.x), fma(a, x.y, c.y)); }
    static __device__ __forceinline__ V zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ V axpby(double b, V acc, double a, V y) {
        return make_double2(b * acc.x + a * y.x, b * acc.y + a * y.y);
    }
    static __device__ __forceinline__ V scale(double b, V acc) { return make_double2(b * acc.x, b * acc.y); }
};

// Rows of the forward product A~ X in CTA order.  With n_bins > 0 (ray rows
// i = v * n_bins + d) the 8 warps of a CTA take vb neighbouring views times
// 8 / vb neighbouring bins: rays of nearby views at nearby offsets cross
// mostly the same pixels, so the warps of a CTA gather mostly the same image
// rows and L1 serves the repeats (within one view a pixel meets only one or
// two rays).  The sqrt(lambda) rows follow in natural order.  Returns -1 for
// a warp with no row.
__device__ __forceinline__ int64_t ax_row(int64_t m, int64_t rows, int64_t n_bins, int vb) {
    const int64_t w = threadIdx.x / 32;
    if (n_bins <= 0) {
        const int64_t row = (int64_t)blockIdx.x * 8 + w;
        return row < rows ? row : -1;
    }
    const int64_t bins = 8 / vb;
    const int64_t n_views = m / n_bins;
    const int64_t tiles_d = (n_bins + bins - 1) / bins;
    const int64_t tiles = (n_views + vb - 1) / vb * tiles_d;
    const int64_t b = blockIdx.x;
    if (b >= tiles) {
        const int64_t row = m + (b - tiles) * 8 + w;
        return row < rows ? row : -1;
    }
    const int64_t v = (b / tiles_d) * vb + w % vb;
    const int64_t d = (b % tiles_d) * bins + w / vb;
    return (v < n_views && d < n_bins) ? v * n_bins + d : -1;
}
int64_t ax_blocks(int64_t m, int64_t rows, int64_t n_bins, int vb) {
    if (n_bins <= 0) return ceil_div(rows, 8);
    const int64_t tiles = ceil_div(m / n_bins, (int64_t)vb) * ceil_div(n_bins, (int64_t)(8 / vb));
    return tiles + ceil_div(rows - m, 8);
}
// Columns (pixels) of the back-projection A~^T R in CTA order: with
// n_side > 0 the 8 warps of a CTA take a tile of pw x (8 / pw) pixels, whose
// rays largely coincide.  Returns -1 for a warp with no column.
__device__ __forceinline__ int64_t atr_col(int64_t n, int64_t n_side, int pw) {
    const int64_t w = threadIdx.x / 32;
    if (n_side <= 0) {
        const int64_t j = (int64_t)blockIdx.x * 8 + w;
        return j < n ? j : -1;
    }
    const int64_t ph = 8 / pw;
    const int64_t tiles_x = (n_side + pw - 1) / pw;
    const int64_t ty = blockIdx.x / tiles_x, tx = blockIdx.x % tiles_x;
    const int64_t iy = ty * ph + w / pw, ix = tx * pw + w % pw;
    return (iy < n_side && ix < n_side) ? iy * n_side + ix : -1;
}
int64_t atr_blocks(int64_t n, int64_t n_side, int pw) {
    if (n_side <= 0) return ceil_div(n, 8);
    return ceil_div(n_side, (int64_t)pw) * ceil_div(n_side, (int64_t)(8 / pw));
}
// Tile shapes, measured on the FP32 products of a 256^2 solve (512 slices):
// 8 views x 1 bin per CTA for the forward product (4% less time than 4 x 2
// or 2 x 4), 4 x 2 pixels per CTA for the back-projection (2% less than a
// row of 8).
constexpr int kAxViews = 8;
constexpr int kAtrWidth = 4;

template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) spmm_vec_kernel(int64_t m, int64_t n, int64_t k, T sl,
                                                       const int64_t *ptr, const int32_t *idx,
                                                       const T *val, const T *X, T alpha,
                                                       const T *Y, T beta, T *out, int64_t order, int tile) {
    using VT = Vec<T>;
    using V = typename VT::V;
    constexpr int NV = VT::NV;
    const int lane = threadIdx.x % 32;
    const int64_t rows = TRANS ? n : m + (sl > T(0) ? n : 0);
    int64_t row;
    row = TRANS ? atr_col(n, order, tile) : ax_row(m, rows, order, tile);
    if (row < 0) return;
    const int64_t kv = k / VT::W;
    for (int64_t c0 = 0; c0 < kv; c0 += 32 * NV) {
        V acc[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u) acc[u] = VT::zero();
        const bool ray = TRANS || row < m;
        if (ray) {
            const int64_t q0 = ptr[row], q1 = ptr[row + 1];
            for (int64_t q = q0; q < q1; ++q) {
                const T a = val[q];
                const V *xr = reinterpret_cast<const V *>(X + (int64_t)idx[q] * k);
#pragma unroll
                for (int u = 0; u < NV; ++u) {
                    const int64_t c = c0 + lane + 32 * u;
                    if (c < kv) acc[u] = VT::fma1(a, __ldg(xr + c), acc[u]);
                }
            }
        }
        if (sl > T(0) && (TRANS || !ray)) {  // the sqrt(lambda) I block
            const V *xr = reinterpret_cast<const V *>(X + (TRANS ? (m + row) : (row - m)) * k);
#pragma unroll
            for (int u = 0; u < NV; ++u) {
                const int64_t c = c0 + lane + 32 * u;
                if (c < kv) acc[u] = VT::fma1(sl, xr[c], acc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int64_t c = c0 + lane + 32 * u;
            if (c < kv) {
                const V v = (alpha != T(0)) ? VT::axpby(beta, acc[u], alpha, reinterpret_cast<const V *>(Y + row * k)[c])
                                            : VT::scale(beta, acc[u]);
                reinterpret_cast<V *>(out + row * k)[c] = v;
            }
        }
    }
}

bool vec_ok(int64_t k, int width, const void *a, const void *b, const void *c) {
    return k % width == 0 && (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) == 0;
}

}  // namespace

ct_status spmm_ax(const SparseSys &S, int64_t k, const double *X, double alpha, const double *Y,
                  double beta, double *out, cudaStream_t s) {
    const int64_t rows = S.m + (S.sqrt_lambda > 0.0 ? S.n : 0);
    if (rows == 0 || k == 0) return CT_OK;
    const unsigned blocks = (unsigned)ceil_div(rows * 32, 256);
    ProfScope prof(PROF_SPMM, s, 2.0 * (S.nnz + (rows - S.m)) * k,
                   12.0 * S.nnz + 8.0 * (double)k * (S.n + rows * (alpha != 0.0 ? 2 : 1)));
    const int64_t nb = (S.n_bins > 0 && S.m % S.n_bins == 0) ? S.n_bins : 0;
    if (vec_ok(k, 2, X, alpha != 0.0 ? (const void *)Y : nullptr, out))
        spmm_vec_kernel<double, false><<<(unsigned)ax_blocks(S.m, rows, nb, kAxViews), 256, 0, s>>>(
            S.m, S.n, k, S.sqrt_lambda, S.row_ptr, S.col, S.val, X, alpha, Y, beta, out, nb, kAxViews);
    else
        spmm_ax_kernel<double><<<blocks, 256, 0, s>>>(S.m, S.n, k, S.sqrt_lambda, S.row_ptr, S.col, S.val,
                                                      X, alpha, Y, beta, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status spmm_atr(const SparseSys &S, int64_t k, const double *R, double alpha, const double *Y,
                   double beta, double *out, cudaStream_t s) {
    if (S.n == 0 || k == 0) return CT_OK;
    const unsigned blocks = (unsigned)ceil_div(S.n * 32, 256);
    const int64_t rows = S.m + (S.sqrt_lambda > 0.0 ? S.n : 0);
    ProfScope prof(PROF_SPMM, s, 2.0 * (S.nnz + (rows - S.m)) * k,
                   12.0 * S.nnz + 8.0 * (double)k * (rows + S.n * (alpha != 0.0 ? 2 : 1)));
    const int64_t ns = (S.n_side > 0 && S.n_side * S.n_side == S.n) ? S.n_side : 0;
    if (vec_ok(k, 2, R, alpha != 0.0 ? (const void *)Y : nullptr, out))
        spmm_vec_kernel<double, true><<<(unsigned)atr_blocks(S.n, ns, kAtrWidth), 256, 0, s>>>(
            S.m, S.n, k, S.sqrt_lambda, S.col_ptr, S.csc_row, S.csc_val, R, alpha, Y, beta, out, ns, kAtrWidth);
    else
        spmm_atr_kernel<double><<<blocks, 256, 0, s>>>(S.m, S.n, k, S.sqrt_lambda, S.col_ptr, S.csc_row,
                                                       S.csc_val, R, alpha, Y, beta, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status spmm_ax32(const SparseSys &S, int64_t k, const float *X, float alpha, const float *Y,
                    float beta, float *out, cudaStream_t s) {
    const int64_t rows = S.m + (S.sqrt_lambda > 0.0 ? S.n : 0);
    if (rows == 0 || k == 0) return CT_OK;
    if (!S.val32) return CT_ERR_ARG;
    const unsigned blocks = (unsigned)ceil_div(rows * 32, 256);
    ProfScope prof(PROF_SPMM32, s, 2.0 * (S.nnz + (rows - S.m)) * k,
                   8.0 * S.nnz + 4.0 * (double)k * (S.n + rows * (alpha != 0.0f ? 2 : 1)));
    const int64_t nb = (S.n_bins > 0 && S.m % S.n_bins == 0) ? S.n_bins : 0;
    if (vec_ok(k, 4, X, alpha != 0.0f ? (const void *)Y : nullptr, out))
        spmm_vec_kernel<float, false><<<(unsigned)ax_blocks(S.m, rows, nb, kAxViews), 256, 0, s>>>(
            S.m, S.n, k, (float)S.sqrt_lambda, S.row_ptr, S.col, S.val32, X, alpha, Y, beta, out, nb, kAxViews);
    else
        spmm_ax_kernel<float><<<blocks, 256, 0, s>>>(S.m, S.n, k, (float)S.sqrt_lambda, S.row_ptr, S.col,
                                                     S.val32, X, alpha, Y, beta, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status spmm_atr32(const SparseSys &S, int64_t k, const float *R, float alpha, const float *Y,
                     float beta, float *out, cudaStream_t s) {
    if (S.n == 0 || k == 0) return CT_OK;
    if (!S.csc_val32) return CT_ERR_ARG;
    const unsigned blocks = (unsigned)ceil_div(S.n * 32, 256);
    const int64_t rows = S.m + (S.sqrt_lambda > 0.0 ? S.n : 0);
    ProfScope prof(PROF_SPMM32, s, 2.0 * (S.nnz + (rows - S.m)) * k,
                   8.0 * S.nnz + 4.0 * (double)k * (rows + S.n * (alpha != 0.0f ? 2 : 1)));
    const int64_t ns = (S.n_side > 0 && S.n_side * S.n_side == S.n) ? S.n_side : 0;
    if (vec_ok(k, 4, R, alpha != 0.0f ? (const void *)Y : nullptr, out))
        spmm_vec_kernel<float, true><<<(unsigned)atr_blocks(S.n, ns, kAtrWidth), 256, 0, s>>>(
            S.m, S.n, k, (float)S.sqrt_lambda, S.col_ptr, S.csc_row, S.csc_val32, R, alpha, Y, beta, out, ns,
            kAtrWidth);
    else
        spmm_atr_kernel<float><<<blocks, 256, 0, s>>>(S.m, S.n, k, (float)S.sqrt_lambda, S.col_ptr,
                                                      S.csc_row, S.csc_val32, R, alpha, Y, beta, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ctqr
