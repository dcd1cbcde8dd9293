// panel.cu -- panel factorisation of the blocked Householder QR (the
// 'dgeqrf' step of Sec. 2.1, Eq. 2), the unit-lower top block of V, and the
// T factor of the compact-WY block reflector.
//
// Panel: A[j0:M, j0:j0+nb] is split into G contiguous row slabs, one per CTA
// of a cooperative launch (G <= #SMs), each slab staged in shared memory for
// the whole panel when it fits.  For column c (global jc = j0 + c) every CTA
// accumulates, over its rows below the diagonal, the FP64 sum of squares of
// the column and the FP64 dot products of the column with the panel columns
// to its right; one grid barrier publishes the G partial vectors, and every
// CTA reduces them in the same order (identical reflector everywhere).
// With alpha = A[jc, jc]:
//     beta = -sign(alpha) * sqrt(alpha^2 + ss),  tau = (beta - alpha)/beta,
//     v = [1; x/(alpha - beta)],  and for each column k to the right
//     v^T a_k = a_k[jc] + d_k/(alpha - beta),  a_k <- a_k - tau (v^T a_k) v.
// If the column is already zero below the diagonal, tau = 0 (H = I).
// So one barrier per column suffices: the norm and the dot products come from
// the same pass over the data.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

constexpr int PANEL_THREADS = 256;
constexpr int PANEL_WARPS = PANEL_THREADS / 32;

// Bounded grid barrier (sense by generation counter).  Returns false if the
// wait expired or another CTA raised an error.
__device__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned G, DevStatus *st, int where) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vgen = gen;
        const unsigned my_gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == G - 1) {
            *((volatile unsigned *)count) = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            while (*vgen == my_gen) {
                __nanosleep(20);
                if ((++spins & 255u) == 0) {
                    if (*((volatile int *)&st->code) != 0) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > kWaitLimitNs) {
                        raise_status(st, DEV_TIMEOUT, where, 0);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T, int NB>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
    panel_qr_kernel(T *A, int64_t lda, int64_t M, int64_t j0, int nb, T *tau, double *partials,
                    double *rowbuf, unsigned *bar, DevStatus *st, int64_t rows_per, int use_smem) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ double red[PANEL_WARPS][NB + 1];
    __shared__ double tot[NB + 1];
    __shared__ double coef[NB];  // tau * (v^T a_k) for k > c
    __shared__ T coefs[NB];      // coef[k] / (alpha - beta), in the storage type
    __shared__ double scal_s, beta_s;
    __shared__ int skip_s;

    const unsigned G = gridDim.x;
    const int64_t r0 = j0 + (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(M, r0 + rows_per);
    const int64_t nloc = max((int64_t)0, r1 - r0);
    T *P;
    int64_t ldp;
    if (use_smem) {
        P = (T *)dsm;
        ldp = rows_per;
        for (int k = 0; k < nb; ++k)
            for (int64_t r = threadIdx.x; r < nloc; r += PANEL_THREADS)
                P[r + k * ldp] = A[(r0 + r) + (j0 + k) * lda];
        __syncthreads();
    } else {
        P = A + r0 + j0 * lda;
        ldp = lda;
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    for (int c = 0; c < nb; ++c) {
        const int64_t jc = j0 + c;
        const int par = c & 1;
        // ---- phase 1: partial sums over local rows strictly below jc ----
        double acc[NB + 1];
#pragma unroll
        for (int q = 0; q <= NB; ++q) acc[q] = 0.0;
        const int64_t rstart = max((int64_t)0, jc + 1 - r0);
        for (int64_t r = rstart + threadIdx.x; r < nloc; r += PANEL_THREADS) {
            const double x = (double)P[r + c * ldp];
            acc[0] += x * x;
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (k > c && k < nb) acc[1 + k] += x * (double)P[r + k * ldp];
        }
#pragma unroll
        for (int q = 0; q <= NB; ++q) {
            double v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][q] = v;
        }
        __syncthreads();
        double *my_part = partials + ((size_t)par * G + blockIdx.x) * (NB + 1);
        if (threadIdx.x <= NB) {
            double v = 0.0;
            for (int w = 0; w < PANEL_WARPS; ++w) v += red[w][threadIdx.x];
            my_part[threadIdx.x] = v;
        }
        // the owner of the diagonal row publishes that row (columns c..nb-1)
        if (jc >= r0 && jc < r1 && threadIdx.x < nb && threadIdx.x >= c)
            rowbuf[par * NB + threadIdx.x] = (double)P[(jc - r0) + threadIdx.x * ldp];
        if (!grid_barrier(bar, bar + 1, G, st, 10 + c)) return;
        // ---- phase 2: every CTA reduces the partials in the same order ----
        if (threadIdx.x <= NB) {
            double v = 0.0;
            const double *pp = partials + (size_t)par * G * (NB + 1) + threadIdx.x;
            for (unsigned b = 0; b < G; ++b) v += __ldcg(pp + (size_t)b * (NB + 1));
            tot[threadIdx.x] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double ss = tot[0];
            const double alpha = __ldcg(rowbuf + par * NB + c);
            if (!isfinite(ss) || !isfinite(alpha)) raise_status(st, DEV_NONFINITE, 20, (int)jc);
            if (ss == 0.0) {
                skip_s = 1;
                if (blockIdx.x == 0) tau[jc] = T(0);
            } else {
                skip_s = 0;
                const double norm = sqrt(alpha * alpha + ss);
                const double beta = (alpha >= 0.0) ? -norm : norm;
                const double t = (beta - alpha) / beta;
                const double scale = 1.0 / (alpha - beta);
                scal_s = scale;
                beta_s = beta;
                if (blockIdx.x == 0) tau[jc] = (T)t;
                for (int k = c + 1; k < nb; ++k) {
                    const double ak = __ldcg(rowbuf + par * NB + k);
                    coef[k] = t * (ak + scale * tot[1 + k]);
                    coefs[k] = (T)(coef[k] * scale);
                }
            }
        }
        __syncthreads();
        if (skip_s) continue;
        const double scale = scal_s;
        // rows strictly below the diagonal: a_rk -= coef_k * scale * x_r ; x_r <- scale*x_r
        for (int64_t r = rstart + threadIdx.x; r < nloc; r += PANEL_THREADS) {
            const T x = P[r + c * ldp];
            for (int k = c + 1; k < nb; ++k) P[r + k * ldp] -= coefs[k] * x;
            P[r + c * ldp] = (T)(scale * (double)x);
        }
        // the diagonal row: a_k[jc] -= coef_k ; A[jc, jc] = beta
        if (jc >= r0 && jc < r1) {
            const int64_t rl = jc - r0;
            for (int k = c + 1 + threadIdx.x; k < nb; k += PANEL_THREADS)
                P[rl + k * ldp] -= (T)coef[k];
            if (threadIdx.x == 0) P[rl + c * ldp] = (T)beta_s;
        }
        __syncthreads();
    }
    if (use_smem) {
        __syncthreads();
        for (int k = 0; k < nb; ++k)
            for (int64_t r = threadIdx.x; r < nloc; r += PANEL_THREADS)
                A[(r0 + r) + (j0 + k) * lda] = P[r + k * ldp];
    }
}

template <typename T>
__global__ void extract_vtop_kernel(const T *A, int64_t lda, int64_t j0, int nb, T *Vt, int64_t ldv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;  // row
    int j = blockIdx.y;                              // col
    if (i >= nb) return;
    T v;
    if (i == j) v = T(1);
    else if (i < j) v = T(0);
    else v = A[(j0 + i) + (j0 + j) * lda];
    Vt[i + (int64_t)j * ldv] = v;
}

// Forward, columnwise T of H_0 H_1 ... H_{nb-1} = I - V T V^T:
//   T[j, j] = tau_j,  T[0:j, j] = -tau_j * T[0:j, 0:j] * G[0:j, j],  G = V^T V.
template <typename T>
__global__ void larft_kernel(int nb, const T *G, int64_t ldg, const T *tau, T *Tm, int64_t ldt) {
    extern __shared__ double gcol[];
    for (int j = 0; j < nb; ++j) {
        for (int i = threadIdx.x; i < j; i += blockDim.x) gcol[i] = (double)G[i + (int64_t)j * ldg];
        __syncthreads();
        const double tj = (double)tau[j];
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            double y = 0.0;
            if (i < j)
                for (int l = i; l < j; ++l) y += (double)Tm[i + (int64_t)l * ldt] * gcol[l];
            T out;
            if (i < j) out = (T)(-tj * y);
            else if (i == j) out = (T)tj;
            else out = T(0);
            Tm[i + (int64_t)j * ldt] = out;
        }
        __syncthreads();
    }
}

template <typename T, int NB>
ct_status panel_launch(T *A, int64_t lda, int64_t M, int64_t j0, int nb, T *tau, Scratch &ws,
                       cudaStream_t s) {
    const int64_t rows = M - j0;
    const int sms = num_sms();
    int G = (int)std::min<int64_t>(sms, std::max<int64_t>(1, ceil_div(rows, 256)));
    int64_t rows_per = ceil_div(rows, G);
    G = (int)ceil_div(rows, rows_per);
    const size_t slab = (size_t)rows_per * nb * sizeof(T);
    const int use_smem = slab <= 200 * 1024 ? 1 : 0;
    const size_t dyn = use_smem ? slab : 0;
    static bool attr[2] = {false, false};
    auto fn = panel_qr_kernel<T, NB>;
    if (!attr[NB == 32]) {
        CT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr[NB == 32] = true;
    }
    int per_sm = 0;
    CT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PANEL_THREADS, dyn));
    if (per_sm * sms < G) {
        set_error("panel: cooperative grid %d does not fit (%d per SM)", G, per_sm);
        return CT_ERR_CUDA;
    }
    // workspace: barrier words | partials [2][G][NB+1] | rowbuf [2][NB]
    const size_t need = 256 + sizeof(double) * (2 * (size_t)G * (NB + 1) + 2 * NB);
    CT_TRY(ws.ensure(need));
    unsigned *bar = (unsigned *)ws.ptr;
    double *partials = (double *)((char *)ws.ptr + 256);
    double *rowbuf = partials + 2 * (size_t)G * (NB + 1);
    CT_CUDA(cudaMemsetAsync(bar, 0, 256, s));
    DevStatus *st = device_status();
    void *args[] = {&A, &lda, &M, &j0, &nb, &tau, &partials, &rowbuf, &bar, &st, &rows_per,
                    (void *)&use_smem};
    CT_CUDA(cudaLaunchCooperativeKernel((const void *)fn, dim3(G), dim3(PANEL_THREADS), args, dyn, s));
    return CT_OK;
}

}  // namespace

ct_status panel_qr(bool fp64, void *A, int64_t lda, int64_t M, int64_t j0, int nb, void *tau,
                   Scratch &ws, cudaStream_t s) {
    if (nb <= 0 || nb > 32 || M - j0 < 1) return CT_ERR_ARG;
    if (fp64) {
        if (nb <= 16) return panel_launch<double, 16>((double *)A, lda, M, j0, nb, (double *)tau, ws, s);
        return panel_launch<double, 32>((double *)A, lda, M, j0, nb, (double *)tau, ws, s);
    }
    if (nb <= 16) return panel_launch<float, 16>((float *)A, lda, M, j0, nb, (float *)tau, ws, s);
    return panel_launch<float, 32>((float *)A, lda, M, j0, nb, (float *)tau, ws, s);
}

ct_status extract_vtop(bool fp64, const void *A, int64_t lda, int64_t j0, int nb, void *Vtop,
                       int64_t ldv, cudaStream_t s) {
    dim3 grid((unsigned)ceil_div(nb, 128), (unsigned)nb);
    if (fp64)
        extract_vtop_kernel<double><<<grid, 128, 0, s>>>((const double *)A, lda, j0, nb, (double *)Vtop, ldv);
    else
        extract_vtop_kernel<float><<<grid, 128, 0, s>>>((const float *)A, lda, j0, nb, (float *)Vtop, ldv);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status larft_from_gram(bool fp64, int nb, const void *G, int64_t ldg, const void *tau, void *T,
                          int64_t ldt, cudaStream_t s) {
    const int threads = std::min(1024, std::max(32, nb));
    const size_t smem = sizeof(double) * nb;
    if (fp64)
        larft_kernel<double><<<1, threads, smem, s>>>(nb, (const double *)G, ldg,
                                                      (const double *)tau, (double *)T, ldt);
    else
        larft_kernel<float><<<1, threads, smem, s>>>(nb, (const float *)G, ldg, (const float *)tau,
                                                     (float *)T, ldt);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ctqr
