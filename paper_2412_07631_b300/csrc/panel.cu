// panel.cu -- panel factorisation of the blocked Householder QR (the
// 'dgeqrf' step of Sec. 2.1, Eq. 2), the unit-lower top block of V, and the
// T factor of the compact-WY block reflector.
//
// Panel: A[j0:M, j0:j0+nb] is split into G contiguous row slabs, one per CTA
// of a cooperative launch (G <= #SMs), each slab staged in shared memory for
// the whole panel when it fits.  For column c (global jc = j0 + c) every CTA
// accumulates, over its rows below the diagonal, the FP64 sum of squares of
// the column and the dot products of the column with the panel columns to its
// right (storage type); one flag-based exchange publishes the G partial
// vectors, and every CTA reduces them in the same order (identical reflector
// everywhere).
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

// Reduce-scatter over a warp: on entry every lane holds 32 values; on exit
// lane l returns the warp-wide sum of value l (31 shuffles in all).
template <typename D>
__device__ __forceinline__ D warp_reduce_scatter32(D (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const D send = upper ? v[i] : v[i + o];
            const D keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exchange area (global): flags[2][G] epoch words; sums of squares
// ssq[2][G] (FP64); dot products dots[2][32][G] (storage type); the
// diagonal row rowbuf[2][32] (FP64).  Index [c & 1] alternates between
// columns.
//
// Per column c (jc = j0 + c) each CTA forms, over its rows strictly below
// jc, the sum of squares of column c -- in FP64 from the first product
// (the square of a storage value is exact in FP64) -- and the dot products
// of column c with the columns k > c in the storage type (FP64 FMA runs at a
// small fraction of the FP32 rate on this part, so only the norm uses it).
// It stores them, the owner of row jc also stores that row, and a fence
// followed by a store of epoch jc+1 to the CTA's flag publishes them.  Warp 0
// of every CTA polls all G flags (bounded), fences, and then every CTA
// reduces the G partials in the same order.
template <typename T, int NB>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
    panel_qr_kernel(T *A, int64_t lda, int64_t M, int64_t j0, int nb, T *tau, double *ssq,
                    T *dots, double *rowbuf, unsigned *flags, DevStatus *st, int64_t rows_per,
                    int use_smem) {
    static_assert(NB <= 32, "panel width");
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ T red[PANEL_WARPS][32];
    __shared__ double red_ss[PANEL_WARPS];
    __shared__ T tot[32];
    __shared__ double tot_ss;
    __shared__ double coef[32];  // tau * (v^T a_k) for k > c
    __shared__ T coefs[32];      // coef[k] / (alpha - beta), in the storage type
    __shared__ double scal_s, beta_s, tau_s;
    __shared__ T scal_t;
    __shared__ int skip_s, ok_s;

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
        const unsigned epoch = (unsigned)(jc + 1);
        double *my_ssq = ssq + (size_t)par * G;
        T *my_dots = dots + (size_t)par * 32 * G;
        unsigned *flg = flags + (size_t)par * G;
        // ---- phase 1: partial sums over local rows strictly below jc ----
        double ss = 0.0;
        T acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = T(0);
        const int64_t rstart = max((int64_t)0, jc + 1 - r0);
        if (nb == NB) {
            // Full-width panel: every column exists, so the products with the
            // already-factored columns k <= c are formed too (and ignored) --
            // a loop without per-column predicates runs several times faster.
            for (int64_t r = rstart + threadIdx.x; r < nloc; r += PANEL_THREADS) {
                const T xv = P[r + c * ldp];
                const double xd = (double)xv;
                ss += xd * xd;
#pragma unroll
                for (int k = 0; k < NB; ++k) acc[k] += xv * P[r + k * ldp];
            }
        } else {
            for (int64_t r = rstart + threadIdx.x; r < nloc; r += PANEL_THREADS) {
                const T xv = P[r + c * ldp];
                const double xd = (double)xv;
                ss += xd * xd;
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (k > c && k < nb) acc[k] += xv * P[r + k * ldp];
            }
        }
        red[warp][lane] = warp_reduce_scatter32<T>(acc, lane);
        ss = warp_sum(ss);
        if (lane == 0) red_ss[warp] = ss;
        __syncthreads();
        if (threadIdx.x < 32) {
            T v = T(0);
#pragma unroll
            for (int w = 0; w < PANEL_WARPS; ++w) v += red[w][threadIdx.x];
            my_dots[(size_t)threadIdx.x * G + blockIdx.x] = v;
            if (threadIdx.x == 0) {
                double v2 = 0.0;
#pragma unroll
                for (int w = 0; w < PANEL_WARPS; ++w) v2 += red_ss[w];
                my_ssq[blockIdx.x] = v2;
            }
        }
        if (jc >= r0 && jc < r1 && threadIdx.x < nb && threadIdx.x >= c)
            rowbuf[par * 32 + threadIdx.x] = (double)P[(jc - r0) + threadIdx.x * ldp];
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();  // orders this CTA's partials and row before the flag
            *((volatile unsigned *)(flg + blockIdx.x)) = epoch;
        }
        // ---- wait until every CTA has published column c (bounded) ----
        if (warp == 0) {
            const uint64_t t0 = globaltimer_ns();
            int ok = 1;
            uint32_t spins = 0;
            while (true) {
                bool mine = true;
                for (unsigned b = lane; b < G; b += 32)
                    mine = mine && (*((volatile const unsigned *)(flg + b)) == epoch);
                if (__all_sync(0xffffffffu, mine)) break;
                if ((++spins & 63u) == 0) {
                    int bad = 0;
                    if (lane == 0) {
                        if (*((volatile int *)&st->code) != 0) bad = 1;
                        else if (globaltimer_ns() - t0 > kWaitLimitNs) {
                            raise_status(st, DEV_TIMEOUT, 10, (int)jc);
                            bad = 1;
                        }
                    }
                    if (__shfl_sync(0xffffffffu, bad, 0)) { ok = 0; break; }
                }
            }
            __threadfence();  // orders the flag reads before the reads of the partials
            if (lane == 0) ok_s = ok;
        }
        __syncthreads();
        if (!ok_s) return;
        // ---- phase 2: every CTA reduces the G partials in the same order ----
        {
            T v[32 / PANEL_WARPS];
#pragma unroll
            for (int qq = 0; qq < 32 / PANEL_WARPS; ++qq) v[qq] = T(0);
            for (unsigned b = lane; b < G; b += 32) {
#pragma unroll
                for (int qq = 0; qq < 32 / PANEL_WARPS; ++qq)
                    v[qq] += __ldcg(my_dots + (size_t)(warp + PANEL_WARPS * qq) * G + b);
            }
#pragma unroll
            for (int qq = 0; qq < 32 / PANEL_WARPS; ++qq) {
                T x = v[qq];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) tot[warp + PANEL_WARPS * qq] = x;
            }
            if (warp == PANEL_WARPS - 1) {
                double x = 0.0;
                for (unsigned b = lane; b < G; b += 32) x += __ldcg(my_ssq + b);
                x = warp_sum(x);
                if (lane == 0) tot_ss = x;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double ssum = tot_ss;
            const double alpha = __ldcg(rowbuf + par * 32 + c);
            if (!isfinite(ssum) || !isfinite(alpha)) raise_status(st, DEV_NONFINITE, 20, (int)jc);
            if (ssum == 0.0) {
                skip_s = 1;
                if (blockIdx.x == 0) tau[jc] = T(0);
            } else {
                skip_s = 0;
                const double norm = sqrt(alpha * alpha + ssum);
                const double beta = (alpha >= 0.0) ? -norm : norm;
                const double t = (beta - alpha) / beta;
                scal_s = 1.0 / (alpha - beta);
                scal_t = (T)scal_s;
                beta_s = beta;
                tau_s = t;
                if (blockIdx.x == 0) tau[jc] = (T)t;
            }
        }
        __syncthreads();
        if (!skip_s && threadIdx.x < 32) {
            const int k = threadIdx.x;
            if (k > c && k < nb) {
                coef[k] = tau_s * (__ldcg(rowbuf + par * 32 + k) + scal_s * (double)tot[k]);
                coefs[k] = (T)(coef[k] * scal_s);
            } else {
                coef[k] = 0.0;
                coefs[k] = T(0);
            }
        }
        __syncthreads();
        if (skip_s) continue;
        const T scale_t = scal_t;
        // rows strictly below the diagonal: a_rk -= coef_k * scale * x_r ; x_r <- scale*x_r
        if (nb == NB) {
            // coefs[k] = 0 for k <= c, so the unpredicated update leaves those
            // columns as they are (column c is rewritten just after).
            for (int64_t r = rstart + threadIdx.x; r < nloc; r += PANEL_THREADS) {
                const T x = P[r + c * ldp];
#pragma unroll
                for (int k = 0; k < NB; ++k) P[r + k * ldp] -= coefs[k] * x;
                P[r + c * ldp] = x * scale_t;
            }
        } else {
            for (int64_t r = rstart + threadIdx.x; r < nloc; r += PANEL_THREADS) {
                const T x = P[r + c * ldp];
                for (int k = c + 1; k < nb; ++k) P[r + k * ldp] -= coefs[k] * x;
                P[r + c * ldp] = x * scale_t;
            }
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

// ---- register-resident variant (FP32, full 32-column panels) ----------------
//
// Same reflectors as panel_qr_kernel, for slabs of up to RPT rows per thread
// (RPT x 256 rows per CTA): each thread keeps its RPT rows of the 32 panel
// columns in registers for the whole panel, so the per-column passes touch
// no shared memory.  Per column, every CTA writes its partial record (dot
// products, sum of squares, and the diagonal row if it owns it), fences, and
// takes a ticket from a counter; the CTA that draws the last ticket sums the
// G records in a fixed order (records split over its warps by index, then
// the warps in order) and publishes the totals as self-validating words
// (epoch << 32 | 32 value bits), which every CTA polls without a fence.  One
// reducer and one published total replace G x G reads of partials, and the
// fixed order keeps the reflector identical in every CTA and run.  The norm
// is accumulated per thread in FP64 and summed across threads in FP32; the
// reflector scalars are FP32 (beta - alpha and alpha - beta never cancel).
constexpr int RP_THREADS = 256;
constexpr int RP_WARPS = RP_THREADS / 32;
constexpr int RP_REC = 72;   // partial record: dots[32] | row[32] | ss  (floats, padded)
constexpr int RP_TOT = 72;   // total record (64-bit words): dots[32] | row[32] | ss
constexpr int RP_MAX_PER_WARP = 19;  // records per warp of the reducing CTA: G <= 152
// leading bytes of the column-by-column kernel's workspace that must be zero
// at launch: the totals [2][RP_TOT] words and the counters (256 bytes)
constexpr size_t regs_zero_bytes() { return sizeof(uint64_t) * 2 * RP_TOT + 256; }

__device__ __forceinline__ void st_word(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_word(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t tag(unsigned epoch, float v) {
    return ((uint64_t)epoch << 32) | __float_as_uint(v);
}

// After a fallback column sweep (the Gram kernel declined the panel), the
// T_p of the panel's block reflector and the unit-lower top of its V, which
// the Gram kernel would otherwise have written: each CTA forms the partial
// V^T V of its rows (read back from A, the top rows as unit lower, rolled
// loops: this path is rare), takes a ticket, and the last CTA sums the
// partials in a fixed order and runs the forward columnwise T recurrence
// T[j, j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j].
__device__ __noinline__ void fallback_t(const float *A, int64_t lda, int64_t j0, int64_t r0, int64_t nloc,
                                        const float *tau, float *Tp, float *Vtp, int64_t ldt, float *trec,
                                        unsigned *tcount) {
    __shared__ double gs[32][33];
    __shared__ int last;
    constexpr int NTRI = 528;
    for (int e = threadIdx.x; e < NTRI; e += RP_THREADS) {
        int j = 0;
        while ((j + 1) * (j + 2) / 2 <= e) ++j;
        const int i = e - j * (j + 1) / 2;  // i <= j
        float acc = 0.0f;
        for (int64_t lr = 0; lr < nloc; ++lr) {
            const int64_t gr = r0 + lr, r = gr - j0;
            const float vi = (r > i) ? A[gr + (j0 + i) * lda] : (r == i ? 1.0f : 0.0f);
            const float vj = (r > j) ? A[gr + (j0 + j) * lda] : (r == j ? 1.0f : 0.0f);
            acc = fmaf(vi, vj, acc);
        }
        trec[(size_t)blockIdx.x * NTRI + e] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(tcount, 1u) == gridDim.x - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;
    for (int e = threadIdx.x; e < NTRI; e += RP_THREADS) {
        int j = 0;
        while ((j + 1) * (j + 2) / 2 <= e) ++j;
        const int i = e - j * (j + 1) / 2;
        double v = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) v += (double)__ldcg(trec + (size_t)b * NTRI + e);
        gs[i][j] = v;
        gs[j][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // lane i owns row i of T
        __shared__ float ts[32][33];
        const int lane = threadIdx.x;
        for (int j = 0; j < 32; ++j) {
            const float tj = __ldcg(tau + j0 + j);
            double y = 0.0;
            for (int l = lane; l < j; ++l) y += (double)ts[lane][l] * gs[l][j];
            ts[lane][j] = (lane < j) ? (float)(-(double)tj * y) : (lane == j ? tj : 0.0f);
        }
        __syncwarp();
        for (int k = 0; k < 32; ++k) {
            Tp[lane + k * ldt] = ts[lane][k];
            Vtp[lane + k * ldt] = (lane == k) ? 1.0f : (lane > k ? __ldcg(A + (j0 + lane) + (j0 + k) * lda) : 0.0f);
        }
    }
}

template <int RPT>
__global__ void __launch_bounds__(RP_THREADS, 1)
    panel_qr_regs_kernel(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, float *rec,
                         uint64_t *tot, unsigned *counter, DevStatus *st, int64_t rows_per,
                         const int *only_if, float *Tp, float *Vtp, int64_t ldt, float *trec,
                         unsigned *tcount, uint8_t *V16, int64_t ld16) {
    // after the Gram-based kernel: run only if it declined this panel
    if (only_if != nullptr && *only_if == 0) return;
    __shared__ float red[RP_WARPS][32];
    __shared__ float red_ss[RP_WARPS];
    __shared__ float rowsm[32];
    __shared__ float coefs_sm[32];
    __shared__ float coef_row[32];
    __shared__ float scal_sm, beta_sm;
    __shared__ int skip_sm, ok_sm, last_sm;

    const unsigned G = gridDim.x;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t r0 = j0 + (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(M, r0 + rows_per);
    const int64_t nloc = max((int64_t)0, r1 - r0);

    float a[RPT][32];
    float xc[RPT];  // column c of each row
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t lr = threadIdx.x + (int64_t)i * RP_THREADS;
#pragma unroll
        for (int k = 0; k < 32; ++k) a[i][k] = (lr < nloc) ? A[(r0 + lr) + (j0 + k) * lda] : 0.0f;
    }
    if (threadIdx.x == 0) ok_sm = 1;
    __syncthreads();

    for (int c = 0; c < 32; ++c) {
        const int64_t jc = j0 + c;
        const int par = c & 1;
        const unsigned epoch = (unsigned)(jc + 1);
        float *rec_par = rec + (size_t)par * G * RP_REC;
        uint64_t *tot_par = tot + (size_t)par * RP_TOT;
        // ---- local partials over rows strictly below jc ----
        float acc[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = 0.0f;
        double ssd = 0.0;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            float xv = 0.0f;
#pragma unroll
            for (int k = 0; k < 32; ++k) xv = (k == c) ? a[i][k] : xv;
            xc[i] = xv;
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int64_t lr = threadIdx.x + (int64_t)i * RP_THREADS;
            const int64_t gr = r0 + lr;
            if (lr < nloc && gr > jc) {
                const float x = xc[i];
                ssd += (double)x * (double)x;
#pragma unroll
                for (int k = 0; k < 32; ++k) acc[k] += x * a[i][k];
            }
            if (lr < nloc && gr == jc) {
#pragma unroll
                for (int k = 0; k < 32; ++k) rowsm[k] = a[i][k];
            }
        }
        red[warp][lane] = warp_reduce_scatter32<float>(acc, lane);
        float ss = (float)ssd;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) red_ss[warp] = ss;
        __syncthreads();
        const bool owner = jc >= r0 && jc < r1;
        const unsigned b_own = (unsigned)((jc - j0) / rows_per);
        // ---- publish the partial record, take a ticket ----
        if (warp == 0) {
            float v = 0.0f;
#pragma unroll
            for (int w = 0; w < RP_WARPS; ++w) v += red[w][lane];
            float *mine = rec_par + (size_t)blockIdx.x * RP_REC;
            mine[lane] = v;
            if (owner) mine[32 + lane] = rowsm[lane];
            if (lane == 0) {
                float t = 0.0f;
#pragma unroll
                for (int w = 0; w < RP_WARPS; ++w) t += red_ss[w];
                mine[64] = t;
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence();  // the record before the ticket
                const unsigned ticket = atomicAdd(counter + par, 1u);
                last_sm = ticket == G - 1;
                if (ticket == G - 1) __threadfence();  // every record before the reads below
            }
        }
        __syncthreads();
        if (last_sm) {
            // ---- the last CTA sums the G records in a fixed order ----
            // all loads of a warp's records are issued before the first add
            float dv[RP_MAX_PER_WARP], sv2[RP_MAX_PER_WARP];
#pragma unroll
            for (int q = 0; q < RP_MAX_PER_WARP; ++q) {
                const unsigned b = warp + q * RP_WARPS;
                const float *r = rec_par + (size_t)b * RP_REC;
                dv[q] = (b < G) ? __ldcg(r + lane) : 0.0f;
                sv2[q] = (b < G && lane == 0) ? __ldcg(r + 64) : 0.0f;
            }
            float v = 0.0f, sv = 0.0f;
#pragma unroll
            for (int q = 0; q < RP_MAX_PER_WARP; ++q) {
                v += dv[q];
                sv += sv2[q];
            }
            red[warp][lane] = v;
            if (lane == 0) red_ss[warp] = sv;
            __syncthreads();
            if (warp == 0) {
                float t = 0.0f, ts = 0.0f;
#pragma unroll
                for (int w = 0; w < RP_WARPS; ++w) {
                    t += red[w][lane];
                    ts += red_ss[w];
                }
                const float rowv = __ldcg(rec_par + (size_t)b_own * RP_REC + 32 + lane);
                if (lane == 0) counter[par] = 0u;  // no CTA takes a ticket for this parity before the total
                st_word(tot_par + lane, tag(epoch, t));
                st_word(tot_par + 32 + lane, tag(epoch, rowv));
                if (lane == 0) st_word(tot_par + 64, tag(epoch, ts));
            }
        }
        // ---- every CTA reads the published totals (warp 0, bounded) ----
        if (warp == 0) {
            const uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            uint64_t wd, wr, ws;
            while (true) {
                wd = ld_word(tot_par + lane);
                wr = ld_word(tot_par + 32 + lane);
                ws = ld_word(tot_par + 64);
                const bool here = (unsigned)(wd >> 32) == epoch && (unsigned)(wr >> 32) == epoch &&
                                  (unsigned)(ws >> 32) == epoch;
                if (__all_sync(0xffffffffu, here)) break;
                if ((++spins & 15u) == 0) {
                    int bad = 0;
                    if (lane == 0) {
                        if (*((volatile int *)&st->code) != 0) bad = 1;
                        else if (globaltimer_ns() - t0 > kWaitLimitNs) {
                            raise_status(st, DEV_TIMEOUT, 21, (int)jc);
                            bad = 1;
                        }
                    }
                    if (__shfl_sync(0xffffffffu, bad, 0)) {
                        if (lane == 0) ok_sm = 0;
                        break;
                    }
                }
            }
            if (ok_sm) {
                // ---- reflector scalars and coefficients (FP32) ----
                const float totk = __uint_as_float((uint32_t)wd);
                const float rowk = __uint_as_float((uint32_t)wr);
                const float ssum = __uint_as_float((uint32_t)ws);
                const float alpha = __shfl_sync(0xffffffffu, rowk, c);
                if (lane == 0 && (!isfinite(ssum) || !isfinite(alpha))) raise_status(st, DEV_NONFINITE, 23, (int)jc);
                if (ssum == 0.0f) {
                    if (lane == 0) {
                        skip_sm = 1;
                        if (blockIdx.x == 0) tau[jc] = 0.0f;
                    }
                } else {
                    const float norm = sqrtf(fmaf(alpha, alpha, ssum));
                    const float beta = (alpha >= 0.0f) ? -norm : norm;
                    const float t = (beta - alpha) / beta;
                    const float scal = 1.0f / (alpha - beta);
                    const float cf = (lane > c) ? t * fmaf(scal, totk, rowk) : 0.0f;
                    coef_row[lane] = cf;
                    coefs_sm[lane] = cf * scal;
                    if (lane == 0) {
                        skip_sm = 0;
                        scal_sm = scal;
                        beta_sm = beta;
                        if (blockIdx.x == 0) tau[jc] = t;
                    }
                }
            }
        }
        __syncthreads();
        if (!ok_sm) return;
        if (skip_sm) continue;
        // ---- update the rows in registers ----
        {
            const float scal_t = scal_sm, beta_t = beta_sm;
            // rows below the diagonal: a_k -= coefs_k x, column c <- scal x;
            // the diagonal row: a_k -= coef_k, column c <- beta; others as they are.
            // Branch-free: m1 = x below the diagonal (else 0), m2 = 1 on the
            // diagonal row (else 0); cs and cr are 0 for k <= c.
            float m1[RPT], m2[RPT], newc[RPT];
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int64_t lr = threadIdx.x + (int64_t)i * RP_THREADS;
                const int64_t gr = r0 + lr;
                const bool below = lr < nloc && gr > jc, diag = lr < nloc && gr == jc;
                m1[i] = below ? xc[i] : 0.0f;
                m2[i] = diag ? 1.0f : 0.0f;
                newc[i] = below ? xc[i] * scal_t : (diag ? beta_t : xc[i]);
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float cs = coefs_sm[k], cr = coef_row[k];
#pragma unroll
                for (int i = 0; i < RPT; ++i)
                    a[i][k] = (k == c) ? newc[i] : fmaf(-cr, m2[i], fmaf(-cs, m1[i], a[i][k]));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t lr = threadIdx.x + (int64_t)i * RP_THREADS;
        if (lr < nloc) {
#pragma unroll
            for (int k = 0; k < 32; ++k) A[(r0 + lr) + (j0 + k) * lda] = a[i][k];
            const int64_t gr = r0 + lr;
            if (V16 != nullptr && gr >= j0 + 32) store_bf16_row32(V16 + 2 * (size_t)((gr - j0 - 32) * ld16), a[i]);
        }
    }
    if (only_if != nullptr && Tp != nullptr) fallback_t(A, lda, j0, r0, nloc, tau, Tp, Vtp, ldt, trec, tcount);
}

template <int RPT>
ct_status panel_regs_launch(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, char *wsp,
                            int G, int64_t rows_per, const int *only_if, float *Tp, float *Vtp, int64_t ldt,
                            float *trec, unsigned *tcount, void *V16, int64_t ld16, cudaStream_t s) {
    const int64_t rows = M - j0;
    auto fn = panel_qr_regs_kernel<RPT>;
    int per_sm = 0;
    CT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RP_THREADS, 0));
    if (per_sm * num_sms() < G) {
        set_error("panel: cooperative grid %d does not fit (%d per SM)", G, per_sm);
        return CT_ERR_CUDA;
    }
    // workspace (regs_ws_bytes): totals [2][RP_TOT] words | counters [2] | records [2][G][RP_REC]
    // floats; the caller has zeroed the first regs_zero_bytes() on the stream
    uint64_t *tot = (uint64_t *)wsp;
    unsigned *counter = (unsigned *)(wsp + regs_zero_bytes() - 256);
    float *rec = (float *)(wsp + regs_zero_bytes());
    DevStatus *st = device_status();
    uint8_t *v16 = (uint8_t *)V16;
    void *args[] = {&A,         &lda, &M,   &j0,   &tau,  &rec,  &tot,    &counter,
                    &st,        &rows_per, (void *)&only_if, &Tp, &Vtp, &ldt, &trec, &tcount, &v16, &ld16};
    ProfScope prof(PROF_PANEL, s, 2.0 * rows * 32 * 32, 2.0 * sizeof(float) * rows * 32, rows, 32, G,
                   2 + RPT);
    CT_CUDA(cudaLaunchCooperativeKernel((const void *)fn, dim3(G), dim3(RP_THREADS), args, 0, s));
    count_launch();
    return CT_OK;
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
    static PerContextOnce attr;  // per instantiation; the attribute belongs to each device's context
    auto fn = panel_qr_kernel<T, NB>;
    CT_CUDA(attr.run([&] { return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); }));
    int per_sm = 0;
    CT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PANEL_THREADS, dyn));
    if (per_sm * sms < G) {
        set_error("panel: cooperative grid %d does not fit (%d per SM)", G, per_sm);
        return CT_ERR_CUDA;
    }
    // workspace: flags [2][G] | ssq [2][G] | rowbuf [2][32] | dots [2][32][G]
    const size_t flag_bytes = round_up(sizeof(unsigned) * 2 * G, 256);
    const size_t ssq_bytes = round_up(sizeof(double) * (2 * (size_t)G + 64), 256);
    const size_t need = flag_bytes + ssq_bytes + sizeof(T) * 2 * 32 * (size_t)G;
    CT_TRY(ws.ensure(need));
    unsigned *flags = (unsigned *)ws.ptr;
    double *ssq = (double *)((char *)ws.ptr + flag_bytes);
    double *rowbuf = ssq + 2 * (size_t)G;
    T *dots = (T *)((char *)ws.ptr + flag_bytes + ssq_bytes);
    CT_CUDA(cudaMemsetAsync(flags, 0, flag_bytes, s));
    DevStatus *st = device_status();
    void *args[] = {&A, &lda, &M, &j0, &nb, &tau, &ssq, &dots, &rowbuf, &flags, &st, &rows_per,
                    (void *)&use_smem};
    ProfScope prof(PROF_PANEL, s, 2.0 * rows * nb * nb, 2.0 * sizeof(T) * rows * nb, rows, nb, G,
                   use_smem);
    CT_CUDA(cudaLaunchCooperativeKernel((const void *)fn, dim3(G), dim3(PANEL_THREADS), args, dyn, s));
    count_launch();
    return CT_OK;
}

}  // namespace

size_t regs_ws_bytes(int G) {
    return regs_zero_bytes() + sizeof(float) * 2 * (size_t)G * RP_REC;
}

ct_status panel_qr(bool fp64, void *A, int64_t lda, int64_t M, int64_t j0, int nb, void *tau,
                   Scratch &ws, cudaStream_t s, bool use_gram, void *Tp, void *Vtp, int64_t ldt,
                   bool *made_t, void *V16, int64_t ld16, bool *made_v16) {
    if (made_t) *made_t = false;
    if (made_v16) *made_v16 = false;
    if (V16 != nullptr && (((uintptr_t)V16 & 15) || (ld16 & 7))) return CT_ERR_ARG;
    if (nb <= 0 || nb > 32 || M - j0 < 1) return CT_ERR_ARG;
    if (fp64) {
        if (nb <= 16) return panel_launch<double, 16>((double *)A, lda, M, j0, nb, (double *)tau, ws, s);
        return panel_launch<double, 32>((double *)A, lda, M, j0, nb, (double *)tau, ws, s);
    }
    if (nb <= 16) return panel_launch<float, 16>((float *)A, lda, M, j0, nb, (float *)tau, ws, s);
    if (nb == 32) {
        // register-resident slabs when each CTA's share fits 4 rows per thread
        const int64_t rows = M - j0;
        int G = (int)std::min<int64_t>(num_sms(), std::max<int64_t>(1, ceil_div(rows, 256)));
        int64_t rows_per = ceil_div(rows, G);
        G = (int)ceil_div(rows, rows_per);
        const int64_t rpt = ceil_div(rows_per, RP_THREADS);
        if (rows >= 32 && rpt <= 4 && G <= RP_WARPS * RP_MAX_PER_WARP) {
            // workspace: fallback flag, T counter, Gram grid-meet counters | column-by-column
            // kernel | Gram kernel | partial Gram records of a fallback's T.  One memset
            // zeroes every flag and counter of both kernels.
            const size_t rb = round_up((int64_t)regs_ws_bytes(G), 256);
            const size_t gb = round_up((int64_t)panel_gram_ws_bytes(G), 256);
            CT_TRY(ws.ensure(256 + rb + gb + sizeof(float) * 528 * (size_t)G));
            int *fallback = (int *)ws.ptr;
            unsigned *tcount = (unsigned *)((char *)ws.ptr + 64);
            unsigned *gbar = (unsigned *)((char *)ws.ptr + 128);
            char *wr = (char *)ws.ptr + 256;
            float *trec = (float *)(wr + rb + gb);
            const int *only_if = nullptr;
            const bool want_t = use_gram && Tp != nullptr && Vtp != nullptr;
            CT_CUDA(cudaMemsetAsync(ws.ptr, 0, 256 + regs_zero_bytes(), s));
            if (use_gram) {
                ProfScope prof(PROF_PANEL, s, 4.0 * rows * 32 * 32, 2.0 * sizeof(float) * rows * 32, rows, 32,
                               G, 10 + (int)rpt);
                CT_TRY(panel_gram((float *)A, lda, M, j0, (float *)tau, wr + rb, gbar, G, rows_per, (int)rpt,
                                  fallback, want_t ? (float *)Tp : nullptr, (float *)Vtp, ldt, V16, ld16, s));
                only_if = fallback;
            }
            float *tp = want_t ? (float *)Tp : nullptr;
            float *vp = want_t ? (float *)Vtp : nullptr;
            ct_status st;
            if (rpt <= 1) st = panel_regs_launch<1>((float *)A, lda, M, j0, (float *)tau, wr, G, rows_per, only_if, tp, vp, ldt, trec, tcount, V16, ld16, s);
            else if (rpt <= 2) st = panel_regs_launch<2>((float *)A, lda, M, j0, (float *)tau, wr, G, rows_per, only_if, tp, vp, ldt, trec, tcount, V16, ld16, s);
            else if (rpt <= 3) st = panel_regs_launch<3>((float *)A, lda, M, j0, (float *)tau, wr, G, rows_per, only_if, tp, vp, ldt, trec, tcount, V16, ld16, s);
            else st = panel_regs_launch<4>((float *)A, lda, M, j0, (float *)tau, wr, G, rows_per, only_if, tp, vp, ldt, trec, tcount, V16, ld16, s);
            if (st == CT_OK && made_t) *made_t = want_t;
            if (st == CT_OK && made_v16) *made_v16 = V16 != nullptr;
            return st;
        }
    }
    return panel_launch<float, 32>((float *)A, lda, M, j0, nb, (float *)tau, ws, s);
}

ct_status extract_vtop(bool fp64, const void *A, int64_t lda, int64_t j0, int nb, void *Vtop,
                       int64_t ldv, cudaStream_t s) {
    dim3 grid((unsigned)ceil_div(nb, 128), (unsigned)nb);
    if (fp64) {
        extract_vtop_kernel<double><<<grid, 128, 0, s>>>((const double *)A, lda, j0, nb, (double *)Vtop, ldv);
        count_launch();
    }
    else {
        extract_vtop_kernel<float><<<grid, 128, 0, s>>>((const float *)A, lda, j0, nb, (float *)Vtop, ldv);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// One warp, nb <= 32: lane i owns row i of T in registers; column j is
//   T[i, j] = -tau_j * sum_{i <= l < j} T[i, l] G[l, j]   (i < j),
// with G's column read from shared memory.  Fully unrolled (register indices
// are compile-time), in the factor's precision.
template <typename T>
__global__ void __launch_bounds__(32) larft_warp_kernel(int nb, const T *G, int64_t ldg, const T *tau,
                                                        T *Tm, int64_t ldt) {
    __shared__ T gs[32][33];
    __shared__ T ts[32];
    const int lane = threadIdx.x;
    for (int j = 0; j < 32; ++j) gs[lane][j] = (lane < nb && j < nb) ? G[lane + (int64_t)j * ldg] : T(0);
    ts[lane] = lane < nb ? tau[lane] : T(0);
    __syncwarp();
    T row[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        T y = T(0);
#pragma unroll
        for (int l = 0; l < j; ++l) y += (l >= lane) ? row[l] * gs[l][j] : T(0);
        row[j] = (lane < j) ? -ts[j] * y : (lane == j ? ts[j] : T(0));
    }
    if (lane < nb) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < nb) Tm[lane + (int64_t)j * ldt] = row[j];
    }
}

// One column block of the outer T (FP32):  for the panel at offset o (width
// wp <= 32) of a block reflector with Gram matrix G = V^T V,
//     T[0:o, o:o+wp] = -T[0:o, 0:o] * (G[0:o, o:o+wp] * T_p),  T_p = T[o:o+wp, o:o+wp],
// the off-diagonal block of the product of the block reflectors (I - V1 T1 V1^T)
// (I - Vp T_p Vp^T).  CTA b computes rows [32b, 32b+32): first
// Y[l, :] = G[l, o:o+wp] T_p for l in [32b, o) into shared memory, then
// out[r, :] = -sum_{l >= r} T[r, l] Y[l, :]  (T upper triangular).
__global__ void __launch_bounds__(256) tassemble_kernel(int64_t o, int wp, const float *G, int64_t ldg,
                                                        float *Tm, int64_t ldt) {
    extern __shared__ float ys[];  // [(o - rb)][33]
    __shared__ float tp[32][33];
    const int64_t rb = (int64_t)blockIdx.x * 32;
    const int t = threadIdx.x;
    for (int e = t; e < 32 * 32; e += 256) {
        const int q = e % 32, j = e / 32;
        tp[q][j] = (q < wp && j < wp) ? Tm[(o + q) + (o + j) * ldt] : 0.0f;
    }
    __syncthreads();
    for (int64_t l = rb + t; l < o; l += 256) {
        float g[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) g[q] = (q < wp) ? G[l + (o + q) * ldg] : 0.0f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float y = 0.0f;
#pragma unroll
            for (int q = 0; q <= j; ++q) y += g[q] * tp[q][j];
            ys[(l - rb) * 33 + j] = y;
        }
    }
    __syncthreads();
    const int64_t r = rb + (t % 32);
    const int j0 = 4 * (t / 32);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (r < o) {
        for (int64_t l = r; l < o; ++l) {
            const float tv = Tm[r + l * ldt];
            const float *yr = ys + (l - rb) * 33 + j0;
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += tv * yr[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j0 + u < wp) Tm[r + (o + j0 + u) * ldt] = -acc[u];
    }
}

ct_status t_assemble(int64_t o, int wp, const float *G, int64_t ldg, float *Tm, int64_t ldt,
                     cudaStream_t s) {
    if (o <= 0 || wp <= 0) return CT_OK;
    if (wp > 32) return CT_ERR_ARG;
    const size_t smem = sizeof(float) * (size_t)o * 33;
    if (smem > 200 * 1024) return CT_ERR_UNSUPPORTED;
    static PerContextOnce attr;
    CT_CUDA(attr.run([] {
        return cudaFuncSetAttribute(tassemble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }));
    tassemble_kernel<<<(unsigned)ceil_div(o, 32), 256, smem, s>>>(o, wp, G, ldg, Tm, ldt);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status larft_from_gram(bool fp64, int nb, const void *G, int64_t ldg, const void *tau, void *T,
                          int64_t ldt, cudaStream_t s) {
    if (nb <= 32) {
        if (fp64) larft_warp_kernel<double><<<1, 32, 0, s>>>(nb, (const double *)G, ldg, (const double *)tau,
                                                             (double *)T, ldt);
        else larft_warp_kernel<float><<<1, 32, 0, s>>>(nb, (const float *)G, ldg, (const float *)tau,
                                                       (float *)T, ldt);
        count_launch();
        CT_CUDA(cudaGetLastError());
        return CT_OK;
    }
    const int threads = std::min(1024, std::max(32, nb));
    const size_t smem = sizeof(double) * nb;
    if (fp64) {
        larft_kernel<double><<<1, threads, smem, s>>>(nb, (const double *)G, ldg,
                                                      (const double *)tau, (double *)T, ldt);
        count_launch();
    }
    else {
        larft_kernel<float><<<1, threads, smem, s>>>(nb, (const float *)G, ldg, (const float *)tau,
                                                     (float *)T, ldt);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ctqr
