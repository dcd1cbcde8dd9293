// panel_regs.cuh -- the column-by-column panel sweep with rows in registers
// (Sec. 2, Eq. 2; 'dgeqrf' of Sec. 2.1), shared by its own kernel (panel.cu)
// and the Gram-based panel kernel (panel_gram.cu), which runs it in the same
// launch when it declines a panel.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {
namespace {

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

// The column sweep of one panel by the whole grid (RP_THREADS threads per
// CTA, rows_per rows per CTA): the body of the column-by-column kernel, and
// of the Gram kernel when it declines a panel.  With Tp given (the Gram
// route's caller wants T), it also forms the panel's T and the top of V.
template <int RPT>
__device__ __noinline__ void panel_regs_body(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, float *rec,
                                             uint64_t *tot, unsigned *counter, DevStatus *st, int64_t rows_per,
                                             float *Tp, float *Vtp, int64_t ldt, float *trec, unsigned *tcount,
                                             uint8_t *V16, int64_t ld16) {
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
    if (Tp != nullptr) fallback_t(A, lda, j0, r0, nloc, tau, Tp, Vtp, ldt, trec, tcount);
}

}  // namespace
}  // namespace ctqr
