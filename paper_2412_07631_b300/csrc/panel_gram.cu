// panel_gram.cu -- panel factorisation from Gram matrices (FP32 storage,
// 32-column panels, rows in registers).
//
// The reflectors of a panel A (rows j0 .. M-1, 32 columns) are the ones the
// column-by-column Householder sweep (Sec. 2, Eq. 2; Sec. 2.1 'dgeqrf')
// produces, obtained with two grid-wide exchanges instead of one per column:
//   1. CholeskyQR twice: G1 = A^T A, R1 = chol(G1), Q = A R1^-1;
//      G2 = Q^T Q, R2 = chol(G2), Q <- Q R2^-1, R = R2 R1 (A = Q R, Q with
//      orthonormal columns to working precision after the second pass).
//   2. Householder reconstruction: the thin Q of the Householder form is
//      Q D for a diagonal D of signs, with Q D = [I - V1 T V1^T; -V2 T V1^T].
//      So I - Q1 D = V1 U is an LU factorisation (V1 unit lower, U = T V1^T
//      upper), whose signs d_j are chosen during the elimination so every
//      pivot is 1 + |w_jj| >= 1; then tau_j = U_jj, V2 = -Q2 D U^-1 and the
//      triangle is D R.  (In exact arithmetic these are exactly the
//      reflectors, tau and R of the Householder sweep with the sign rule
//      beta = -sign(alpha) ||x||, up to that sign choice.)
// Each exchange: every CTA writes its partial Gram matrix (upper triangle,
// FP32 sums over its rows), the grid meets, CTA b sums its share of the 528
// entries over all CTAs in a fixed order (FP64), the grid meets again and
// every CTA reads the totals.  Every CTA then repeats the same small
// 32 x 32 steps (in FP32) on identical inputs, so
// all hold identical factors.  A Cholesky pivot that is not safely positive
// (the panel's columns nearly dependent in FP32) or a second Gram matrix
// far from the identity makes every CTA leave the panel untouched and raise
// the fallback flag; the column-by-column kernel then factors it.
#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {
namespace {

constexpr int GQ_THREADS = 256;
constexpr int GQ_WARPS = GQ_THREADS / 32;
constexpr int GQ_TRI = 528;  // upper triangle of a 32 x 32 matrix
constexpr int GQ_LD = 36;    // row stride of the shared copy of the rows (16-byte rows, 4-way stores)
constexpr int GQ_MAX_GRID = 160;  // most CTAs of a launch (one per SM)

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (i, j), i <= j, of the column-packed upper triangle: j is the largest
// integer with j (j + 1) / 2 <= e (the square root estimate, then one
// integer correction either way)
__device__ __forceinline__ void tri_ij(int e, int &i, int &j) {
    j = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    if ((j + 1) * (j + 2) / 2 <= e) ++j;
    if (j * (j + 1) / 2 > e) --j;
    i = e - j * (j + 1) / 2;
}

constexpr int GQ_PER = (GQ_TRI + GQ_THREADS - 1) / GQ_THREADS;  // entries of the triangle per thread

// All CTAs meet (bounded wait).  Returns false on timeout or another CTA's
// error; the caller then leaves.
__device__ bool grid_meet(unsigned *ctr, unsigned G, DevStatus *st, int site, int *ok_s) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        const uint64_t t0 = globaltimer_ns();
        int ok = 1;
        unsigned spins = 0;
        while (*((volatile unsigned *)ctr) < G) {
            __nanosleep(40);
            if ((++spins & 63u) == 0) {
                if (*((volatile int *)&st->code) != 0) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > kWaitLimitNs) {
                    raise_status(st, DEV_TIMEOUT, site, 0);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *ok_s = ok;
    }
    __syncthreads();
    return *ok_s != 0;
}

// A grid meet that cannot complete: one CTA waits for a second that is never
// launched, so the bounded wait gives up (failure-detection check).
__global__ void meet_timeout_kernel(unsigned *ctr, DevStatus *st) {
    __shared__ int ok_s;
    grid_meet(ctr, 2u, st, 90, &ok_s);
}

struct GramShared {
    float g[32][33];             // Gram totals (symmetric), then scratch
    float X[32][33];             // Q1 and its eliminations, then T (reconstruction)
    float Rm[3][32][33];         // R1, R2, U (the three right-hand triangles of the row solves)
    float rinv[3][32];
    float LR[32][33];            // first 32 rows of the result: V1 below the diagonal, D R on and above
    float dsign[32], rw[32], dg[32];
    int ok, bad;
};

// One Gram exchange.  The CTA's rows sit in rows_sm (row-major, GQ_LD floats
// a row).  The 36 4 x 4 blocks on and above the diagonal of their Gram
// matrix are split over 7 groups of rows: thread t < 252 forms block
// t % 36 over row group t / 36 in FP32; after a barrier the partials go
// through rows_sm (no longer needed) and are summed over the groups in a
// fixed order into the CTA's record (upper triangle).  The grid's totals
// (summed in FP64 in a fixed order) end in s.g (full symmetric).
__device__ bool gram_exchange(float *rows_sm, int64_t nloc, GramShared &s, float *rec, double *tot,
                              unsigned *bar, unsigned G, DevStatus *st, int site) {
    constexpr int NGRP = 7, NBLK = 36;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int blk = threadIdx.x % NBLK, grp = threadIdx.x / NBLK;
    // block blk -> (bj, bk), bj <= bk, in row-major order of the upper triangle of 8 x 8
    int bj = 0, rem = blk;
    while (rem >= 8 - bj) {
        rem -= 8 - bj;
        ++bj;
    }
    const int bk = bj + rem;
    float p[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) p[q] = 0.0f;
    if (grp < NGRP) {
        const int64_t chunk = (nloc + NGRP - 1) / NGRP;
        const int64_t ra = grp * chunk, rb = min(nloc, ra + chunk);
#pragma unroll 2
        for (int64_t r = ra; r < rb; ++r) {
            const float4 x = *reinterpret_cast<const float4 *>(rows_sm + r * GQ_LD + 4 * bj);
            const float4 y = *reinterpret_cast<const float4 *>(rows_sm + r * GQ_LD + 4 * bk);
            const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) p[u * 4 + v] = fmaf(xv[u], yv[v], p[u * 4 + v]);
        }
    }
    __syncthreads();  // every thread is done reading the rows
    if (grp < NGRP) {
#pragma unroll
        for (int q = 0; q < 16; ++q) rows_sm[(grp * NBLK + blk) * 16 + q] = p[q];
    }
    __syncthreads();
    float *mine = rec + (size_t)blockIdx.x * GQ_TRI;
#pragma unroll
    for (int u = 0; u < GQ_PER; ++u) {
        const int e = threadIdx.x + u * GQ_THREADS;
        if (e < GQ_TRI) {
            int i, j;
            tri_ij(e, i, j);  // i <= j
            const int ib = i / 4, jbb = j / 4;
            // the block (ib, jbb) of the upper triangle, entry (i % 4, j % 4)
            const int b = ib * 8 - ib * (ib - 1) / 2 + (jbb - ib);
            const int q = (i % 4) * 4 + (j % 4);
            float v = 0.0f;
#pragma unroll
            for (int g2 = 0; g2 < NGRP; ++g2) v += rows_sm[(g2 * NBLK + b) * 16 + q];
            mine[e] = v;
        }
    }
    if (!grid_meet(bar, G, st, site, &s.ok)) return false;
    // CTA b sums entries [b*E, (b+1)*E) over all CTAs, warp by warp, lane l
    // adding records l, l + 32, ... in that order (all loads issued first),
    // then the lanes in a fixed tree
    const int E = (GQ_TRI + (int)G - 1) / (int)G;
    const int e0 = (int)blockIdx.x * E, e1 = min(GQ_TRI, e0 + E);
    for (int e = e0 + warp; e < e1; e += GQ_WARPS) {
        constexpr int PERLANE = (GQ_MAX_GRID + 31) / 32;
        float r[PERLANE];
#pragma unroll
        for (int u = 0; u < PERLANE; ++u) {
            const unsigned b = lane + 32u * u;
            r[u] = (b < G) ? __ldcg(rec + (size_t)b * GQ_TRI + e) : 0.0f;
        }
        double v = 0.0;
#pragma unroll
        for (int u = 0; u < PERLANE; ++u)
            if (lane + 32u * u < G) v += (double)r[u];
        v = warp_sum_d(v);
        if (lane == 0) tot[e] = v;
    }
    if (!grid_meet(bar + 1, G, st, site + 1, &s.ok)) return false;
    float tv[GQ_PER];
#pragma unroll
    for (int u = 0; u < GQ_PER; ++u) {
        const int e = threadIdx.x + u * GQ_THREADS;
        tv[u] = (e < GQ_TRI) ? (float)__ldcg(tot + e) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < GQ_PER; ++u) {
        const int e = threadIdx.x + u * GQ_THREADS;
        if (e < GQ_TRI) {
            int i, j;
            tri_ij(e, i, j);
            const float v = tv[u];
            s.g[i][j] = v;
            s.g[j][i] = v;
        }
    }
    __syncthreads();
    return true;
}

// The small 32 x 32 steps (a few per panel) run on warp 0, one row or
// column per lane.  The dependent chains (the Cholesky steps, the triangular
// solve for Q1, the sign-choosing LU and the solve for T) are unrolled: each
// step reads its pivot from a register named at compile time and updates
// only the trailing entries, one broadcast and one FMA each, which are the
// FMAs of the full-width column sweep in the same order.  The loads and the
// assembly of U and of the outputs go through 32 x 33 shared-memory copies
// as short rolled loops (this code runs once per launch from a cold
// instruction cache, where a short loop costs less than straight-line code).
// Reciprocal square roots use the fast hardware approximation (a few ulp;
// the second Cholesky pass and the FP64 refinement absorb such errors).

// R <- chol(s.g) (upper, R^T R = G) into Rout, 1 / diag(R) into rinv, one
// warp, lane c holding column c.  Returns false (same in every lane) if a
// pivot is not above min_rel times its original diagonal entry or, with
// near_identity, if s.g is not within 0.25 of I entrywise.
__device__ __noinline__ bool chol_warp(GramShared &s, float (*Rout)[33], float *rinv, float min_rel,
                                       bool near_identity) {
    const int lane = threadIdx.x % 32;
    float g[32];
    bool good = true;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        g[r] = s.g[r][lane];
        if (near_identity) good = good && fabsf(g[r] - (r == lane ? 1.0f : 0.0f)) <= 0.25f;
    }
    const float d0 = s.g[lane][lane];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float gi = g[i];
        const float gii = __shfl_sync(0xffffffffu, gi, i);
        const float dii = __shfl_sync(0xffffffffu, d0, i);
        const bool ok = gii > min_rel * dii;
        good = good && ok;
        const float ric = (lane >= i && ok) ? gi * rsqrtf(gii) : 0.0f;  // R_ic (R_ii for lane i)
        Rout[i][lane] = ric;  // zero below the diagonal (lane < i)
        // trailing update: rows k > i of the column (rows <= i are not read again)
#pragma unroll
        for (int k = i + 1; k < 32; ++k) g[k] = fmaf(-__shfl_sync(0xffffffffu, ric, k), ric, g[k]);
    }
    __syncwarp();
    const float rl = Rout[lane][lane];
    rinv[lane] = (rl > 0.0f) ? __frcp_rn(rl) : 1.0f;
    __syncwarp();
    return __all_sync(0xffffffffu, good);
}

// Householder reconstruction (see the top of the file), one warp, lane = row
// (R = R2 R1 already in s.g): Q1 = A1 R^-1; LU of I - Q1 D with the signs
// d_j chosen on the way; U (with 1 / diag U), V1 and D R into s; tau = diag(U).
__device__ __noinline__ void reconstruct_warp(GramShared &s, const float *topbuf, float *tau, bool write_tau,
                                              float *Tp, float *Vtp, int64_t ldt) {
    const int lane = threadIdx.x % 32;
    float (*X)[33] = s.X;
    s.rw[lane] = __frcp_rn(s.g[lane][lane]);
#pragma unroll 4
    for (int r = 0; r < 32; ++r) X[r][lane] = __ldcg(topbuf + r * 32 + lane);  // A1, row by row
    __syncwarp();
    float x[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = X[lane][k];
    // x <- A1 R^-1, forward over the columns: x_j = x_j / R_jj is removed
    // from the later columns k > j (x_k -= x_j R_jk, j ascending)
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float xj = x[j] * s.rw[j];
#pragma unroll
        for (int k = j + 1; k < 32; ++k) x[k] = fmaf(-xj, s.g[j][k], x[k]);
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] *= s.rw[k];
    // LU of I - Q1 D: step j picks d_j = -sign(w_jj), pivot 1 + |w_jj|,
    // multipliers l_rj = -d_j w_rj / (1 + |w_jj|) (rows below j), eliminates
    // them from the later columns k > j
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float wjj = __shfl_sync(0xffffffffu, x[j], j);
        const float dj = (wjj >= 0.0f) ? -1.0f : 1.0f;
        const float l = (lane > j) ? -dj * x[j] * __frcp_rn(1.0f + fabsf(wjj)) : 0.0f;
        if (lane > j) s.LR[lane][j] = l;
        if (lane == j) s.dsign[j] = dj;
#pragma unroll
        for (int k = j + 1; k < 32; ++k) x[k] = fmaf(-l, __shfl_sync(0xffffffffu, x[k], j), x[k]);
    }
    // row r now holds w_rr and w_rk (k > r) as they stood at step r
#pragma unroll
    for (int k = 0; k < 32; ++k) X[lane][k] = x[k];
    __syncwarp();
    float (*U)[33] = s.Rm[2];
    const float ujj = 1.0f + fabsf(X[lane][lane]), dl = s.dsign[lane];
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        U[lane][k] = (k > lane) ? -s.dsign[k] * X[lane][k] : (k == lane ? ujj : 0.0f);
        if (k >= lane) s.LR[lane][k] = dl * s.g[lane][k];
    }
    s.rinv[2][lane] = __frcp_rn(ujj);
    if (write_tau) tau[lane] = ujj;
    __syncwarp();
    if (write_tau && Tp != nullptr) {
        // T = U V1^-T (U = T V1^T), row `lane`: t V1^T = u, forward over the
        // columns (V1 unit lower, below the diagonal in s.LR)
        float t[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) t[k] = U[lane][k];
#pragma unroll
        for (int l = 0; l < 32; ++l) {
#pragma unroll
            for (int k = l + 1; k < 32; ++k) t[k] = fmaf(-t[l], s.LR[k][l], t[k]);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) X[lane][k] = t[k];
        __syncwarp();
        // column k of T and of the unit-lower top of V: lane = row
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            Tp[lane + k * ldt] = (k >= lane) ? X[lane][k] : 0.0f;
            Vtp[lane + k * ldt] = (k == lane) ? 1.0f : (k < lane ? s.LR[lane][k] : 0.0f);
        }
    }
}

// R = R2 R1 (upper) into s.g, whole CTA.
__device__ void r_product(GramShared &s) {
    for (int e = threadIdx.x; e < 1024; e += GQ_THREADS) {
        const int i = e >> 5, k = e & 31;
        float v = 0.0f;
        for (int l = i; l <= k; ++l) v = fmaf(s.Rm[1][i][l], s.Rm[0][l][k], v);
        s.g[i][k] = v;  // zero below the diagonal (empty sum)
    }
    __syncthreads();
}

template <int RPT>
__global__ void __launch_bounds__(GQ_THREADS, 1)
    panel_gram_kernel(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, float *rec, double *tot,
                      float *topbuf, unsigned *bar, int *fallback, DevStatus *st, int64_t rows_per,
                      float *Tp, float *Vtp, int64_t ldt, uint8_t *V16, int64_t ld16) {
    __shared__ GramShared s;
    extern __shared__ float rows_sm[];  // [RPT * GQ_THREADS][GQ_LD], row-major
    const unsigned G = gridDim.x;
    const int64_t r0 = j0 + (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(M, r0 + rows_per);
    const int64_t nloc = max((int64_t)0, r1 - r0);

    float a[RPT][32];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t lr = threadIdx.x + (int64_t)i * GQ_THREADS;
#pragma unroll
        for (int k = 0; k < 32; ++k) a[i][k] = (lr < nloc) ? A[(r0 + lr) + (j0 + k) * lda] : 0.0f;
    }
    // the first 32 rows of the panel (CTA 0, rows 0..31 of its first slice)
    if (blockIdx.x == 0 && threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < 32; ++k) topbuf[threadIdx.x * 32 + k] = a[0][k];
    }

    // phase 0: G1 = A^T A, R1 = chol(G1), rows <- rows R1^-1
    // phase 1: G2 = Q^T Q, R2 = chol(G2), rows <- rows R2^-1
    // phase 2: reconstruction (D, U, V1, D R), rows <- -rows D U^-1
#pragma unroll 1
    for (int phase = 0; phase < 3; ++phase) {
        if (phase < 2) {
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                float4 *dst = reinterpret_cast<float4 *>(rows_sm + (threadIdx.x + i * GQ_THREADS) * GQ_LD);
#pragma unroll
                for (int k = 0; k < 8; ++k) dst[k] = make_float4(a[i][4 * k], a[i][4 * k + 1], a[i][4 * k + 2], a[i][4 * k + 3]);
            }
            __syncthreads();
            if (!gram_exchange(rows_sm, nloc, s, rec + (size_t)phase * G * GQ_TRI, tot + phase * GQ_TRI,
                               bar + 2 * phase, G, st, 40 + 2 * phase))
                return;
            // after one pass Q^T Q must already be near the identity
            if (threadIdx.x < 32) {
                const bool good = chol_warp(s, s.Rm[phase], s.rinv[phase], phase == 0 ? 2e-5f : 0.25f, phase == 1);
                if (threadIdx.x == 0) s.bad = good ? 0 : 1;
            }
            __syncthreads();
            if (s.bad) {
                if (blockIdx.x == 0 && threadIdx.x == 0) *fallback = 1;
                return;
            }
        } else {
            r_product(s);
            if (threadIdx.x < 32) reconstruct_warp(s, topbuf, tau + j0, blockIdx.x == 0, Tp, Vtp, ldt);
            __syncthreads();
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int k = 0; k < 32; ++k) a[i][k] = -a[i][k] * s.dsign[k];
        }
        // rows <- rows Rm[phase]^-1: x_k = (x_k - sum_{j<k} x_j R_jk) / R_kk, j ascending
        const float (*R)[33] = s.Rm[phase];
        const float *ri = s.rinv[phase];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            float sm[RPT];
#pragma unroll
            for (int i = 0; i < RPT; ++i) sm[i] = a[i][k];
#pragma unroll
            for (int j = 0; j < k; ++j) {
                const float r = R[j][k];
#pragma unroll
                for (int i = 0; i < RPT; ++i) sm[i] = fmaf(-a[i][j], r, sm[i]);
            }
            const float rk = ri[k];
#pragma unroll
            for (int i = 0; i < RPT; ++i) a[i][k] = sm[i] * rk;
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t lr = threadIdx.x + (int64_t)i * GQ_THREADS;
        const int64_t gr = r0 + lr;
        if (lr >= nloc) continue;
        if (gr < j0 + 32) {  // the first 32 rows: V1 below the diagonal, D R on and above
            const int r = (int)(gr - j0);
#pragma unroll
            for (int k = 0; k < 32; ++k) A[gr + (j0 + k) * lda] = s.LR[r][k];
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) A[gr + (j0 + k) * lda] = a[i][k];
            if (V16 != nullptr) store_bf16_row32(V16 + 2 * (size_t)((gr - j0 - 32) * ld16), a[i]);
        }
    }
}

template <int RPT>
ct_status gram_launch(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, void *ws, unsigned *bar, int G,
                      int64_t rows_per, int *fallback, float *Tp, float *Vtp, int64_t ldt, void *V16,
                      int64_t ld16, cudaStream_t s) {
    auto fn = panel_gram_kernel<RPT>;
    const size_t dyn = sizeof(float) * GQ_LD * RPT * GQ_THREADS;
    static PerContextOnce attr;  // the attribute belongs to each device's context
    CT_CUDA(attr.run([&] { return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn); }));
    if (G < 1 || G > GQ_MAX_GRID) {
        set_error("gram panel: grid of %d CTAs outside 1..%d", G, GQ_MAX_GRID);
        return CT_ERR_ARG;
    }
    int per_sm = 0;
    CT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, GQ_THREADS, dyn));
    if (per_sm * num_sms() < G) {
        set_error("gram panel: cooperative grid %d does not fit (%d per SM)", G, per_sm);
        return CT_ERR_CUDA;
    }
    // ws: totals [2][528] FP64 | top block [1024] | records [2][G][528]
    double *tot = (double *)ws;
    float *top = (float *)((char *)tot + sizeof(double) * 2 * GQ_TRI);
    float *rec = top + 1024;
    DevStatus *st = device_status();
    uint8_t *v16 = (uint8_t *)V16;
    void *args[] = {&A, &lda, &M, &j0, &tau, &rec, &tot, &top, &bar, &fallback, &st, &rows_per, &Tp, &Vtp, &ldt,
                    &v16, &ld16};
    CT_CUDA(cudaLaunchCooperativeKernel((const void *)fn, dim3(G), dim3(GQ_THREADS), args, dyn, s));
    count_launch();
    return CT_OK;
}

}  // namespace

ct_status wait_selftest(cudaStream_t s) {
    CT_TRY(check_device_status(s));  // start from a clear status word
    unsigned *ctr = nullptr;
    CT_CUDA(cudaMalloc((void **)&ctr, 256));
    ct_status st = CT_OK;
    if (cudaMemsetAsync(ctr, 0, 256, s) != cudaSuccess) st = CT_ERR_CUDA;
    if (st == CT_OK) {
        meet_timeout_kernel<<<1, 32, 0, s>>>(ctr, device_status());
        count_launch();
        st = cudaGetLastError() == cudaSuccess ? check_device_status(s) : CT_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    cudaFree(ctr);
    return st;
}

size_t panel_gram_ws_bytes(int G) {
    return sizeof(double) * 2 * GQ_TRI + sizeof(float) * (1024 + 2 * (size_t)G * GQ_TRI);
}

ct_status panel_gram(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, void *ws, unsigned *bar,
                     int G, int64_t rows_per, int rpt, int *fallback, float *Tp, float *Vtp, int64_t ldt,
                     void *V16, int64_t ld16, cudaStream_t s) {
    switch (rpt) {
        case 1: return gram_launch<1>(A, lda, M, j0, tau, ws, bar, G, rows_per, fallback, Tp, Vtp, ldt, V16, ld16, s);
        case 2: return gram_launch<2>(A, lda, M, j0, tau, ws, bar, G, rows_per, fallback, Tp, Vtp, ldt, V16, ld16, s);
        case 3: return gram_launch<3>(A, lda, M, j0, tau, ws, bar, G, rows_per, fallback, Tp, Vtp, ldt, V16, ld16, s);
        case 4: return gram_launch<4>(A, lda, M, j0, tau, ws, bar, G, rows_per, fallback, Tp, Vtp, ldt, V16, ld16, s);
        default: return CT_ERR_ARG;
    }
}

}  // namespace ctqr
