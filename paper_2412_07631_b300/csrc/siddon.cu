// siddon.cu -- system-matrix builder: a_ij = length of ray i inside pixel j
// (Sec. 2 Eq. 1 defines a_ij as the contribution of ray i to pixel j; the
// exact intersection length is Siddon's choice of that contribution).
//
// One thread per ray.  The ray is p(s) = (x0 - s*sn, y0 + s*c), x0 = t*c,
// y0 = t*sn, unit speed.  Grid line k (k = 0..n_side) of either axis is at
// -h + k*w, h = n_side*w/2.  The walk merges the two monotone sequences of
// line crossings (x lines and y lines) in increasing s, between the entry and
// exit of the square; each pair of consecutive crossings is one segment whose
// pixel contains its midpoint.  Segments of length <= 1e-12*w are dropped.
//
// Every floating-point operation of the walk is an explicitly rounded IEEE
// double operation (__dadd_rn & co.), so no FMA contraction can change a
// length or a pixel decision; the results are reproducible bit for bit by any
// IEEE double implementation that performs the same operations.
#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

struct Geo {
    int n_side, n_views, n_bins;
    double w, bw;
    int kind;  // CT_GEOM_PARALLEL: cs = per-view (cos, sin); CT_GEOM_FAN: cs = per-ray (c, s, t)
    int projector;  // CT_PROJ_SIDDON / CT_PROJ_JOSEPH
};

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// Crossing parameter of grid line k of the x axis / y axis.
__device__ __forceinline__ double line_pos(double h, int k, double w) {
    return dadd(-h, dmul((double)k, w));
}

// Walks ray (c, sn, t); calls emit(pixel, length) for each kept segment in
// walk order; returns the number of kept segments.
template <class Emit>
__device__ int siddon_walk(const Geo &g, double c, double sn, double t, Emit emit) {
    const double h = dmul(dmul(0.5, (double)g.n_side), g.w);
    const double x0 = dmul(t, c);
    const double y0 = dmul(t, sn);
    double s_in = -INFINITY, s_out = INFINITY;
    if (sn != 0.0) {
        double sa = ddiv(dsub(x0, dadd(-h, dmul(0.0, g.w))), sn);
        double sb = ddiv(dsub(x0, dadd(-h, dmul((double)g.n_side, g.w))), sn);
        s_in = fmax(s_in, fmin(sa, sb));
        s_out = fmin(s_out, fmax(sa, sb));
    } else if (!(x0 > -h && x0 < h)) {
        return 0;
    }
    if (c != 0.0) {
        double sa = ddiv(dsub(dadd(-h, dmul(0.0, g.w)), y0), c);
        double sb = ddiv(dsub(dadd(-h, dmul((double)g.n_side, g.w)), y0), c);
        s_in = fmax(s_in, fmin(sa, sb));
        s_out = fmin(s_out, fmax(sa, sb));
    } else if (!(y0 > -h && y0 < h)) {
        return 0;
    }
    if (!(s_out > s_in)) return 0;

    // Iterators over the crossings in increasing s.
    const int n = g.n_side;
    int kx = (sn > 0.0) ? n : 0, dkx = (sn > 0.0) ? -1 : 1, nx = (sn != 0.0) ? n + 1 : 0;
    int ky = (c > 0.0) ? 0 : n, dky = (c > 0.0) ? 1 : -1, ny = (c != 0.0) ? n + 1 : 0;
    auto next_x = [&]() -> double {
        while (nx > 0) {
            double sk = ddiv(dsub(x0, line_pos(h, kx, g.w)), sn);
            kx += dkx;
            --nx;
            if (sk > s_in) {
                if (sk < s_out) return sk;
                nx = 0;
                break;
            }
        }
        return INFINITY;
    };
    auto next_y = [&]() -> double {
        while (ny > 0) {
            double sk = ddiv(dsub(line_pos(h, ky, g.w), y0), c);
            ky += dky;
            --ny;
            if (sk > s_in) {
                if (sk < s_out) return sk;
                ny = 0;
                break;
            }
        }
        return INFINITY;
    };
    double sx = next_x(), sy = next_y();
    double s_prev = s_in;
    const double thr = dmul(1e-12, g.w);
    int nseg = 0;
    bool done = false;
    while (!done) {
        double s_next;
        if (sx <= sy && sx < s_out) {
            s_next = sx;
            sx = next_x();
        } else if (sy < s_out) {
            s_next = sy;
            sy = next_y();
        } else {
            s_next = s_out;
            done = true;
        }
        double L = dsub(s_next, s_prev);
        if (L > thr) {
            double sm = dmul(dadd(s_prev, s_next), 0.5);
            double xm = dsub(x0, dmul(sm, sn));
            double ym = dadd(y0, dmul(sm, c));
            int ix = (int)floor(ddiv(dadd(xm, h), g.w));
            int iy = (int)floor(ddiv(dadd(ym, h), g.w));
            ix = min(max(ix, 0), n - 1);
            iy = min(max(iy, 0), n - 1);
            emit(nseg, iy * n + ix, L);
            ++nseg;
        }
        s_prev = s_next;
    }
    return nseg;
}

// Joseph's projector for ray (c, s, t): sampled once per pixel row when
// |c| >= |s| (else per column) on its centre line, the crossing point
// interpolated linearly between the two nearest pixel centres, weights
// scaled by the ray length per row (column).  Pixels outside the grid and
// zero weights are dropped; a pair's lower pixel index comes first.  The
// operations are the oracle's, one IEEE rounding each.
template <class Emit>
__device__ int joseph_walk(const Geo &g, double c, double s, double t, Emit emit) {
    const double h = dmul(dmul(0.5, (double)g.n_side), g.w);
    const bool rows = fabs(c) >= fabs(s);
    const double L = ddiv(g.w, rows ? fabs(c) : fabs(s));
    int n = 0;
    for (int k = 0; k < g.n_side; ++k) {
        const double q = dsub(dmul(dadd((double)k, 0.5), g.w), h);
        double p;
        if (rows) {
            const double a = ddiv(dsub(q, dmul(t, s)), c);  // x = t c - u s at y = q
            p = dsub(dmul(t, c), dmul(s, a));
        } else {
            const double a = ddiv(dsub(dmul(t, c), q), s);  // y = t s + u c at x = q
            p = dadd(dmul(t, s), dmul(c, a));
        }
        const double fp = dsub(ddiv(dadd(p, h), g.w), 0.5);
        const double fl = floor(fp);
        if (!(fl >= -1.0 && fl <= (double)g.n_side - 1.0)) continue;
        const double f = dsub(fp, fl);
        const int j = (int)fl;
        if (j >= 0) {
            emit(n, rows ? k * g.n_side + j : j * g.n_side + k, dmul(dsub(1.0, f), L));
            ++n;
        }
        if (j + 1 < g.n_side && f > 0.0) {
            emit(n, rows ? k * g.n_side + (j + 1) : (j + 1) * g.n_side + k, dmul(f, L));
            ++n;
        }
    }
    return n;
}

template <class Emit>
__device__ __forceinline__ int project_walk(const Geo &g, double c, double sn, double t, Emit emit) {
    return g.projector == CT_PROJ_JOSEPH ? joseph_walk(g, c, sn, t, emit) : siddon_walk(g, c, sn, t, emit);
}

__device__ __forceinline__ void ray_params(const Geo &g, const double *cs, int i, double &c,
                                           double &sn, double &t) {
    if (g.kind == CT_GEOM_FAN) {  // host-computed table of the ray lines
        c = cs[3 * (int64_t)i];
        sn = cs[3 * (int64_t)i + 1];
        t = cs[3 * (int64_t)i + 2];
        return;
    }
    int v = i / g.n_bins, d = i - v * g.n_bins;
    c = cs[2 * v];
    sn = cs[2 * v + 1];
    t = dmul(dsub((double)d, dmul(0.5, (double)(g.n_bins - 1))), g.bw);
}

__global__ void siddon_count_kernel(Geo g, const double *cs, int32_t *row_nnz) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_views * g.n_bins) return;
    double c, sn, t;
    ray_params(g, cs, i, c, sn, t);
    row_nnz[i] = project_walk(g, c, sn, t, [](int, int, double) {});
}

// Writes the CSR row of ray i and adds its lengths into the dense column-major
// matrix (runs of equal pixels are summed in FP64 before the store).
template <typename T>
__global__ void siddon_fill_kernel(Geo g, const double *cs, const int64_t *row_ptr,
                                   int32_t *col_idx, double *val, T *dense, int64_t lda) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_views * g.n_bins) return;
    double c, sn, t;
    ray_params(g, cs, i, c, sn, t);
    const int64_t base = row_ptr[i];
    int run_pix = -1;
    double run_len = 0.0;
    project_walk(g, c, sn, t, [&](int q, int pix, double L) {
        col_idx[base + q] = pix;
        val[base + q] = L;
        if (dense) {
            if (pix == run_pix) {
                run_len = dadd(run_len, L);
            } else {
                if (run_pix >= 0) dense[i + (int64_t)run_pix * lda] += (T)run_len;
                run_pix = pix;
                run_len = L;
            }
        }
    });
    if (dense && run_pix >= 0) dense[i + (int64_t)run_pix * lda] += (T)run_len;
}

template <typename T>
__global__ void lambda_rows_kernel(T *dense, int64_t lda, int64_t m, int64_t n, double sl) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dense[(m + j) + j * lda] = (T)sl;
}

// ---- exclusive scan of int32 counts into int64 offsets (3 phases) ----------
constexpr int kScanBlock = 1024;

__global__ void scan_block_kernel(const int32_t *in, int64_t n, int64_t *out, int64_t *block_sums) {
    __shared__ int64_t s[kScanBlock];
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t add = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

// Single block: exclusive scan of the block sums (sequential per thread chunk).
__global__ void scan_top_kernel(int64_t *block_sums, int64_t nb, int64_t *total) {
    __shared__ int64_t s[kScanBlock];
    const int64_t per = (nb + kScanBlock - 1) / kScanBlock;
    int64_t lo = threadIdx.x * per, hi = min(nb, lo + per);
    int64_t acc = 0;
    for (int64_t q = lo; q < hi; ++q) acc += block_sums[q];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t add = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t run = s[threadIdx.x] - acc;
    for (int64_t q = lo; q < hi; ++q) {
        int64_t v = block_sums[q];
        block_sums[q] = run;
        run += v;
    }
    if (threadIdx.x == kScanBlock - 1) *total = s[threadIdx.x];
}

__global__ void scan_add_kernel(int64_t *out, int64_t n, const int64_t *block_sums,
                                const int64_t *total) {
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += block_sums[blockIdx.x];
    if (i == n - 1) out[n] = *total;
}

// ---- CSC of A (for A^T r) ---------------------------------------------------
__global__ void row_of_entry_kernel(const int64_t *row_ptr, int64_t m, int32_t *row_of) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) row_of[q] = (int32_t)i;
}

__global__ void col_count_kernel(const int32_t *col_idx, int64_t nnz, int32_t *col_cnt) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nnz) atomicAdd(&col_cnt[col_idx[q]], 1);
}

// Places entry q at a free slot of its column (order fixed later by the sort).
__global__ void csc_place_kernel(const int32_t *col_idx, int64_t nnz, const int64_t *col_ptr,
                                 int32_t *cursor, int64_t *slot_entry) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    int j = col_idx[q];
    int pos = atomicAdd(&cursor[j], 1);
    slot_entry[col_ptr[j] + pos] = q;
}

// One block per column: sort the column's entry ids ascending (ids grow with
// the ray index and with walk order), then gather row and value.
constexpr int kColSortMax = 4096;
__global__ void csc_sort_kernel(const int64_t *col_ptr, const int64_t *slot_entry,
                                const int32_t *row_of, const double *val, int32_t *csc_row,
                                double *csc_val, DevStatus *st) {
    __shared__ int64_t key[kColSortMax];
    const int j = blockIdx.x;
    const int64_t lo = col_ptr[j], len = col_ptr[j + 1] - lo;
    if (len > kColSortMax) {
        if (threadIdx.x == 0) raise_status(st, DEV_BADARG, 100, (int)len);
        return;
    }
    int P = 1;
    while (P < len) P <<= 1;
    for (int q = threadIdx.x; q < P; q += blockDim.x) key[q] = (q < len) ? slot_entry[lo + q] : INT64_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int q = threadIdx.x; q < P; q += blockDim.x) {
                int partner = q ^ jj;
                if (partner > q) {
                    bool up = (q & k) == 0;
                    int64_t a = key[q], b = key[partner];
                    if ((a > b) == up) {
                        key[q] = b;
                        key[partner] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int q = threadIdx.x; q < len; q += blockDim.x) {
        int64_t e = key[q];
        csc_row[lo + q] = row_of[e];
        csc_val[lo + q] = val[e];
    }
}

}  // namespace

ct_status exclusive_scan(const int32_t *in, int64_t n, int64_t *out_np1, Scratch &tmp,
                         cudaStream_t s) {
    const int64_t nb = ceil_div(n, kScanBlock);
    CT_TRY(tmp.ensure(sizeof(int64_t) * (nb + 1)));
    int64_t *bs = (int64_t *)tmp.ptr;
    int64_t *total = bs + nb;
    scan_block_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, out_np1, bs);
    count_launch();
    scan_top_kernel<<<1, kScanBlock, 0, s>>>(bs, nb, total);
    count_launch();
    scan_add_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(out_np1, n, bs, total);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status siddon_build(const SiddonArgs &a, cudaStream_t s) {
    Geo g{a.n_side, a.n_views, a.n_bins, a.pixel_width, a.bin_width, a.kind, a.projector};
    const int m = a.n_views * a.n_bins;
    const int threads = 128;
    const unsigned blocks = (unsigned)ceil_div(m, threads);
    ProfScope prof(PROF_SIDDON, s, 0.0, 4.0 * m);
    siddon_count_kernel<<<blocks, threads, 0, s>>>(g, a.d_cs, a.d_row_nnz);
    count_launch();
    CT_CUDA(cudaGetLastError());
    CT_TRY(exclusive_scan(a.d_row_nnz, m, a.d_row_ptr, *a.tmp, s));
    return CT_OK;
}

ct_status siddon_fill(const SiddonArgs &a, void *dense, bool dense_fp64, int64_t lda,
                      cudaStream_t s) {
    Geo g{a.n_side, a.n_views, a.n_bins, a.pixel_width, a.bin_width, a.kind, a.projector};
    const int m = a.n_views * a.n_bins;
    const int threads = 128;
    const unsigned blocks = (unsigned)ceil_div(m, threads);
    const int64_t n = (int64_t)a.n_side * a.n_side;
    if (dense_fp64) {
        siddon_fill_kernel<double><<<blocks, threads, 0, s>>>(g, a.d_cs, a.d_row_ptr, a.d_col,
                                                              a.d_val, (double *)dense, lda);
        count_launch();
        if (dense && a.sqrt_lambda > 0) {
            lambda_rows_kernel<double><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(
                (double *)dense, lda, m, n, a.sqrt_lambda);
            count_launch();
        }
    } else {
        siddon_fill_kernel<float><<<blocks, threads, 0, s>>>(g, a.d_cs, a.d_row_ptr, a.d_col,
                                                             a.d_val, (float *)dense, lda);
        count_launch();
        if (dense && a.sqrt_lambda > 0) {
            lambda_rows_kernel<float><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(
                (float *)dense, lda, m, n, a.sqrt_lambda);
            count_launch();
        }
    }
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status build_csc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col_idx, const double *val, int64_t *col_ptr, int32_t *csc_row,
                    double *csc_val, Scratch &tmp, Scratch &tmp2, cudaStream_t s) {
    // scratch layout: row_of[nnz] int32 | col_cnt[n] int32 | slot_entry[nnz] int64
    size_t off_cnt = round_up(sizeof(int32_t) * nnz, 256);
    size_t off_slot = off_cnt + round_up(sizeof(int32_t) * n, 256);
    size_t need = off_slot + sizeof(int64_t) * nnz;
    CT_TRY(tmp.ensure(need));
    char *base = (char *)tmp.ptr;
    int32_t *row_of = (int32_t *)base;
    int32_t *col_cnt = (int32_t *)(base + off_cnt);
    int64_t *slot = (int64_t *)(base + off_slot);
    row_of_entry_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(row_ptr, m, row_of);
    count_launch();
    CT_CUDA(cudaMemsetAsync(col_cnt, 0, sizeof(int32_t) * n, s));
    if (nnz > 0) {
        col_count_kernel<<<(unsigned)ceil_div(nnz, 256), 256, 0, s>>>(col_idx, nnz, col_cnt);
        count_launch();
    }
    CT_TRY(exclusive_scan(col_cnt, n, col_ptr, tmp2, s));
    CT_CUDA(cudaMemsetAsync(col_cnt, 0, sizeof(int32_t) * n, s));
    if (nnz > 0) {
        csc_place_kernel<<<(unsigned)ceil_div(nnz, 256), 256, 0, s>>>(col_idx, nnz, col_ptr,
                                                                       col_cnt, slot);
        count_launch();
    }
    csc_sort_kernel<<<(unsigned)n, 256, 0, s>>>(col_ptr, slot, row_of, val, csc_row, csc_val,
                                                device_status());
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ctqr
