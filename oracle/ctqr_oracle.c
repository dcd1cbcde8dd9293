/*
 * ctqr_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no header, helper, table or constant with the
 * CUDA path: the view table, the ray geometry, the Siddon walk, the Householder
 * reflectors and the triangular solves are all written out again here.
 *
 * What it computes (arxiv 2412.07631):
 *   - the linear model A X = B, a_ij = contribution of ray i to pixel j
 *     (Sec. 2, Eq. 1); here a_ij is the exact length of ray i inside pixel j
 *     (Siddon's ray-pixel intersection lengths), with the rows sqrt(lambda)*I
 *     appended below A (Tikhonov regularisation, the build's extension);
 *   - A = QR by Householder reflectors, Q kept implicitly as reflectors plus
 *     tau scalars, never formed (Sec. 2, Eq. 2 and the text after Eq. 3);
 *   - C = Q^T B, then R X = C by back-substitution (Sec. 2, Eq. 3; Sec. 2.1);
 *   - brute-force normal equations in long double (a pin for the QR route);
 *   - the residual r = b~ - A~ x and A~^T r in long double (the optimality
 *     certificate ||x - x*|| <= ||A~^T r|| / lambda, used where a dense oracle
 *     solve is too large).
 *
 * Compiled with -O2 -ffp-contract=off (no FMA contraction) so that every
 * floating-point operation of the Siddon walk is a single IEEE-rounded
 * double operation.  OpenMP is used only to run independent columns / rays
 * in parallel; no operation order inside one column or ray depends on it.
 *
 * Conventions: dense matrices are column-major (Fortran/LAPACK), element
 * (i, j) at A[i + j*lda].  Ray index i = v*n_bins + d, pixel index
 * j = iy*n_side + ix.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Geometry (parallel beam).                                                  */
/* ------------------------------------------------------------------------ */

/* Angle of view v: theta_v = v * arc / n_views (arc in degrees, endpoint
 * excluded).  cos/sin come from libm; values within 1e-15 of 0 are set to 0
 * and the partner to +-1, so axis-aligned views are exact. */
EXPORT void oracle_view_table(int n_views, double arc_deg, double *cs)
{
    for (int v = 0; v < n_views; ++v) {
        double theta = ((double)v * arc_deg / (double)n_views) * (M_PI / 180.0);
        double c = cos(theta), s = sin(theta);
        if (fabs(c) < 1e-15) { c = 0.0; s = (s > 0.0) ? 1.0 : -1.0; }
        if (fabs(s) < 1e-15) { s = 0.0; c = (c > 0.0) ? 1.0 : -1.0; }
        cs[2 * v] = c;
        cs[2 * v + 1] = s;
    }
}

/* Fan-beam rays (equiangular arc detector centred on the source): source v
 * at beta_v = v * arc / n_views (degrees, endpoint excluded), at distance
 * sid from the rotation axis, S = sid (cos beta, sin beta); detector d at
 * fan angle gamma_d = (d - (n_det - 1)/2) * fan / (n_det - 1) from the central
 * ray, which points from S through the axis.  The ray's line in normal form
 * {t (c, s) + u (-s, c)}: its direction (-cos(beta+gamma), -sin(beta+gamma))
 * gives theta = beta + gamma + pi/2, (c, s) = (cos theta, sin theta), and
 * t = S . (c, s) = -sid sin(gamma).  Values below 1e-15 in magnitude are
 * snapped as in the view table.  out[3i..3i+2] = (c, s, t), i = v n_det + d. */
EXPORT void oracle_fan_rays(int n_views, int n_det, double arc_deg, double fan_deg, double sid,
                            double *out)
{
    for (int v = 0; v < n_views; ++v) {
        const double beta = ((double)v * arc_deg / (double)n_views) * (M_PI / 180.0);
        for (int d = 0; d < n_det; ++d) {
            const double gamma =
                (((double)d - 0.5 * (double)(n_det - 1)) * (fan_deg / (double)(n_det - 1))) * (M_PI / 180.0);
            const double theta = (beta + gamma) + 0.5 * M_PI;
            double c = cos(theta), s = sin(theta);
            if (fabs(c) < 1e-15) { c = 0.0; s = (s > 0.0) ? 1.0 : -1.0; }
            if (fabs(s) < 1e-15) { s = 0.0; c = (c > 0.0) ? 1.0 : -1.0; }
            const int64_t i = (int64_t)v * n_det + d;
            out[3 * i] = c;
            out[3 * i + 1] = s;
            out[3 * i + 2] = -(sid * sin(gamma));
        }
    }
}

/* Detector coordinate of bin d: bin centres spaced bin_width apart, centred
 * on the rotation axis. */
static double bin_centre(int d, int n_bins, double bin_width)
{
    return ((double)d - 0.5 * (double)(n_bins - 1)) * bin_width;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* Siddon intersection lengths of one ray with the n_side x n_side pixel grid.
 *
 * The ray is p(s) = (x0 - s*sn, y0 + s*c) with x0 = t*c, y0 = t*sn: the line
 * at signed distance t from the centre, direction (-sn, c), unit speed, so a
 * parameter difference is a length.  The image covers [-h, h]^2 with
 * h = n_side*w/2; grid line k (k = 0..n_side) sits at -h + k*w on each axis.
 *
 * Every grid-line crossing strictly between entry and exit is collected,
 * together with the entry and exit, and the list is sorted; each pair of
 * neighbours is one segment, whose pixel is the one containing its midpoint.
 * Segments of length <= 1e-12*w (corner ties) are dropped.
 *
 * work must hold 2*n_side + 4 doubles; pix/len must hold 2*n_side + 2.
 * Returns the number of segments written. */
EXPORT int oracle_siddon_ray(int n_side, double w, double c, double sn, double t,
                             int32_t *pix, double *len, double *work)
{
    const double h = 0.5 * (double)n_side * w;
    const double x0 = t * c;
    const double y0 = t * sn;
    double s_in = -INFINITY, s_out = INFINITY;

    if (sn != 0.0) {
        double sa = (x0 - (-h + 0.0 * w)) / sn;
        double sb = (x0 - (-h + (double)n_side * w)) / sn;
        s_in = fmax(s_in, fmin(sa, sb));
        s_out = fmin(s_out, fmax(sa, sb));
    } else if (!(x0 > -h && x0 < h)) {
        return 0;
    }
    if (c != 0.0) {
        double sa = ((-h + 0.0 * w) - y0) / c;
        double sb = ((-h + (double)n_side * w) - y0) / c;
        s_in = fmax(s_in, fmin(sa, sb));
        s_out = fmin(s_out, fmax(sa, sb));
    } else if (!(y0 > -h && y0 < h)) {
        return 0;
    }
    if (!(s_out > s_in)) return 0;

    int nv = 0;
    work[nv++] = s_in;
    if (sn != 0.0) {
        for (int k = 0; k <= n_side; ++k) {
            double sk = (x0 - (-h + (double)k * w)) / sn;
            if (sk > s_in && sk < s_out) work[nv++] = sk;
        }
    }
    if (c != 0.0) {
        for (int k = 0; k <= n_side; ++k) {
            double sk = ((-h + (double)k * w) - y0) / c;
            if (sk > s_in && sk < s_out) work[nv++] = sk;
        }
    }
    work[nv++] = s_out;
    qsort(work, (size_t)nv, sizeof(double), cmp_double);

    int nseg = 0;
    for (int q = 0; q + 1 < nv; ++q) {
        double L = work[q + 1] - work[q];
        if (L <= 1e-12 * w) continue;
        double sm = (work[q] + work[q + 1]) * 0.5;
        double xm = x0 - sm * sn;
        double ym = y0 + sm * c;
        int ix = (int)floor((xm + h) / w);
        int iy = (int)floor((ym + h) / w);
        if (ix < 0) ix = 0;
        if (ix > n_side - 1) ix = n_side - 1;
        if (iy < 0) iy = 0;
        if (iy > n_side - 1) iy = n_side - 1;
        pix[nseg] = iy * n_side + ix;
        len[nseg] = L;
        ++nseg;
    }
    return nseg;
}

/* Ray parameters for ray i (view-major). */
static void ray_params(int i, int n_bins, double bin_width, const double *cs,
                       double *c, double *sn, double *t)
{
    int v = i / n_bins, d = i % n_bins;
    *c = cs[2 * v];
    *sn = cs[2 * v + 1];
    *t = bin_centre(d, n_bins, bin_width);
}

/* Number of segments of every ray (row_nnz[m]); returns the total. */
EXPORT int64_t oracle_siddon_count(int n_side, int n_views, int n_bins, double w,
                                   double bin_width, double arc_deg, int32_t *row_nnz)
{
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)n_views);
    oracle_view_table(n_views, arc_deg, cs);
    const int m = n_views * n_bins;
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int32_t *pix = (int32_t *)malloc(sizeof(int32_t) * (2 * (size_t)n_side + 2));
        double *len = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 2));
        double *work = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 4));
#pragma omp for schedule(static)
        for (int i = 0; i < m; ++i) {
            double c, sn, t;
            ray_params(i, n_bins, bin_width, cs, &c, &sn, &t);
            int ns = oracle_siddon_ray(n_side, w, c, sn, t, pix, len, work);
            row_nnz[i] = ns;
            total += ns;
        }
        free(pix); free(len); free(work);
    }
    free(cs);
    return total;
}

/* Joseph's projector for one ray (the paper's matrices come from Joseph's
 * method, Sec. 3.1).  The ray {t (c, s) + u (-s, c)} is sampled once per
 * pixel row when |c| >= |s| (the ray runs closer to the y axis), else once per
 * pixel column, on the row's (column's) centre line.  Its position across
 * that line is interpolated linearly between the two nearest pixel centres,
 * and both weights are scaled by the ray length per row (column), w/|c|
 * (w/|s|).  Pixels outside the grid take no weight and zero weights are not
 * stored; entries come in sampling order, the lower pixel index of a pair
 * first.  pix/val must hold 2*n_side entries.  Returns the count. */
EXPORT int oracle_joseph_ray(int n_side, double w, double c, double s, double t, int32_t *pix,
                             double *val)
{
    const double h = 0.5 * (double)n_side * w;
    int n = 0;
    const int rows = fabs(c) >= fabs(s);
    const double L = w / (rows ? fabs(c) : fabs(s));
    for (int k = 0; k < n_side; ++k) {
        /* centre line of row (column) k, the ray's crossing point on it, and
         * its fractional pixel coordinate along the line */
        const double q = ((double)k + 0.5) * w - h;
        double p;
        if (rows) {
            const double a = (q - t * s) / c; /* x = t c - u s at y = q */
            p = t * c - s * a;
        } else {
            const double a = (t * c - q) / s; /* y = t s + u c at x = q */
            p = t * s + c * a;
        }
        const double fp = (p + h) / w - 0.5;
        const double fl = floor(fp);
        if (!(fl >= -1.0 && fl <= (double)n_side - 1.0)) continue;
        const double f = fp - fl;
        const int j = (int)fl;
        if (j >= 0) {
            pix[n] = rows ? k * n_side + j : j * n_side + k;
            val[n] = (1.0 - f) * L;
            ++n;
        }
        if (j + 1 < n_side && f > 0.0) {
            pix[n] = rows ? k * n_side + (j + 1) : (j + 1) * n_side + k;
            val[n] = f * L;
            ++n;
        }
    }
    return n;
}

EXPORT int64_t oracle_joseph_count_rays(int n_side, double w, int64_t m, const double *rays,
                                        int32_t *row_nnz)
{
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int32_t *pix = (int32_t *)malloc(sizeof(int32_t) * (2 * (size_t)n_side + 2));
        double *val = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 2));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            int ns = oracle_joseph_ray(n_side, w, rays[3 * i], rays[3 * i + 1], rays[3 * i + 2], pix, val);
            row_nnz[i] = ns;
            total += ns;
        }
        free(pix); free(val);
    }
    return total;
}

EXPORT void oracle_joseph_fill_rays(int n_side, double w, int64_t m, const double *rays,
                                    const int64_t *row_ptr, int32_t *col_idx, double *val)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        oracle_joseph_ray(n_side, w, rays[3 * i], rays[3 * i + 1], rays[3 * i + 2], col_idx + row_ptr[i],
                          val + row_ptr[i]);
}

/* As oracle_siddon_count / oracle_siddon_fill for an explicit ray table
 * rays[3i..3i+2] = (c, s, t) (any geometry, e.g. oracle_fan_rays). */
EXPORT int64_t oracle_siddon_count_rays(int n_side, double w, int64_t m, const double *rays,
                                        int32_t *row_nnz)
{
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int32_t *pix = (int32_t *)malloc(sizeof(int32_t) * (2 * (size_t)n_side + 2));
        double *len = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 2));
        double *work = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 4));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            int ns = oracle_siddon_ray(n_side, w, rays[3 * i], rays[3 * i + 1], rays[3 * i + 2], pix, len, work);
            row_nnz[i] = ns;
            total += ns;
        }
        free(pix); free(len); free(work);
    }
    return total;
}

EXPORT void oracle_siddon_fill_rays(int n_side, double w, int64_t m, const double *rays,
                                    const int64_t *row_ptr, int32_t *col_idx, double *val)
{
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 4));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            oracle_siddon_ray(n_side, w, rays[3 * i], rays[3 * i + 1], rays[3 * i + 2], col_idx + row_ptr[i],
                              val + row_ptr[i], work);
        free(work);
    }
}

/* CSR of the ray rows of A (m rows, n_side^2 columns), segments in walk order.
 * row_ptr[m+1] must already hold the exclusive prefix sum of the counts. */
EXPORT void oracle_siddon_fill(int n_side, int n_views, int n_bins, double w,
                               double bin_width, double arc_deg, const int64_t *row_ptr,
                               int32_t *col_idx, double *val)
{
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)n_views);
    oracle_view_table(n_views, arc_deg, cs);
    const int m = n_views * n_bins;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * (2 * (size_t)n_side + 4));
#pragma omp for schedule(static)
        for (int i = 0; i < m; ++i) {
            double c, sn, t;
            ray_params(i, n_bins, bin_width, cs, &c, &sn, &t);
            oracle_siddon_ray(n_side, w, c, sn, t, col_idx + row_ptr[i], val + row_ptr[i], work);
        }
        free(work);
    }
    free(cs);
}

/* Dense A~ = [A; sqrt_lambda*I] (column-major, M' x n, leading dimension lda)
 * from the CSR of A.  Entries of one ray that land on the same pixel are
 * summed in walk order.  The caller zeroes A first. */
EXPORT void oracle_dense_from_csr(int64_t m, int64_t n, const int64_t *row_ptr,
                                  const int32_t *col_idx, const double *val,
                                  double sqrt_lambda, double *A, int64_t lda)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
            A[i + (int64_t)col_idx[q] * lda] += val[q];
    if (sqrt_lambda > 0.0)
        for (int64_t j = 0; j < n; ++j) A[(m + j) + j * lda] = sqrt_lambda;
}

/* p = A x (ray rows only), FP64, for k images (x: n x k, p: m x k). */
EXPORT void oracle_forward(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                           const double *val, int64_t k, const double *x, int64_t ldx,
                           double *p, int64_t ldp)
{
    (void)n;
#pragma omp parallel for schedule(static) collapse(2)
    for (int64_t s = 0; s < k; ++s)
        for (int64_t i = 0; i < m; ++i) {
            double acc = 0.0;
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                acc += val[q] * x[col_idx[q] + s * ldx];
            p[i + s * ldp] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* Householder QR, LAPACK conventions (Sec. 2 Eq. 2; Sec. 2.1 'dgeqrf').      */
/* ------------------------------------------------------------------------ */

/* Reflector for column j: H = I - tau v v^T with v(0) = 1 that maps
 * x = A[j:, j] to beta*e1, beta = -sign(alpha)*||x||.  If the part of x below
 * its first entry is zero, tau = 0 and H = I.  Then H is applied to every
 * remaining column, one column at a time:  a <- a - tau*(v^T a)*v. */
EXPORT void oracle_householder_qr(int64_t M, int64_t n, double *A, int64_t lda, double *tau)
{
    for (int64_t j = 0; j < n && j < M; ++j) {
        double *x = A + j + j * lda;
        const int64_t len = M - j;
        double alpha = x[0];
        double ss = 0.0;
        for (int64_t i = 1; i < len; ++i) ss += x[i] * x[i];
        if (ss == 0.0) {
            tau[j] = 0.0;
            continue;
        }
        double norm = sqrt(alpha * alpha + ss);
        double beta = (alpha >= 0.0) ? -norm : norm;
        tau[j] = (beta - alpha) / beta;
        double scale = 1.0 / (alpha - beta);
        for (int64_t i = 1; i < len; ++i) x[i] *= scale;
        x[0] = beta;
        const double tj = tau[j];
#pragma omp parallel for schedule(static)
        for (int64_t k = j + 1; k < n; ++k) {
            double *a = A + j + k * lda;
            double dot = a[0];
            for (int64_t i = 1; i < len; ++i) dot += x[i] * a[i];
            double wk = tj * dot;
            a[0] -= wk;
            for (int64_t i = 1; i < len; ++i) a[i] -= wk * x[i];
        }
    }
}

/* B <- Q^T B for k right-hand sides (B is M x k): H_0 first, then H_1, ... */
EXPORT void oracle_apply_qt(int64_t M, int64_t n, const double *A, int64_t lda, const double *tau,
                            int64_t k, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < k; ++s) {
        double *b = B + s * ldb;
        for (int64_t j = 0; j < n && j < M; ++j) {
            if (tau[j] == 0.0) continue;
            const double *v = A + j + j * lda;
            double dot = b[j];
            for (int64_t i = 1; i < M - j; ++i) dot += v[i] * b[j + i];
            double wk = tau[j] * dot;
            b[j] -= wk;
            for (int64_t i = 1; i < M - j; ++i) b[j + i] -= wk * v[i];
        }
    }
}

/* B <- Q B for k right-hand sides: H_{n-1} first, down to H_0 (Q = H_0 H_1 ...). */
EXPORT void oracle_apply_q(int64_t M, int64_t n, const double *A, int64_t lda, const double *tau,
                           int64_t k, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < k; ++s) {
        double *b = B + s * ldb;
        for (int64_t j = ((n < M) ? n : M) - 1; j >= 0; --j) {
            if (tau[j] == 0.0) continue;
            const double *v = A + j + j * lda;
            double dot = b[j];
            for (int64_t i = 1; i < M - j; ++i) dot += v[i] * b[j + i];
            double wk = tau[j] * dot;
            b[j] -= wk;
            for (int64_t i = 1; i < M - j; ++i) b[j + i] -= wk * v[i];
        }
    }
}

/* Solve R X = C in place (C = first n rows of B), R = upper triangle of A[0:n, 0:n].
 * Back-substitution from the last unknown up (Sec. 2.1 'dtrsm'). */
EXPORT void oracle_backsolve(int64_t n, const double *A, int64_t lda, int64_t k, double *B, int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < k; ++s) {
        double *b = B + s * ldb;
        for (int64_t j = n - 1; j >= 0; --j) {
            b[j] /= A[j + j * lda];
            const double xj = b[j];
            for (int64_t i = 0; i < j; ++i) b[i] -= A[i + j * lda] * xj;
        }
    }
}

/* Solve R^T Y = G in place (forward substitution; R^T is lower triangular). */
EXPORT void oracle_forwardsolve_rt(int64_t n, const double *A, int64_t lda, int64_t k, double *B,
                                   int64_t ldb)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < k; ++s) {
        double *b = B + s * ldb;
        for (int64_t j = 0; j < n; ++j) {
            double acc = b[j];
            for (int64_t i = 0; i < j; ++i) acc -= A[i + j * lda] * b[i];
            b[j] = acc / A[j + j * lda];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Brute force and certificate, long double.                                  */
/* ------------------------------------------------------------------------ */

/* (A^T A + lambda I) x = A^T b by Cholesky in long double, A given as CSR of
 * its m ray rows.  G is formed ray by ray from the sparse rows.  For small n
 * only (G is n x n long double).  Returns 0, or j+1 if the pivot at j is not
 * positive. */
EXPORT int oracle_normal_eq_ld(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *val, double sqrt_lambda, int64_t k, const double *b,
                               int64_t ldb, double *x, int64_t ldx)
{
    long double *G = (long double *)calloc((size_t)(n * n), sizeof(long double));
    long double *y = (long double *)malloc(sizeof(long double) * (size_t)n);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                G[col_idx[p] + (int64_t)col_idx[q] * n] += (long double)val[p] * (long double)val[q];
    const long double lam = (long double)sqrt_lambda * (long double)sqrt_lambda;
    for (int64_t j = 0; j < n; ++j) G[j + j * n] += lam;
    /* Cholesky G = L L^T, L stored in the lower triangle. */
    for (int64_t j = 0; j < n; ++j) {
        long double d = G[j + j * n];
        for (int64_t p = 0; p < j; ++p) d -= G[j + p * n] * G[j + p * n];
        if (!(d > 0.0L)) { free(G); free(y); return (int)(j + 1); }
        d = sqrtl(d);
        G[j + j * n] = d;
        for (int64_t i = j + 1; i < n; ++i) {
            long double e = G[i + j * n];
            for (int64_t p = 0; p < j; ++p) e -= G[i + p * n] * G[j + p * n];
            G[i + j * n] = e / d;
        }
    }
    for (int64_t s = 0; s < k; ++s) {
        for (int64_t j = 0; j < n; ++j) y[j] = 0.0L;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                y[col_idx[p]] += (long double)val[p] * (long double)b[i + s * ldb];
        for (int64_t j = 0; j < n; ++j) { /* L z = y */
            long double e = y[j];
            for (int64_t p = 0; p < j; ++p) e -= G[j + p * n] * y[p];
            y[j] = e / G[j + j * n];
        }
        for (int64_t j = n - 1; j >= 0; --j) { /* L^T x = z */
            long double e = y[j];
            for (int64_t i = j + 1; i < n; ++i) e -= G[i + j * n] * y[i];
            y[j] = e / G[j + j * n];
        }
        for (int64_t j = 0; j < n; ++j) x[j + s * ldx] = (double)y[j];
    }
    free(G);
    free(y);
    return 0;
}

/* Residual of the regularised system, long double accumulation:
 *   r  = b~ - A~ x,  b~ = [b; 0],  A~ = [A; sqrt_lambda*I]   (r: (m+n) x k)
 *   g  = A~^T r                                               (g: n x k)
 * ||x - x*|| <= ||g|| / lambda since every singular value of A~ is at least
 * sqrt_lambda.  r and g are rounded to double on output. */
EXPORT void oracle_residual_ld(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *val, double sqrt_lambda, int64_t k, const double *b,
                               int64_t ldb, const double *x, int64_t ldx, double *r, int64_t ldr,
                               double *g, int64_t ldg)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < k; ++s) {
        long double *gs = (long double *)calloc((size_t)n, sizeof(long double));
        for (int64_t i = 0; i < m; ++i) {
            long double acc = (long double)b[i + s * ldb];
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                acc -= (long double)val[q] * (long double)x[col_idx[q] + s * ldx];
            if (r) r[i + s * ldr] = (double)acc;
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                gs[col_idx[q]] += (long double)val[q] * acc;
        }
        for (int64_t j = 0; j < n; ++j) {
            long double rj = -(long double)sqrt_lambda * (long double)x[j + s * ldx];
            if (r) r[m + j + s * ldr] = (double)rj;
            gs[j] += (long double)sqrt_lambda * rj;
            if (g) g[j + s * ldg] = (double)gs[j];
        }
        free(gs);
    }
}
