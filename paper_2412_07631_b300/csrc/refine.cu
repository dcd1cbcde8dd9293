// refine.cu -- FP64 iterative refinement on top of the low-precision factors.
//
// The direct solve x0 = R~^-1 [Q~^T b~]_{0:n} with TF32/BF16 factors carries
// an error of order kappa(A~) * u_low, and for the regularised, noisy
// problems kappa(A~) * u_low can exceed 1, where classical refinement
// (x += R~^-1 Q~^T (b~ - A~ x)) has the wrong fixed point or diverges.  The
// refinement here is two-level.
//
// Outer steps (FP64, at most refine_max_iter):
//     r = b~ - A~ x,  g = A~^T r        (exact sparse FP64 Siddon matrix)
//     stop if the certified bound ||g|| / (lambda ||x||) <= tol for every
//     slice (every singular value of A~ is >= sqrt_lambda, so it bounds
//     ||x - x*|| / ||x||); without regularisation rows, once the last
//     correction ||d|| / ||x|| was <= tol
//     x += d,  d ~ argmin_d || A~ d - r ||   (inner solve)
// Inner solve (FP32): conjugate gradients on the preconditioned normal
// equations of the correction problem min_d || A~ d - r ||,
//     (R~^-T A~^T A~ R~^-1) y = R~^-T g,   d = R~^-1 y,
// whose convergence depends on kappa(A~ R~^-1) (close to 1 when R~ is a good
// factor) rather than on kappa(A~).  The normal residual s is updated with
// products of the search direction only (s -= alpha R~^-T A~^T A~ t), never
// recomputed from r: for noisy data r keeps the large least-squares residual
// r* = b~ - A~ x*, and A~^T r taken in FP32 would drown the small part that
// the correction needs in r*'s rounding errors.  g = A~^T r itself comes from
// the FP64 outer step.  Vectors and sparse products are FP32 (FP32 copies of
// the Siddon values), inner products accumulate in FP64, triangular solves
// use the factor.  The inner solve stops once ||s|| of every slice has dropped
// by kInnerRed (or after kInnerMax steps).  An inexact correction only slows
// the outer contraction; the outer residual and the certificate are always
// FP64, so the FP32 inner arithmetic never limits the final accuracy.
//
// Inner step:  t = R~^-1 p,  q = A~ t,  alpha = gamma / ||q||^2,  d += alpha t,
//              s -= alpha R~^-T (A~^T q),  gamma' = ||s||^2,
//              p = s + (gamma'/gamma) p.
#include <algorithm>
#include <cmath>
#include <vector>

#include "handles.cuh"

namespace ctqr {

namespace {

constexpr int RB = 256;                // rows per reduction block
constexpr double kInnerRed = 1e-4;     // inner CGLS: relative reduction of ||s||
constexpr int kInnerMax = 40;          // inner CGLS: step limit per outer step

// part[b*k + s] = sum over rows [b*RB, (b+1)*RB) of U[i,s]*V[i,s] (row-major,
// slice fastest), accumulated in FP64
template <typename T>
__global__ void coldot_partial(int64_t rows, int64_t k, const T *U, const T *V, double *part) {
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int64_t r1 = min(rows, r0 + RB);
    for (int64_t s = threadIdx.x; s < k; s += blockDim.x) {
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) acc += (double)U[i * k + s] * (double)V[i * k + s];
        part[(int64_t)blockIdx.x * k + s] = acc;
    }
}

__global__ void coldot_final(int64_t nblk, int64_t k, const double *part, double *out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k) return;
    double acc = 0.0;
    for (int64_t b = 0; b < nblk; ++b) acc += part[b * k + s];
    out[s] = acc;
}

// Y[i,s] += sign * a[s] * X[i,s]   (a per slice)
template <typename T>
__global__ void axpy_cols(int64_t rows, int64_t k, const double *a, double sign, const T *X, T *Y) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    int64_t s = idx % k;
    Y[idx] += (T)(sign * a[s]) * X[idx];
}

// P[i,s] = S[i,s] + b[s] * P[i,s]
template <typename T>
__global__ void xpby_cols(int64_t rows, int64_t k, const T *S, const double *b, T *P) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    int64_t s = idx % k;
    P[idx] = S[idx] + (T)b[s] * P[idx];
}

// alpha[s] = gamma[s] / qq[s] (0 if qq is 0)
__global__ void step_scalars(int64_t k, const double *gamma, const double *qq, double *alpha) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k) return;
    alpha[s] = (qq[s] > 0.0) ? gamma[s] / qq[s] : 0.0;
}

__global__ void beta_scalars(int64_t k, const double *gnew, double *gamma, double *beta) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k) return;
    beta[s] = (gamma[s] > 0.0) ? gnew[s] / gamma[s] : 0.0;
    gamma[s] = gnew[s];
}

__global__ void to_f32_kernel(int64_t total, const double *src, float *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) dst[i] = (float)src[i];
}

// out = A - B (elementwise)
__global__ void sub_kernel(int64_t total, const double *A, const double *B, double *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) out[i] = A[i] - B[i];
}

// x += (double) d
__global__ void add_f32_kernel(int64_t total, const float *d, double *x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) x[i] += (double)d[i];
}

template <typename T>
ct_status launch_coldot(int64_t rows, int64_t k, const T *U, const T *V, double *part, double *out,
                        cudaStream_t s) {
    const int64_t nblk = ceil_div(rows, RB);
    coldot_partial<T><<<(unsigned)nblk, 128, 0, s>>>(rows, k, U, V, part);
    count_launch();
    coldot_final<<<(unsigned)ceil_div(k, 128), 128, 0, s>>>(nblk, k, part, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

static ct_status residual_sub(int64_t rows, int64_t k, const double *A, const double *B,
                              double *out, cudaStream_t s) {
    const int64_t total = rows * k;
    sub_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(total, A, B, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Per-slice inner products of row-major k-column blocks (deterministic order).
static ct_status coldot(int64_t rows, int64_t k, const double *U, const double *V, double *part,
                        double *out, cudaStream_t s) {
    return launch_coldot<double>(rows, k, U, V, part, out, s);
}

// t = R~^-1 u (trans = false) or R~^-T u (trans = true) for row-major u
// (n x k, FP64 or FP32 by u_kind 1/0): to the factor's column-major storage,
// triangular solve, back.
static ct_status apply_rinv(ct_factor f, bool trans, int u_kind, const void *u, void *t, int64_t k,
                            void *lp, cudaStream_t s) {
    const int64_t n = f->n, ldl = round_up(n, 32);
    const int dk = f->fp64 ? 1 : 0;
    CT_TRY(transpose_any(u_kind, u, k, dk, lp, ldl, k, n, s));  // (k x n row view) -> n x k col-major
    CT_TRY(trsm_factor(f, trans, lp, ldl, k, s));
    return transpose_any(dk, lp, ldl, u_kind, t, k, n, k, s);   // n x k col-major -> row-major
}
static ct_status apply_rinv(ct_factor f, bool trans, const double *u, double *t, int64_t k, void *lp,
                            cudaStream_t s) {
    return apply_rinv(f, trans, 1, u, t, k, lp, s);
}

// FP32 copies of the Siddon values for the inner solves (made once per system).
static ct_status ensure_f32_values(ct_system sys, cudaStream_t s) {
    if (sys->val32) return CT_OK;
    const int64_t nnz = std::max<int64_t>(sys->nnz, 1);
    float *a = nullptr, *b = nullptr;
    CT_CUDA(cudaMalloc(&a, sizeof(float) * nnz));
    if (cudaMalloc(&b, sizeof(float) * nnz) != cudaSuccess) {
        cudaFree(a);
        return CT_ERR_OOM;
    }
    const unsigned g = (unsigned)ceil_div(nnz, 256);
    if (sys->nnz > 0) {
        to_f32_kernel<<<g, 256, 0, s>>>(sys->nnz, sys->val, a);
        count_launch();
        to_f32_kernel<<<g, 256, 0, s>>>(sys->nnz, sys->csc_val, b);
        count_launch();
    }
    CT_CUDA(cudaGetLastError());
    sys->val32 = a;
    sys->csc_val32 = b;
    return CT_OK;
}

ct_status refine_run(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                     const ct_opts *o, cudaStream_t st, ct_solve_info *info) {
    const ct_system sys = f->sys;
    const int64_t n = f->n, m = f->m, M = f->M;
    const int max_outer = (o && o->refine_max_iter > 0) ? o->refine_max_iter : 10;
    const double tol = (o && o->refine_tol > 0) ? o->refine_tol : 1e-7;
    if (o && o->refine_max_iter < 0) return check_device_status(st);  // refinement disabled
    CT_TRY(ensure_f32_values(sys, st));
    const SparseSys S = sys->sparse();

    // workspace: FP64 x, r, b~, g | FP32 q, d, p, s, t, u | reductions | factor-precision n x k
    const int64_t nblk = ceil_div(std::max(M, n), RB);
    const size_t nk = (size_t)n * k, Mk = (size_t)M * k;
    const size_t ldl = round_up(n, 32);
    const size_t bytes = sizeof(double) * (2 * Mk + 2 * nk + (size_t)nblk * k + 12 * (size_t)k) +
                         sizeof(float) * (Mk + 5 * nk) + f->es() * ldl * k + 4096;
    CT_TRY(f->refine_ws.ensure(bytes));
    char *base = (char *)f->refine_ws.ptr;
    auto take = [&](size_t b) { char *p = base; base += round_up((int64_t)b, 256); return p; };
    double *r = (double *)take(sizeof(double) * Mk);
    double *btil = (double *)take(sizeof(double) * Mk);
    double *x = (double *)take(sizeof(double) * nk);
    double *g = (double *)take(sizeof(double) * nk);
    float *q = (float *)take(sizeof(float) * Mk);
    float *d = (float *)take(sizeof(float) * nk);
    float *p = (float *)take(sizeof(float) * nk);
    float *sv = (float *)take(sizeof(float) * nk);
    float *t = (float *)take(sizeof(float) * nk);
    float *u = (float *)take(sizeof(float) * nk);
    double *part = (double *)take(sizeof(double) * nblk * k);
    double *vec = (double *)take(sizeof(double) * 12 * k);
    void *lp = take(f->es() * ldl * k);
    double *gamma = vec, *qq = vec + k, *alpha = vec + 2 * k, *beta = vec + 3 * k, *gnew = vec + 4 * k,
           *gg = vec + 5 * k, *xx = vec + 6 * k, *dd = vec + 7 * k;
    const unsigned bn = (unsigned)ceil_div((int64_t)nk, 256), bk = (unsigned)ceil_div(k, 128);

    // per-slice scalars come back through pinned host memory: gg, xx, dd, gamma
    if (f->pinned_count < 4 * (size_t)k) {
        if (f->pinned) cudaFreeHost(f->pinned);
        f->pinned = nullptr;
        f->pinned_count = 0;
        CT_CUDA(cudaMallocHost((void **)&f->pinned, sizeof(double) * 4 * (size_t)k));
        f->pinned_count = 4 * (size_t)k;
    }
    double *h_gg = f->pinned, *h_xx = f->pinned + k, *h_dd = f->pinned + 2 * k, *h_gamma = f->pinned + 3 * k;
    std::vector<double> gamma0(k);

    // b~ (row-major, zero sqrt(lambda) rows), x0 (row-major)
    CT_CUDA(cudaMemsetAsync(btil, 0, sizeof(double) * Mk, st));
    CT_TRY(transpose_any(1, B, ldb, 1, btil, k, m, k, st));
    CT_TRY(transpose_any(1, X, ldx, 1, x, k, n, k, st));

    const bool use_cert = S.sqrt_lambda > 0.0;
    const double lam = S.sqrt_lambda * S.sqrt_lambda;

    // One inner CG step (captured once as a CUDA graph and replayed).
    auto inner_step = [&](cudaStream_t s2) -> ct_status {
        CT_TRY(apply_rinv(f, false, 0, p, t, k, lp, s2));              // t = R^-1 p
        CT_TRY(spmm_ax32(S, k, t, 0.0f, nullptr, 1.0f, q, s2));        // q = A~ t
        CT_TRY(launch_coldot<float>(M, k, q, q, part, qq, s2));
        step_scalars<<<bk, 128, 0, s2>>>(k, gamma, qq, alpha);
        count_launch();
        axpy_cols<float><<<bn, 256, 0, s2>>>(n, k, alpha, 1.0, t, d);   // d += a t
        count_launch();
        CT_TRY(spmm_atr32(S, k, q, 0.0f, nullptr, 1.0f, u, s2));       // u = A~^T q
        CT_TRY(apply_rinv(f, true, 0, u, u, k, lp, s2));               // w = R^-T u
        axpy_cols<float><<<bn, 256, 0, s2>>>(n, k, alpha, -1.0, u, sv);  // s -= a w
        count_launch();
        CT_TRY(launch_coldot<float>(n, k, sv, sv, part, gnew, s2));
        beta_scalars<<<bk, 128, 0, s2>>>(k, gnew, gamma, beta);
        count_launch();
        xpby_cols<float><<<bn, 256, 0, s2>>>(n, k, sv, beta, p);
        count_launch();
        CT_CUDA(cudaGetLastError());
        CT_CUDA(cudaMemcpyAsync(h_gamma, gamma, sizeof(double) * k, cudaMemcpyDeviceToHost, s2));
        return CT_OK;
    };
    const uint64_t key = graph_key(f, k, r) ^ ((uint64_t)M << 20) ^ 0x5152ull;

    int outer = 0, inner_total = 0;
    double last = INFINITY;
    bool converged = false, have_dd = false;
    while (true) {
        // FP64 residual, back-projection and the stopping quantity
        CT_TRY(spmm_ax(S, k, x, 1.0, btil, -1.0, r, st));        // r = b~ - A~ x
        CT_TRY(spmm_atr(S, k, r, 0.0, nullptr, 1.0, g, st));    // g = A~^T r
        CT_TRY(coldot(n, k, g, g, part, gg, st));
        CT_TRY(coldot(n, k, x, x, part, xx, st));
        CT_CUDA(cudaMemcpyAsync(h_gg, gg, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaMemcpyAsync(h_xx, xx, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        if (have_dd) CT_CUDA(cudaMemcpyAsync(h_dd, dd, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        double worst = 0.0;
        bool bad_data = false;  // NaN/Inf in the residual or the iterate
        for (int32_t sl = 0; sl < k; ++sl) {
            if (!std::isfinite(h_gg[sl]) || !std::isfinite(h_xx[sl]) || (have_dd && !std::isfinite(h_dd[sl])))
                bad_data = true;
            const double xn = std::max(std::sqrt(h_xx[sl]), 1e-300);
            double v;
            if (use_cert) v = std::sqrt(h_gg[sl]) / (lam * xn);
            else v = have_dd ? std::sqrt(h_dd[sl]) / xn : INFINITY;  // no measure before a step
            if (!std::isfinite(v)) { worst = INFINITY; continue; }
            worst = std::max(worst, v);
        }
        last = worst;
        if (worst <= tol) {
            converged = true;
            break;
        }
        // non-finite data cannot be refined away
        if (outer >= max_outer || bad_data) break;
        ++outer;
        // inner CG from y = 0: s = R^-T g with the FP64 back-projection g = A~^T r
        to_f32_kernel<<<bn, 256, 0, st>>>((int64_t)nk, g, u);
        count_launch();
        CT_CUDA(cudaGetLastError());
        CT_CUDA(cudaMemsetAsync(d, 0, sizeof(float) * nk, st));
        CT_TRY(apply_rinv(f, true, 0, u, sv, k, lp, st));       // s = R^-T g
        CT_CUDA(cudaMemcpyAsync(p, sv, sizeof(float) * nk, cudaMemcpyDeviceToDevice, st));
        CT_TRY(launch_coldot<float>(n, k, sv, sv, part, gamma, st));
        CT_CUDA(cudaMemcpyAsync(h_gamma, gamma, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaStreamSynchronize(st));
        for (int32_t sl = 0; sl < k; ++sl) gamma0[sl] = h_gamma[sl];
        for (int it = 0; it < kInnerMax; ++it) {
            CT_TRY(run_graphed(f, f->g_iter, key, st, inner_step));
            ++inner_total;
            CT_CUDA(cudaStreamSynchronize(st));
            double red = 0.0;
            for (int32_t sl = 0; sl < k; ++sl) {
                const double v = gamma0[sl] > 0.0 ? std::sqrt(h_gamma[sl] / gamma0[sl]) : 0.0;
                if (!std::isfinite(v)) { red = INFINITY; break; }
                red = std::max(red, v);
            }
            if (red <= kInnerRed) break;
        }
        // x += d (FP64 accumulation); ||d|| for the unregularised stop
        add_f32_kernel<<<bn, 256, 0, st>>>((int64_t)nk, d, x);
        count_launch();
        CT_CUDA(cudaGetLastError());
        CT_TRY(launch_coldot<float>(n, k, d, d, part, dd, st));
        have_dd = true;
    }
    CT_TRY(transpose_any(1, x, k, 1, X, ldx, k, n, st));  // row-major -> X (n x k col-major)
    if (info) {
        info->iterations = outer;
        info->inner_iterations = inner_total;
        info->stop_measure = last;
    }
    CT_TRY(check_device_status(st));
    if (!converged) {
        set_error("refinement: %d steps, stopping measure %.3g > tol %.3g", outer, last, tol);
        return CT_ERR_NOCONV;
    }
    return CT_OK;
}

// Adjoint of the refined solve map b -> x*(b) = (A~^T A~)^-1 A~^T b~ (a linear
// map once the refinement has converged): grad_b = [A~ u]_{0:m} with
// A~^T A~ u = grad_x.  u is found by preconditioned CG on the normal
// equations with M = R~^T R~ (two triangular solves with the low-precision
// factor), every vector and inner product in FP64 and the products A~^T A~ p
// formed with the sparse FP64 Siddon matrix.  Stop (sqrt_lambda > 0) when the
// certified bound ||g - A~^T A~ u|| / (lambda ||u||) >= ||u - u*|| / ||u||
// is <= tol for every slice, verified on a recomputed residual; without
// regularisation rows when the relative update is <= tol.
ct_status adjoint_refine_run(ct_factor f, const void *gX, int64_t ldgx, int32_t k, void *gB,
                             int64_t ldgb, const ct_opts *o, cudaStream_t st,
                             ct_solve_info *info) {
    const ct_system sys = f->sys;
    const SparseSys S = sys->sparse();
    const int64_t n = f->n, m = f->m, M = f->M;
    const int max_iter = (o && o->refine_max_iter > 0) ? o->refine_max_iter : 10;
    const double tol = (o && o->refine_tol > 0) ? o->refine_tol : 1e-7;
    const int64_t nblk = ceil_div(std::max(M, n), RB);
    const size_t nk = (size_t)n * k, Mk = (size_t)M * k;
    const size_t ldl = round_up(n, 32);
    const size_t bytes = sizeof(double) * (Mk + 6 * nk + (size_t)nblk * k + 8 * (size_t)k) +
                         f->es() * ldl * k + 1024;
    CT_TRY(f->refine_ws.ensure(bytes));
    char *base = (char *)f->refine_ws.ptr;
    auto take = [&](size_t b) { char *p = base; base += round_up((int64_t)b, 256); return p; };
    double *q = (double *)take(sizeof(double) * Mk);   // A~ p (M' x k)
    double *g = (double *)take(sizeof(double) * nk);   // right-hand side (row-major)
    double *u = (double *)take(sizeof(double) * nk);
    double *r = (double *)take(sizeof(double) * nk);
    double *z = (double *)take(sizeof(double) * nk);
    double *p = (double *)take(sizeof(double) * nk);
    double *w = (double *)take(sizeof(double) * nk);   // A~^T A~ p
    double *part = (double *)take(sizeof(double) * nblk * k);
    double *vec = (double *)take(sizeof(double) * 8 * k);
    void *lp = take(f->es() * ldl * k);
    double *rho = vec, *pw = vec + k, *alpha = vec + 2 * k, *beta = vec + 3 * k,
           *rnew = vec + 4 * k, *rr = vec + 5 * k, *uu = vec + 6 * k, *pp = vec + 7 * k;
    const unsigned bn = (unsigned)ceil_div((int64_t)nk, 256), bk = (unsigned)ceil_div(k, 128);
    const bool use_cert = S.sqrt_lambda > 0.0;
    const double lam = S.sqrt_lambda * S.sqrt_lambda;

    // normal-equations product: out = A~^T (A~ v)
    auto normal = [&](const double *v, double *out) -> ct_status {
        CT_TRY(spmm_ax(S, k, v, 0.0, nullptr, 1.0, q, st));
        return spmm_atr(S, k, q, 0.0, nullptr, 1.0, out, st);
    };
    auto precond = [&](const double *v, double *out) -> ct_status {  // out = R^-1 R^-T v
        CT_TRY(apply_rinv(f, true, v, out, k, lp, st));
        return apply_rinv(f, false, out, out, k, lp, st);
    };
    CT_TRY(transpose_any(1, gX, ldgx, 1, g, k, n, k, st));
    // u0 = M^-1 g ; r = g - A~^T A~ u0 ; z = M^-1 r ; p = z ; rho = <r, z>
    CT_TRY(precond(g, u));
    // r = g - w  (w = A~^T A~ u)
    CT_TRY(normal(u, w));
    CT_TRY(residual_sub(n, k, g, w, r, st));
    CT_TRY(precond(r, z));
    CT_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
    CT_TRY(coldot(n, k, r, z, part, rho, st));

    std::vector<double> h_rr(k), h_uu(k), h_pp(k), h_al(k);
    auto measure = [&](bool with_update) -> ct_status {
        CT_TRY(coldot(n, k, r, r, part, rr, st));
        CT_TRY(coldot(n, k, u, u, part, uu, st));
        CT_CUDA(cudaMemcpyAsync(h_rr.data(), rr, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CT_CUDA(cudaMemcpyAsync(h_uu.data(), uu, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        if (with_update) {
            CT_TRY(coldot(n, k, p, p, part, pp, st));
            CT_CUDA(cudaMemcpyAsync(h_pp.data(), pp, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            CT_CUDA(cudaMemcpyAsync(h_al.data(), alpha, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        }
        CT_CUDA(cudaStreamSynchronize(st));
        return CT_OK;
    };
    auto stop_value = [&](bool with_update) {
        double worst = 0.0;
        for (int32_t s2 = 0; s2 < k; ++s2) {
            const double un = std::max(std::sqrt(h_uu[s2]), 1e-300);
            double v = use_cert ? std::sqrt(h_rr[s2]) / (lam * un)
                                : (with_update ? std::fabs(h_al[s2]) * std::sqrt(h_pp[s2]) / un : INFINITY);
            if (!std::isfinite(v)) return (double)INFINITY;
            worst = std::max(worst, v);
        }
        return worst;
    };
    int it = 0;
    double last = INFINITY;
    bool converged = false;
    while (it < max_iter) {
        ++it;
        CT_TRY(normal(p, w));                                 // w = A~^T A~ p
        CT_TRY(coldot(n, k, p, w, part, pw, st));
        step_scalars<<<bk, 128, 0, st>>>(k, rho, pw, alpha);  // alpha = rho / <p, w>
        count_launch();
        axpy_cols<double><<<bn, 256, 0, st>>>(n, k, alpha, 1.0, p, u);   // u += a p
        count_launch();
        axpy_cols<double><<<bn, 256, 0, st>>>(n, k, alpha, -1.0, w, r);  // r -= a w
        count_launch();
        CT_TRY(measure(true));
        last = stop_value(true);
        bool bad_data = false;  // NaN/Inf in the residual or the iterate: no step can fix it
        for (int32_t s2 = 0; s2 < k; ++s2)
            if (!std::isfinite(h_rr[s2]) || !std::isfinite(h_uu[s2])) bad_data = true;
        if (bad_data) break;
        if (last <= tol) {
            if (!use_cert) { converged = true; break; }
            CT_TRY(normal(u, w));                              // verify on the true residual
            CT_TRY(residual_sub(n, k, g, w, r, st));
            CT_TRY(measure(false));
            last = stop_value(false);
            if (last <= tol) { converged = true; break; }
            CT_TRY(precond(r, z));                             // restart from it
            CT_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
            CT_TRY(coldot(n, k, r, z, part, rho, st));
            continue;
        }
        CT_TRY(precond(r, z));
        CT_TRY(coldot(n, k, r, z, part, rnew, st));
        beta_scalars<<<bk, 128, 0, st>>>(k, rnew, rho, beta);
        count_launch();
        xpby_cols<double><<<bn, 256, 0, st>>>(n, k, z, beta, p);      // p = z + b p
        count_launch();
        CT_CUDA(cudaGetLastError());
    }
    // grad_b = [A~ u]_{0:m}: the ray rows of the forward product
    CT_TRY(spmm_ax(S, k, u, 0.0, nullptr, 1.0, q, st));
    CT_TRY(transpose_any(1, q, k, 1, gB, ldgb, k, m, st));  // rows 0..m-1 (row-major) -> m x k
    if (info) {
        info->iterations = it;
        info->inner_iterations = it;
        info->stop_measure = last;
        info->rjj_min_abs = f->rjj_min;
        info->rjj_max_abs = f->rjj_max;
    }
    CT_TRY(check_device_status(st));
    if (!converged) {
        set_error("adjoint refinement: %d steps, stopping measure %.3g > tol %.3g", it, last, tol);
        return CT_ERR_NOCONV;
    }
    return CT_OK;
}

}  // namespace ctqr
