// refine.cu -- FP64 iterative refinement on top of the low-precision factors.
//
// The direct solve x0 = R~^-1 [Q~^T b~]_{0:n} with TF32/BF16 factors carries
// an error of order kappa(A~) * u_low, and for the regularised, noisy
// problems kappa(A~) * u_low can exceed 1, where classical refinement
// (x += R~^-1 Q~^T (b~ - A~ x)) has the wrong fixed point or diverges.  The
// refinement here is Krylov-based: CGLS on the right-preconditioned problem
//     min_y || A~ R~^-1 y - r0 ||,   r0 = b~ - A~ x0,   x = x0 + R~^-1 y,
// whose convergence depends on kappa(A~ R~^-1) (close to 1 when R~ is a good
// factor) rather than on kappa(A~).  The iterate x, the residual r, the
// search directions and every inner product are FP64; the residual and the
// back-projection use the exact sparse FP64 Siddon matrix (never the
// low-precision dense copy); only the two triangular solves with R~ per step
// run in the factor's precision.  Each slice has its own step lengths.
//
// Per step:  t = R~^-1 p,  q = A~ t,  alpha = gamma / ||q||^2,
//            x += alpha t,  r -= alpha q,  s = R~^-T (A~^T r),
//            gamma' = ||s||^2,  p = s + (gamma'/gamma) p.
// Stop (regularised systems) when the certified relative error bound
// ||A~^T r|| / (lambda ||x||) is <= tol for every slice, verified on a
// recomputed residual; without regularisation rows when the relative update
// ||alpha t|| / ||x|| is <= tol; or after max_iter steps (CT_ERR_NOCONV, x
// holds the last iterate).
#include <algorithm>
#include <cmath>
#include <vector>

#include "handles.cuh"

namespace ctqr {

namespace {

constexpr int RB = 256;  // rows per reduction block

// part[b*k + s] = sum over rows [b*RB, (b+1)*RB) of U[i,s]*V[i,s] (row-major, slice fastest)
__global__ void coldot_partial(int64_t rows, int64_t k, const double *U, const double *V,
                               double *part) {
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int64_t r1 = min(rows, r0 + RB);
    for (int64_t s = threadIdx.x; s < k; s += blockDim.x) {
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) acc += U[i * k + s] * V[i * k + s];
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

// Y[i,s] += a[s] * X[i,s]   (a per slice)
__global__ void axpy_cols(int64_t rows, int64_t k, const double *a, double sign, const double *X,
                          double *Y) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    int64_t s = idx % k;
    Y[idx] += sign * a[s] * X[idx];
}

// P[i,s] = S[i,s] + b[s] * P[i,s]
__global__ void xpby_cols(int64_t rows, int64_t k, const double *S, const double *b, double *P) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    int64_t s = idx % k;
    P[idx] = S[idx] + b[s] * P[idx];
}

// alpha[s] = gamma[s] / qq[s] (0 if qq is 0);  upd[s] = alpha^2 * tt[s]
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

// out = A - B (elementwise)
__global__ void sub_kernel(int64_t total, const double *A, const double *B, double *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) out[i] = A[i] - B[i];
}

struct Ws {
    double *x, *r, *p, *s, *t, *q, *btil;  // row-major FP64
    double *part, *vec;                    // reductions
    void *lp;                              // low-precision column-major n x k
};

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
    const int64_t nblk = ceil_div(rows, RB);
    coldot_partial<<<(unsigned)nblk, 128, 0, s>>>(rows, k, U, V, part);
    count_launch();
    coldot_final<<<(unsigned)ceil_div(k, 128), 128, 0, s>>>(nblk, k, part, out);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// t = R~^-1 u (trans = false) or R~^-T u (trans = true) for row-major FP64 u (n x k):
// convert to the factor's column-major storage, triangular solve, convert back.
static ct_status apply_rinv(ct_factor f, bool trans, const double *u, double *t, int64_t k,
                            void *lp, cudaStream_t s) {
    const int64_t n = f->n, ldl = round_up(n, 32);
    const int dk = f->fp64 ? 1 : 0;
    CT_TRY(transpose_any(1, u, k, dk, lp, ldl, k, n, s));  // (k x n row view) -> n x k col-major
    CT_TRY(trsm_factor(f, trans, lp, ldl, k, s));
    return transpose_any(dk, lp, ldl, 1, t, k, n, k, s);   // n x k col-major -> row-major
}

ct_status refine_run(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                     const ct_opts *o, cudaStream_t st, ct_solve_info *info) {
    const ct_system sys = f->sys;
    const SparseSys S = sys->sparse();
    const int64_t n = f->n, m = f->m, M = f->M;
    const int max_iter = (o && o->refine_max_iter > 0) ? o->refine_max_iter : 10;
    const double tol = (o && o->refine_tol > 0) ? o->refine_tol : 1e-7;
    if (o && o->refine_max_iter < 0) return check_device_status(st);  // refinement disabled

    // workspace
    const int64_t nblk = ceil_div(std::max(M, n), RB);
    const size_t nk = (size_t)n * k, Mk = (size_t)M * k;
    const size_t ldl = round_up(n, 32);
    const size_t bytes = sizeof(double) * (3 * Mk + 4 * nk + (size_t)nblk * k + 8 * (size_t)k) +
                         f->es() * ldl * k + 1024;
    CT_TRY(f->refine_ws.ensure(bytes));
    char *base = (char *)f->refine_ws.ptr;
    auto take = [&](size_t b) { char *p = base; base += round_up((int64_t)b, 256); return p; };
    Ws w;
    w.r = (double *)take(sizeof(double) * Mk);
    w.q = (double *)take(sizeof(double) * Mk);
    w.btil = (double *)take(sizeof(double) * Mk);
    w.x = (double *)take(sizeof(double) * nk);
    w.p = (double *)take(sizeof(double) * nk);
    w.s = (double *)take(sizeof(double) * nk);
    w.t = (double *)take(sizeof(double) * nk);
    w.part = (double *)take(sizeof(double) * nblk * k);
    w.vec = (double *)take(sizeof(double) * 8 * k);
    w.lp = take(f->es() * ldl * k);
    double *gamma = w.vec, *qq = w.vec + k, *alpha = w.vec + 2 * k, *beta = w.vec + 3 * k,
           *gnew = w.vec + 4 * k, *tt = w.vec + 5 * k, *xx = w.vec + 6 * k;
    const unsigned bn = (unsigned)ceil_div((int64_t)nk, 256), bk = (unsigned)ceil_div(k, 128);

    // b~ (row-major, zero sqrt(lambda) rows), x0 (row-major)
    CT_CUDA(cudaMemsetAsync(w.btil, 0, sizeof(double) * Mk, st));
    CT_TRY(transpose_any(1, B, ldb, 1, w.btil, k, m, k, st));
    CT_TRY(transpose_any(1, X, ldx, 1, w.x, k, n, k, st));
    // r = b~ - A~ x0 ; s = R^-T A~^T r ; p = s ; gamma = ||s||^2
    CT_TRY(spmm_ax(S, k, w.x, 1.0, w.btil, -1.0, w.r, st));
    CT_TRY(spmm_atr(S, k, w.r, 0.0, nullptr, 1.0, w.t, st));
    CT_TRY(apply_rinv(f, true, w.t, w.s, k, w.lp, st));
    CT_CUDA(cudaMemcpyAsync(w.p, w.s, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
    CT_TRY(coldot(n, k, w.s, w.s, w.part, gamma, st));

    // Stopping quantity.  Regularised systems (sqrt_lambda > 0): the certified
    // bound ||x - x*|| / ||x|| <= ||A~^T r|| / (lambda ||x||) (every singular
    // value of A~ is >= sqrt_lambda), with r the FP64 residual; once the
    // recursively updated residual meets it, the residual is recomputed from
    // scratch (r = b~ - A~ x) and the bound checked again, restarting CG from
    // the true residual if it fails.  Otherwise the relative update.
    const bool use_cert = S.sqrt_lambda > 0.0;
    const double lam = S.sqrt_lambda * S.sqrt_lambda;
    double *gg = w.vec + 7 * k;
    // per-slice scalars come back through pinned host memory (tt, xx, alpha, gg)
    if (f->pinned_count < 4 * (size_t)k) {
        if (f->pinned) cudaFreeHost(f->pinned);
        f->pinned = nullptr;
        f->pinned_count = 0;
        CT_CUDA(cudaMallocHost((void **)&f->pinned, sizeof(double) * 4 * (size_t)k));
        f->pinned_count = 4 * (size_t)k;
    }
    double *h_tt = f->pinned, *h_xx = f->pinned + k, *h_alpha = f->pinned + 2 * k,
           *h_gg = f->pinned + 3 * k;
    auto read_back = [&](bool with_update, cudaStream_t s2) -> ct_status {
        if (with_update) {
            CT_CUDA(cudaMemcpyAsync(h_tt, tt, sizeof(double) * k, cudaMemcpyDeviceToHost, s2));
            CT_CUDA(cudaMemcpyAsync(h_alpha, alpha, sizeof(double) * k, cudaMemcpyDeviceToHost, s2));
        }
        CT_CUDA(cudaMemcpyAsync(h_xx, xx, sizeof(double) * k, cudaMemcpyDeviceToHost, s2));
        CT_CUDA(cudaMemcpyAsync(h_gg, gg, sizeof(double) * k, cudaMemcpyDeviceToHost, s2));
        return CT_OK;
    };
    auto cert_of = [&]() {
        double worst = 0.0;
        for (int32_t q = 0; q < k; ++q) {
            const double v = std::sqrt(h_gg[q]) / (lam * std::max(std::sqrt(h_xx[q]), 1e-300));
            if (!std::isfinite(v)) return (double)INFINITY;
            worst = std::max(worst, v);
        }
        return worst;
    };
    // One CGLS step (captured once as a CUDA graph and replayed).
    auto step = [&](cudaStream_t s2) -> ct_status {
        CT_TRY(apply_rinv(f, false, w.p, w.t, k, w.lp, s2));       // t = R^-1 p
        CT_TRY(spmm_ax(S, k, w.t, 0.0, nullptr, 1.0, w.q, s2));    // q = A~ t
        CT_TRY(coldot(M, k, w.q, w.q, w.part, qq, s2));
        step_scalars<<<bk, 128, 0, s2>>>(k, gamma, qq, alpha);
        count_launch();
        axpy_cols<<<bn, 256, 0, s2>>>(n, k, alpha, 1.0, w.t, w.x);  // x += a t
        count_launch();
        axpy_cols<<<(unsigned)ceil_div((int64_t)Mk, 256), 256, 0, s2>>>(M, k, alpha, -1.0, w.q, w.r);  // r -= a q
        count_launch();
        CT_TRY(coldot(n, k, w.t, w.t, w.part, tt, s2));
        CT_TRY(coldot(n, k, w.x, w.x, w.part, xx, s2));
        CT_TRY(spmm_atr(S, k, w.r, 0.0, nullptr, 1.0, w.t, s2));   // t = A~^T r (reuse)
        CT_TRY(coldot(n, k, w.t, w.t, w.part, gg, s2));
        CT_TRY(apply_rinv(f, true, w.t, w.s, k, w.lp, s2));        // s = R^-T t
        CT_TRY(coldot(n, k, w.s, w.s, w.part, gnew, s2));
        beta_scalars<<<bk, 128, 0, s2>>>(k, gnew, gamma, beta);
        count_launch();
        xpby_cols<<<bn, 256, 0, s2>>>(n, k, w.s, beta, w.p);
        count_launch();
        CT_CUDA(cudaGetLastError());
        return read_back(true, s2);
    };
    const uint64_t key = graph_key(f, k, w.r) ^ ((uint64_t)M << 20) ^ 0x5151ull;
    int it = 0;
    double last = INFINITY;
    bool converged = false;
    while (it < max_iter) {
        ++it;
        CT_TRY(run_graphed(f, f->g_iter, key, st, step));
        CT_CUDA(cudaStreamSynchronize(st));
        double worst = 0.0;
        if (use_cert) {
            worst = cert_of();
        } else {
            for (int32_t q = 0; q < k; ++q) {
                const double xn = std::sqrt(h_xx[q]);
                const double up = std::fabs(h_alpha[q]) * std::sqrt(h_tt[q]);
                if (!std::isfinite(up)) { worst = INFINITY; break; }
                worst = std::max(worst, xn > 0 ? up / xn : up);
            }
        }
        last = worst;
        if (!(worst <= tol)) continue;
        if (!use_cert) {
            converged = true;
            break;
        }
        // verify with the residual recomputed from x
        CT_TRY(spmm_ax(S, k, w.x, 1.0, w.btil, -1.0, w.r, st));
        CT_TRY(spmm_atr(S, k, w.r, 0.0, nullptr, 1.0, w.t, st));
        CT_TRY(coldot(n, k, w.t, w.t, w.part, gg, st));
        CT_TRY(read_back(false, st));
        CT_CUDA(cudaStreamSynchronize(st));
        last = cert_of();
        if (last <= tol) {
            converged = true;
            break;
        }
        // restart from the true residual
        CT_TRY(apply_rinv(f, true, w.t, w.s, k, w.lp, st));
        CT_CUDA(cudaMemcpyAsync(w.p, w.s, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
        CT_TRY(coldot(n, k, w.s, w.s, w.part, gamma, st));
    }
    CT_TRY(transpose_any(1, w.x, k, 1, X, ldx, k, n, st));  // row-major -> X (n x k col-major)
    if (info) {
        info->iterations = it;
        info->stop_measure = last;
    }
    CT_TRY(check_device_status(st));
    if (!converged) {
        set_error("refinement: %d steps, stopping measure %.3g > tol %.3g", it, last, tol);
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
        axpy_cols<<<bn, 256, 0, st>>>(n, k, alpha, 1.0, p, u);   // u += a p
        count_launch();
        axpy_cols<<<bn, 256, 0, st>>>(n, k, alpha, -1.0, w, r);  // r -= a w
        count_launch();
        CT_TRY(measure(true));
        last = stop_value(true);
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
        xpby_cols<<<bn, 256, 0, st>>>(n, k, z, beta, p);      // p = z + b p
        count_launch();
        CT_CUDA(cudaGetLastError());
    }
    // grad_b = [A~ u]_{0:m}: the ray rows of the forward product
    CT_TRY(spmm_ax(S, k, u, 0.0, nullptr, 1.0, q, st));
    CT_TRY(transpose_any(1, q, k, 1, gB, ldgb, k, m, st));  // rows 0..m-1 (row-major) -> m x k
    if (info) {
        info->iterations = it;
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
