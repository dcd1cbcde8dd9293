// solve.cu -- X = R^-1 (Q^T b~) for a batch of sinograms (Sec. 2 Eq. 3:
// C = Q^T B by the stored reflector blocks, then R X = C by blocked
// back-substitution), and its adjoint gB = [Q [R^-T gX; 0]]_{0:m}.
#include <algorithm>

#include "handles.cuh"

namespace ctqr {

namespace {

// Element kind of caller buffers: float for a CT_FP32 factor, double otherwise.
inline int io_kind(ct_factor f) { return f->prec == CT_FP32 ? 0 : 1; }
inline int fac_kind(ct_factor f) { return f->fp64 ? 1 : 0; }

}  // namespace

// Low-precision (factor-precision) solve of the M' x k right-hand sides in Bt.
static ct_status direct_solve_inplace(ct_factor f, void *Bt, int64_t ldbt, int64_t k,
                                      cudaStream_t s) {
    CT_TRY(apply_q_blocks(f, true, Bt, ldbt, k, s));
    return trsm_factor(f, false, Bt, ldbt, k, s);
}

ct_status refine_run(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                     const ct_opts *o, cudaStream_t s, ct_solve_info *info);

ct_status solve_run(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                    const ct_opts *o, cudaStream_t s, ct_solve_info *info) {
    const int64_t M = f->M, m = f->m, n = f->n, ldbt = f->lda;
    CT_TRY(f->Bt.ensure(f->es() * (size_t)ldbt * k));
    void *Bt = f->Bt.ptr;
    CT_TRY(scan_finite(io_kind(f), B, ldb, m, k, 40, s));  // NaN/Inf sinograms: CT_ERR_NONFINITE
    CT_TRY(copy_convert_2d(io_kind(f), B, ldb, fac_kind(f), Bt, ldbt, m, k, s));
    if (M > m) CT_TRY(fill_zero_2d(f->fp64, (char *)Bt + f->es() * m, ldbt, M - m, k, s));
    CT_TRY(run_graphed(f, f->g_direct, graph_key(f, k, Bt), s,
                       [&](cudaStream_t st) { return direct_solve_inplace(f, Bt, ldbt, k, st); }));
    CT_TRY(copy_convert_2d(fac_kind(f), Bt, ldbt, io_kind(f), X, ldx, n, k, s));
    if (info) {
        info->iterations = 0;
        info->inner_iterations = 0;
        info->stop_measure = 0.0;
        info->rjj_min_abs = f->rjj_min;
        info->rjj_max_abs = f->rjj_max;
    }
    if (is_refine_prec(f->prec))
        return refine_run(f, B, ldb, k, X, ldx, o, s, info);
    return check_device_status(s);
}

ct_status adjoint_refine_run(ct_factor f, const void *gX, int64_t ldgx, int32_t k, void *gB,
                             int64_t ldgb, const ct_opts *o, cudaStream_t st, ct_solve_info *info);

ct_status adjoint_run(ct_factor f, const void *gX, int64_t ldgx, int32_t k, void *gB, int64_t ldgb,
                      const ct_opts *o, cudaStream_t s, ct_solve_info *info) {
    CT_TRY(scan_finite(io_kind(f), gX, ldgx, f->n, k, 41, s));  // NaN/Inf gradients: CT_ERR_NONFINITE
    if (is_refine_prec(f->prec) && !(o && o->refine_max_iter < 0))
        return adjoint_refine_run(f, gX, ldgx, k, gB, ldgb, o, s, info);
    const int64_t M = f->M, m = f->m, n = f->n, ldbt = f->lda;
    CT_TRY(f->Bt.ensure(f->es() * (size_t)ldbt * k));
    void *Bt = f->Bt.ptr;
    CT_TRY(copy_convert_2d(io_kind(f), gX, ldgx, fac_kind(f), Bt, ldbt, n, k, s));
    if (M > n) CT_TRY(fill_zero_2d(f->fp64, (char *)Bt + f->es() * n, ldbt, M - n, k, s));
    CT_TRY(trsm_factor(f, true, Bt, ldbt, k, s));
    CT_TRY(apply_q_blocks(f, false, Bt, ldbt, k, s));
    CT_TRY(copy_convert_2d(fac_kind(f), Bt, ldbt, io_kind(f), gB, ldgb, m, k, s));
    if (info) {
        info->iterations = 0;
        info->inner_iterations = 0;
        info->stop_measure = 0.0;
        info->rjj_min_abs = f->rjj_min;
        info->rjj_max_abs = f->rjj_max;
    }
    return check_device_status(s);
}

}  // namespace ctqr
