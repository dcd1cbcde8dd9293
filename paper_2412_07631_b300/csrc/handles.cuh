// handles.cuh -- the objects behind ct_system and ct_factor.
#pragma once

#include "kernels.cuh"

struct ct_system_s {
    ct_geometry geom{};
    bool fp64 = false;  // dense storage element type
    int64_t m = 0, n = 0, rows = 0, lda = 0, nnz = 0;
    void *dense = nullptr;  // column-major rows x n (NULL once consumed by a factor)
    double *d_cs = nullptr;
    int32_t *row_nnz = nullptr;
    int64_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    double *val = nullptr;
    int64_t *col_ptr = nullptr;
    int32_t *csc_row = nullptr;
    double *csc_val = nullptr;
    ctqr::Scratch tmp, tmp2;
    ctqr::SparseSys sparse() const {
        return {m, n, nnz, geom.sqrt_lambda, row_ptr, col, val, col_ptr, csc_row, csc_val};
    }
};

struct ct_factor_s {
    ct_system sys = nullptr;  // borrowed (sparse rows for FP64 refinement)
    ct_precision prec = CT_FP64;
    bool fp64 = true;
    ctqr::GemmKind kind = ctqr::GEMM_F64;
    int64_t M = 0, n = 0, m = 0, lda = 0;
    void *VR = nullptr;   // owned: R above the diagonal, V below
    void *tau = nullptr;  // owned: n scalars
    int NB = 0, nb = 0;   // outer block / panel widths
    int64_t nblocks = 0;
    void *Tall = nullptr;  // nblocks x (NB x NB), T_J of block J
    void *Vtop = nullptr;  // nblocks x (NB x NB), unit-lower top of V_J
    double rjj_min = 0, rjj_max = 0;
    // triangular-solve aids (built on first solve): inverse diagonal blocks of R
    // and their transposes (trsm_tb x trsm_tb each), R^T for the tensor-core path
    void *Rinv = nullptr, *RinvT = nullptr, *Rt = nullptr;
    int trsm_tb = 0;
    int64_t ldrt = 0;
    // work buffers
    ctqr::Scratch gemm_ws, W, W2, G, panel_ws, Bt, trsm_ws, refine_ws, host_pinned, misc, misc2;
    size_t es() const { return fp64 ? 8 : 4; }
};

namespace ctqr {
ct_status qr_factor_run(ct_factor f, cudaStream_t s);
// R X = C or R^T X = C in place for the factor's R (blocked, inverse diagonal blocks).
ct_status trsm_factor(ct_factor f, bool trans, void *C, int64_t ldc, int64_t k, cudaStream_t s);
// Apply Q^T (forward block order) or Q (reverse order) to the M x k matrix C.
ct_status apply_q_blocks(ct_factor f, bool transpose, void *C, int64_t ldc, int64_t k,
                         cudaStream_t s);
ct_status solve_run(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                    const ct_opts *o, cudaStream_t s, ct_solve_info *info);
ct_status adjoint_run(ct_factor f, const void *gX, int64_t ldgx, int32_t k, void *gB, int64_t ldgb,
                      const ct_opts *o, cudaStream_t s, ct_solve_info *info);
}  // namespace ctqr
