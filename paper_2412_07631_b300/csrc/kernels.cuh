// kernels.cuh -- internal entry points between the library's translation units.
#pragma once

#include "common.cuh"

namespace ctqr {

// ---- system build (siddon.cu) ---------------------------------------------------
struct SiddonArgs {
    int n_side, n_views, n_bins;
    double pixel_width, bin_width, sqrt_lambda;
    const double *d_cs;  // parallel: [2*n_views] (cos, sin) per view; fan: [3*m] (c, s, t) per ray
    int kind;            // CT_GEOM_PARALLEL / CT_GEOM_FAN
    int projector;       // CT_PROJ_SIDDON / CT_PROJ_JOSEPH
    int32_t *d_row_nnz;  // [m]
    int64_t *d_row_ptr;  // [m+1]
    int32_t *d_col;      // [nnz]
    double *d_val;       // [nnz]
    Scratch *tmp;
};
ct_status siddon_build(const SiddonArgs &a, cudaStream_t s);  // counts + row_ptr
ct_status siddon_fill(const SiddonArgs &a, void *dense, bool dense_fp64, int64_t lda,
                      cudaStream_t s);
ct_status exclusive_scan(const int32_t *in, int64_t n, int64_t *out_np1, Scratch &tmp,
                         cudaStream_t s);
ct_status build_csc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col_idx, const double *val, int64_t *col_ptr, int32_t *csc_row,
                    double *csc_val, Scratch &tmp, Scratch &tmp2, cudaStream_t s);

// ---- GEMM engines (gemm_simt.cu, gemm_tc.cu) ---------------------------------------
enum GemmKind : int { GEMM_F64 = 0, GEMM_F32 = 1, GEMM_TF32 = 2, GEMM_BF16 = 3, GEMM_TF32X3 = 4, GEMM_BF16X3 = 5 };
// Precision helpers shared by the factor constructors.
inline bool is_refine_prec(ct_precision p) { return p >= CT_TF32_REFINE && p <= CT_BF16X3_REFINE; }
// GEMMs of the solve (Q^T sweeps, triangular solves) and of the Gram and T
// blocks: TF32 for the single-pass refining precisions, TF32x3 for both
// split ones (close to FP32, so the preconditioner of the inner FP32 solves
// is as good as the split factor).
inline GemmKind solve_kind(ct_precision p) {
    switch (p) {
        case CT_FP64: return GEMM_F64;
        case CT_FP32: return GEMM_F32;
        case CT_TF32X3_REFINE:
        case CT_BF16X3_REFINE: return GEMM_TF32X3;
        default: return GEMM_TF32;
    }
}
inline bool tensor_kind(GemmKind k) { return k == GEMM_TF32 || k == GEMM_BF16 || k == GEMM_TF32X3 || k == GEMM_BF16X3; }
inline GemmKind update_kind(ct_precision p) {
    switch (p) {
        case CT_FP64: return GEMM_F64;
        case CT_FP32: return GEMM_F32;
        case CT_BF16_REFINE: return GEMM_BF16;
        case CT_TF32X3_REFINE: return GEMM_TF32X3;
        case CT_BF16X3_REFINE: return GEMM_BF16X3;
        default: return GEMM_TF32;
    }
}

struct GemmArgs {
    GemmKind kind;
    bool ta, tb;  // op(A) = A^T, op(B) = B^T
    int64_t M, N, K;
    double alpha;
    const void *A;
    int64_t lda;
    const void *B;
    int64_t ldb;
    double beta;
    void *C;
    int64_t ldc;
    int64_t min_chunk = 0;  // least split-K depth (0: the engine's default)
    // BF16 products only: op(A) already rounded to BF16 in the engine's
    // K-major layout (element (k, m) at A16 + k + m * lda16), or NULL
    const void *A16 = nullptr;
    int64_t lda16 = 0;
    // M == N and only C on and above the diagonal is wanted (a symmetric
    // product): the paired kernel skips its 256 x 256 tiles strictly below
    // the diagonal, whose part of C is then left undefined
    bool upper_only = false;
    // BF16 products only: op(B) already rounded to BF16, K-major (element
    // (k, n) at B16 + k + n * ldb16), or NULL
    const void *B16 = nullptr;
    int64_t ldb16 = 0;
    // TF32 / FP32 / FP64 products: when the engine splits K, leave the
    // partial products unreduced (*splits_out of them, each M x N with ld M,
    // at *partials_out in the engine's scratch) instead of writing C; the
    // caller sums them in split order, applies alpha and beta, and does so
    // before the scratch is used again.
    // *splits_out = 0 when C was written as usual.
    void **partials_out = nullptr;
    int *splits_out = nullptr;
};
// C = alpha op(A) op(B) + beta C (column-major).  Chooses split-K when the
// output has too few tiles for the machine; partial sums go through `ws`
// and are reduced in a fixed order (deterministic).
ct_status gemm(const GemmArgs &g, Scratch &ws, cudaStream_t s);

// Kernel-level launchers (no split logic): partial products over K range
// [k0, k0 + kc) of split z written to C + z*split_stride (alpha/beta applied).
// Split-K plan of the GEMM engine: the number of K splits and the depth of
// each (a multiple of align, at least min_chunk) for a grid of `tiles` output
// tiles, so that about two CTAs per SM are busy.
void plan_splits(int64_t tiles, int64_t K, int64_t min_chunk, int64_t align, int64_t *splits_out,
                 int64_t *kchunk_out);
ct_status gemm_simt_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                           cudaStream_t s);
ct_status gemm_tc_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                         cudaStream_t s);
// The same product on SM pairs (2-CTA clusters, 256 x 256 tiles); and the
// number of such tiles of an M x N output.
ct_status gemm_pair_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                           cudaStream_t s, DevStatus *status = nullptr);
int64_t gemm_pair_tiles(int64_t M, int64_t N);
// As gemm_tc_launch, with an explicit device status word and no accounting.
ct_status gemm_tc_launch_status(const GemmArgs &g, int splits, int64_t kchunk,
                                int64_t split_stride, DevStatus *status, cudaStream_t s);
// C = alpha * sum_z P[z] + beta * C  (P: splits x (M x N) packed, ld = M)
ct_status splitk_reduce(bool fp64, int64_t M, int64_t N, int splits, const void *P, double alpha,
                        double beta, void *C, int64_t ldc, cudaStream_t s);

// ---- factorisation pieces (panel.cu) -------------------------------------------------
// Householder QR of the panel A[j0:M, j0:j0+nb] in place (LAPACK convention),
// tau[j0:j0+nb].  Cooperative kernels: for FP32 panels of 32 columns with
// use_gram, the Gram-based kernel (two grid exchanges) and, only if it
// declined the panel, the column-by-column one (one exchange per column).
// With Tp, Vtp (ld ldt) given, the Gram path (or its fallback) also writes
// the panel's T_p and the unit-lower top of its V there and sets *made_t.
// With V16 given, those kernels also store the BF16 rounding of V below its
// top block (rows j0+32 .. M-1), row by row: element (r, k) at
// V16[(r - j0 - 32) * ld16 + k] (16-byte aligned, ld16 a multiple of 8), and
// set *made_v16.
ct_status panel_qr(bool fp64, void *A, int64_t lda, int64_t M, int64_t j0, int nb, void *tau,
                   Scratch &ws, cudaStream_t s, bool use_gram = true, void *Tp = nullptr,
                   void *Vtp = nullptr, int64_t ldt = 0, bool *made_t = nullptr, void *V16 = nullptr,
                   int64_t ld16 = 0, bool *made_v16 = nullptr);
// panel_gram.cu: the Gram-based kernel; ws as sized by panel_gram_ws_bytes(G);
// bar: 4 grid-meet counters the caller has zeroed on the stream;
// *fallback is set to 1 if the panel was left for the column-by-column kernel.
size_t panel_gram_ws_bytes(int G);
ct_status panel_gram(float *A, int64_t lda, int64_t M, int64_t j0, float *tau, void *ws, unsigned *bar,
                     int G, int64_t rows_per, int rpt, int *fallback, float *Tp, float *Vtp, int64_t ldt,
                     void *V16, int64_t ld16, cudaStream_t s);
// One grid meet that cannot complete (failure-detection check): returns
// CT_ERR_TIMEOUT once the bounded wait has given up.
ct_status wait_selftest(cudaStream_t s);
// Copy the unit-lower-triangular top block of V (nb x nb at A[j0, j0]) into
// Vtop (leading dimension ldv): ones on the diagonal, zeros above.
ct_status extract_vtop(bool fp64, const void *A, int64_t lda, int64_t j0, int nb, void *Vtop,
                       int64_t ldv, cudaStream_t s);
// T (nb x nb, upper triangular, leading dimension ldt) of the block reflector
// H = I - V T V^T from the Gram matrix G = V^T V (leading dimension ldg) and tau.
// T[0:o, o:o+wp] of an outer block reflector from its panel T_p and Gram
// matrix (FP32, o * 33 floats of shared memory; CT_ERR_UNSUPPORTED if larger).
ct_status t_assemble(int64_t o, int wp, const float *G, int64_t ldg, float *Tm, int64_t ldt,
                     cudaStream_t s);
ct_status larft_from_gram(bool fp64, int nb, const void *G, int64_t ldg, const void *tau, void *T,
                          int64_t ldt, cudaStream_t s);

// ---- triangular solves (trsm.cu) ---------------------------------------------------------
// Solve R X = C (upper, n x n, ld ldr) for k columns in place in C (ld ldc)
// (trans = false), or R^T X = C (trans = true).  Blocked: diagonal blocks by a
// SIMT kernel, off-diagonal updates by `gemm` of the given kind.
ct_status trsm_upper(GemmKind kind, bool trans, int64_t n, int64_t k, const void *R, int64_t ldr,
                     void *C, int64_t ldc, Scratch &ws, cudaStream_t s);

// ---- elementwise / layout helpers (util.cu) -----------------------------------------------
// K-major operand copy for split-precision products.  Each FP32 value x of
// op(src) (K x MN; src_kmajor: element (k, j) at src[k + j*lds], else at
// src[j + k*lds]) becomes hi = nearest value of the narrow type and
// lo = (x - hi) rounded the same way; the copy holds, along K' = 3K, the
// runs [hi, hi, lo] (second_operand = false) or [hi, lo, hi] (true), so one
// product of the two copies over K' sums hi*hi + hi*lo + lo*hi.  dst_kind 2:
// BF16; 3: TF32 values stored as FP32.  dst: element (k', j) at dst[k' + j*ldt].
ct_status split3_copy(const float *src, int64_t lds, bool src_kmajor, int dst_kind, bool second_operand,
                      void *dst, int64_t ldt, int64_t K, int64_t MN, cudaStream_t s);
// FP32 rows x cols (column-major, ld lds) rounded to BF16 into colm (same
// layout, ld ldc; skipped when NULL) and rowm (transposed: element (r, c) at
// c + r * ldr) with one read of the source.
ct_status convert_bf16_dual(const float *src, int64_t lds, int64_t rows, int64_t cols, void *colm, int64_t ldc,
                            void *rowm, int64_t ldr, cudaStream_t s);
ct_status copy_convert_2d(int src_kind, const void *src, int64_t lds, int dst_kind, void *dst,
                          int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s);
// 0 = float, 1 = double for src/dst kinds above.
// dst (cols x rows, ld ldd) = transpose of src (rows x cols, ld lds), with conversion.
ct_status transpose_any(int src_kind, const void *src, int64_t lds, int dst_kind, void *dst,
                        int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s);
ct_status transpose_d(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t rows,
                      int64_t cols, cudaStream_t s);
ct_status fill_zero_2d(bool fp64, void *dst, int64_t ld, int64_t rows, int64_t cols,
                       cudaStream_t s);
// Device status DEV_NONFINITE (site `where`) if the rows x cols block (kind
// 0 float, 1 double; column-major, leading dimension ld) holds a NaN or Inf.
ct_status scan_finite(int kind, const void *A, int64_t ld, int64_t rows, int64_t cols, int where,
                      cudaStream_t s);
ct_status rdiag_minmax(bool fp64, const void *A, int64_t lda, int64_t n, double *dmin_dmax_dev,
                       cudaStream_t s);

// ---- FP64 sparse products and refinement helpers (spmm.cu) -------------------------------
struct SparseSys {
    int64_t m, n, nnz;
    double sqrt_lambda;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    const int64_t *col_ptr;
    const int32_t *csc_row;
    const double *csc_val;
    const float *val32;      // FP32 copies of val / csc_val (NULL until made)
    const float *csc_val32;
    int64_t n_bins;          // ray rows are i = v * n_bins + d (0: no such order known)
    int64_t n_side;          // pixel columns are j = iy * n_side + ix (0: no such order known)
};
// Row-major (slice-fastest) k-column operands:  Y[i*k + s].
// out = alpha*Y + beta*(A~ X)   (rows m+n if sqrt_lambda > 0, else m)
ct_status spmm_ax(const SparseSys &S, int64_t k, const double *X, double alpha, const double *Y,
                  double beta, double *out, cudaStream_t s);
// out = alpha*Y + beta*(A~^T Rv)  (n rows)
ct_status spmm_atr(const SparseSys &S, int64_t k, const double *Rv, double alpha, const double *Y,
                   double beta, double *out, cudaStream_t s);
// The same products in FP32 (values val32/csc_val32, FP32 vectors and sums).
ct_status spmm_ax32(const SparseSys &S, int64_t k, const float *X, float alpha, const float *Y,
                    float beta, float *out, cudaStream_t s);
ct_status spmm_atr32(const SparseSys &S, int64_t k, const float *Rv, float alpha, const float *Y,
                     float beta, float *out, cudaStream_t s);

}  // namespace ctqr
