/*
 * ctqr.h -- C ABI of libctqr: direct algebraic CT reconstruction by dense
 * Householder QR on one B300 (sm_103a).
 *
 * The three operations follow the paper's statement of the problem
 * (arxiv 2412.07631, Sec. 2): build the system matrix A of the linear model
 * A X = B (Eq. 1), factor A = QR once (Eq. 2), and solve X = R^-1 (Q^T B)
 * for as many sinograms as share A (Eq. 3), with Q kept as Householder
 * reflectors and R^-1 applied by back-substitution, never formed.
 *
 * Conventions used by every call:
 *   - Dense matrices are column-major (Fortran/LAPACK): element (i, j) of a
 *     matrix with leading dimension ld is at p[i + j*ld].  Leading dimensions
 *     are in elements and must be >= the row count.
 *   - Ray (row) index i = v*n_bins + d (view v, detector bin d); pixel
 *     (column) index j = iy*n_side + ix.  The image has n = n_side^2 pixels,
 *     the scan m = n_views*n_bins rays.
 *   - With sqrt_lambda > 0 the factored matrix is A~ = [A; sqrt_lambda*I]
 *     with M' = m + n rows and the right-hand sides are b~ = [b; 0]
 *     (Tikhonov regularisation; the paper's A is square-ish and full rank,
 *     Sec. 3.1.1).  With sqrt_lambda = 0, M' = m and A must have full column
 *     rank.
 *   - "device" pointers are CUDA device addresses of the current device;
 *     "host" pointers are ordinary host memory.  The library never keeps a
 *     caller pointer after a call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated; results
 *     written to device memory are valid once the stream reaches the call.
 *   - Every call returns ct_status and never aborts the process.  A kernel
 *     that times out a bounded wait, or sees a non-finite value, records it in
 *     a device status word that the library reads at its synchronisation
 *     points and returns as CT_ERR_TIMEOUT / CT_ERR_NONFINITE.
 *
 * Ownership: the library owns the storage of a ct_system and a ct_factor
 * (device memory allocated by the library); the caller owns every buffer it
 * passes in.  Handles are not thread-safe: one host thread per handle.
 */
#ifndef CTQR_H
#define CTQR_H

#include <stdint.h>

#if defined(__GNUC__)
#define CT_API __attribute__((visibility("default")))
#else
#define CT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CT_OK = 0,
    CT_ERR_ARG = 1,         /* invalid argument (null pointer, bad size/leading dimension) */
    CT_ERR_OOM = 2,         /* device or pinned-host allocation failed */
    CT_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
    CT_ERR_RANK = 4,        /* |R_jj| < n * u * max|R_jj|: A~ is numerically rank deficient */
    CT_ERR_NOCONV = 5,      /* refinement hit its step limit; best X still written */
    CT_ERR_TIMEOUT = 6,     /* a bounded device-side wait expired; the kernel returned early */
    CT_ERR_NONFINITE = 7,   /* NaN/Inf in the matrix being factored (a reflector, R's diagonal)
                               or in the right-hand sides of a solve */
    CT_ERR_HOSTMEM = 8,     /* host memory (pinned/registered) could not be obtained */
    CT_ERR_STATE = 9,       /* handle in the wrong state (e.g. system already consumed) */
    CT_ERR_UNSUPPORTED = 10, /* option or combination the library does not support */
    CT_ERR_IO = 11,         /* a file read, write or sync failed (disk tier) */
    CT_ERR_INTERRUPTED = 12 /* stopped early on request (ct_opts.stop_after); resumable */
} ct_status;

/* Arithmetic of the factorisation and the solve.
 *  CT_FP64        FP64 storage and arithmetic throughout.
 *  CT_FP32        FP32 storage and arithmetic (the paper's single-precision
 *                 variant, Sec. 2.2 last paragraph and Sec. 3.1.2).
 *  CT_TF32_REFINE FP32 storage, trailing updates and Q^T applications on the
 *                 tensor cores with TF32 operands and FP32 accumulation, then
 *                 FP64 iterative refinement (residual and update in FP64).
 *  CT_BF16_REFINE as CT_TF32_REFINE with BF16 operands.
 *  CT_TF32X3_REFINE, CT_BF16X3_REFINE  split-precision trailing updates:
 *                 each FP32 operand x is split into x_hi (the nearest TF32 or
 *                 BF16 value) and x_lo (x - x_hi, rounded the same way), and
 *                 A B is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi on the
 *                 tensor cores (three times the flops of one product; close to
 *                 FP32 accuracy for TF32x3, about 16 bits for BF16x3), which
 *                 widens the range of conditioning the FP64 refinement
 *                 converges on.  Everything else as CT_TF32_REFINE. */
typedef enum {
    CT_FP64 = 0,
    CT_FP32 = 1,
    CT_TF32_REFINE = 2,
    CT_BF16_REFINE = 3,
    CT_TF32X3_REFINE = 4,
    CT_BF16X3_REFINE = 5
} ct_precision;

/* Parallel-beam scan geometry.  Pixels of width pixel_width tile the square
 * centred on the rotation axis; views at v*arc_deg/n_views degrees
 * (v = 0..n_views-1); bin d centred at (d - (n_bins-1)/2)*bin_width. */
typedef struct {
    int32_t n_side;
    int32_t n_views;
    int32_t n_bins;
    double pixel_width;  /* > 0, usually 1 */
    double bin_width;    /* > 0, usually 1 (parallel beam only) */
    double arc_deg;      /* usually 180 (parallel) or 360 (fan) */
    double sqrt_lambda;  /* >= 0; 0 = no regularisation rows */
    int32_t kind;        /* CT_GEOM_PARALLEL (0, the default) or CT_GEOM_FAN */
    double source_dist;  /* fan: source to rotation axis, > the image half-diagonal */
    double fan_deg;      /* fan: angle spanned by the n_bins detectors, in (0, 180) */
    int32_t projector;   /* CT_PROJ_SIDDON (0, the default) or CT_PROJ_JOSEPH */
} ct_geometry;

/* ct_geometry.projector.  Siddon: a_ij = exact length of ray i in pixel j.
 * Joseph (the method behind the paper's matrices, Sec. 3.1): the ray is
 * sampled once per pixel row when |cos theta| >= |sin theta| (else once per
 * pixel column) on the row's (column's) centre line; its position there is
 * interpolated linearly between the two nearest pixel centres, weights
 * scaled by the ray length per row (column); pixels outside the grid and
 * zero weights are dropped. */
#define CT_PROJ_SIDDON 0
#define CT_PROJ_JOSEPH 1

/* ct_geometry.kind.  Parallel beam: view v at theta_v = v * arc / n_views,
 * bin d at signed distance (d - (n_bins-1)/2) * bin_width from the axis.
 * Fan beam (the scanner of the paper's Sec. 3.1 / 3.2 tables): source v at
 * beta_v = v * arc / n_views and distance source_dist from the axis,
 * detector d of an equiangular arc at fan angle
 * gamma_d = (d - (n_bins-1)/2) * fan_deg / (n_bins-1) from the central ray
 * (which points from the source through the axis).  Ray i = v n_bins + d. */
#define CT_GEOM_PARALLEL 0
#define CT_GEOM_FAN 1

typedef struct {
    ct_precision precision;
    int32_t refine_max_iter; /* refinement step limit (0: 10; < 0: no refinement) */
    double refine_tol;       /* refinement stop (<= 0: 1e-7): with sqrt_lambda > 0, the certified
                                bound max_s ||A~^T r_s|| / (lambda ||x_s||) >= ||x_s - x*_s||/||x_s||;
                                without, the relative update max_s ||dx_s||/||x_s|| */
    int32_t nb_outer;        /* outer WY block width (0: automatic) */
    int32_t nb_inner;        /* panel width (0: automatic) */
    int32_t flags;           /* CT_OPT_* bits */
    int32_t stop_after;      /* disk-tier factorisation: return CT_ERR_INTERRUPTED after this
                                many superpanels (0: run to the end); the file stays resumable */
    int32_t solve_block;     /* solves with a tensor-core factor (TF32/BF16 and split kinds):
                                rows of the triangular solve's diagonal superblocks, each applied
                                as one GEMM with its stored inverse (0: 2048; otherwise 128 times
                                a power of two, at most 16384).  A change rebuilds the inverses. */
    int32_t solve_split;     /* solves: least depth of one split-K slice in the solve's GEMMs
                                (0: 256; otherwise a multiple of 32, at least 32) */
} ct_opts;

/* ct_opts.flags: by default the repeated parts of a solve (the Q^T sweep plus
 * the triangular solve, and each refinement step) are captured once per
 * batch size as CUDA graphs on a library-owned stream and replayed; this bit
 * runs them as individual launches instead.  (Per-launch timing from
 * ct_stats_reset(1) also disables graphs.) */
#define CT_OPT_NO_GRAPHS 1
/* ct_opts.flags for ct_qr_factor / ct_qr_factor_ooc: FP32-storage panels of
 * 32 columns are by default factored from two Gram matrices (CholeskyQR
 * twice, then the Householder reflectors reconstructed from the orthonormal
 * factor: the same reflectors in exact arithmetic, two grid-wide exchanges
 * per panel instead of 32), falling back to the column-by-column sweep for
 * a panel whose columns are nearly dependent in FP32; this bit always uses
 * the column-by-column sweep. */
#define CT_OPT_COLUMN_PANEL 2

typedef struct {
    int32_t iterations;       /* refinement steps taken: FP64 residual + correction
                                 (0 for CT_FP64 / CT_FP32) */
    double stop_measure;      /* the stopping quantity (see refine_tol) after the last step */
    double rjj_min_abs;       /* min |R_jj| */
    double rjj_max_abs;       /* max |R_jj| */
    int32_t inner_iterations; /* FP32 inner CGLS steps over all refinement steps
                                 (ct_solve; PCG steps for ct_solve_adjoint) */
} ct_solve_info;

typedef struct ct_system_s *ct_system;
typedef struct ct_factor_s *ct_factor;

/* Human-readable name of a status code (static string; "CT_ERR_UNKNOWN" for
 * a value outside ct_status).  Error reporting of the library; the paper has
 * no counterpart.  Cannot fail. */
CT_API const char *ct_status_str(ct_status s);

/* Detail of the last error raised on the calling thread (static per-thread
 * buffer, "" if none).  The paper has no counterpart.  Cannot fail. */
CT_API const char *ct_last_error(void);

/* Build the system matrix (Sec. 2 Eq. 1: a_ij = contribution of ray i to
 * pixel j), here the Siddon intersection length of ray i in pixel j.
 * On the device: the dense column-major A~ (M' x n, leading dimension lda,
 * `storage` = CT_FP64 -> double, otherwise float) and an FP64 CSR and CSC of
 * the m ray rows (for FP64 residuals).  The view table is computed once on
 * the host.  `out` receives a new handle; free it with ct_system_free.
 * Errors: CT_ERR_ARG (bad geometry), CT_ERR_OOM, CT_ERR_CUDA. */
CT_API ct_status ct_build_system(const ct_geometry *geom, ct_precision storage, void *stream,
                          ct_system *out);

/* Sizes of a built system: m rays and n pixels of A (Sec. 2 Eq. 1), the
 * rows M' of A~, the dense leading dimension and the CSR's nonzero count.
 * Any output pointer may be NULL.  Errors: CT_ERR_ARG (NULL handle). */
CT_API ct_status ct_system_info(ct_system sys, int64_t *m_rays, int64_t *n_pixels, int64_t *rows,
                         int64_t *lda, int64_t *nnz);

/* Device pointers to the system matrix of Sec. 2 Eq. 1 (owned by the
 * library, valid until ct_system_free; the dense pointer is NULL once ct_qr_factor consumed it).
 * row_ptr: int64[m+1]; col_idx: int32[nnz]; val: double[nnz] (CSR of A, ray
 * rows only, entries of a row in Siddon walk order).  Any output may be NULL.
 * Errors: CT_ERR_ARG (NULL handle). */
CT_API ct_status ct_system_device_ptrs(ct_system sys, void **dense, const int64_t **row_ptr,
                                const int32_t **col_idx, const double **val);

/* Copy the system matrix of Sec. 2 Eq. 1 to HOST buffers (synchronous; any
 * pointer may be NULL):
 * row_ptr int64[m+1], col_idx int32[nnz], val double[nnz] (CSR of the ray
 * rows, each row in Siddon walk order); dense: the column-major M' x n matrix
 * A~ in the storage type (double for CT_FP64, float otherwise) with leading
 * dimension ldd >= M'.  CT_ERR_STATE if dense is requested after
 * ct_qr_factor consumed it. */
CT_API ct_status ct_system_export(ct_system sys, int64_t *row_ptr, int32_t *col_idx, double *val,
                           void *dense, int64_t ldd);

/* P = A X on the device: the forward model of Sec. 2 Eq. 1 (sinograms of
 * images), with the CSR in FP64.  X: device double, n x k, ldx >= n; P:
 * device double, m x k, ldp >= m.  k = 0 does nothing (X and P may then be
 * NULL).  Errors: CT_ERR_ARG, CT_ERR_CUDA. */
CT_API ct_status ct_forward_project(ct_system sys, const double *X, int64_t ldx, int32_t k, double *P,
                             int64_t ldp, void *stream);

/* Householder QR of A~ (Sec. 2 Eq. 2; Sec. 2.1 'dgeqrf'), blocked: panels
 * of nb_inner columns are factored by reflectors H = I - tau v v^T
 * (v(0) = 1, beta = -sign(alpha)||x||, LAPACK convention), and the trailing
 * matrix is updated by compact-WY blocks of nb_outer columns,
 * C <- C - V T^T V^T C ... as (I - V T V^T)^T C.  The factorisation happens in
 * place: the system's dense storage moves into the factor (R in the upper
 * triangle, V below the diagonal), so the system's dense pointer becomes
 * NULL; its CSR stays with the system, which must outlive the factor when a
 * refining precision is used.  opts->precision must match the storage the
 * system was built with (CT_FP64 <-> double, others <-> float).
 * Synchronises `stream` at the end to check the device status and R's
 * diagonal.  Errors: CT_ERR_ARG, CT_ERR_STATE (already consumed), CT_ERR_RANK,
 * CT_ERR_NONFINITE, CT_ERR_TIMEOUT, CT_ERR_OOM, CT_ERR_CUDA. */
CT_API ct_status ct_qr_factor(ct_system sys, const ct_opts *opts, void *stream, ct_factor *out);

/* Device pointers of the factors of Sec. 2 Eq. 2: VR (M' x n, leading
 * dimension lda, R in the upper triangle, Householder vectors below), tau[n]
 * (same element type as VR).  For tests and checkpointing; owned by the
 * library.  Any output may be NULL.  Errors: CT_ERR_ARG (NULL handle),
 * CT_ERR_UNSUPPORTED (out-of-core factor: V and R are in host memory). */
CT_API ct_status ct_factor_device_ptrs(ct_factor f, void **VR, int64_t *lda, void **tau);

/* Copy the factors of Sec. 2 Eq. 2 to HOST buffers (synchronous; any
 * pointer may be NULL):
 * VR (M' x n, leading dimension ldv >= M', R on and above the diagonal,
 * Householder vectors below it), tau[n]; element type double for CT_FP64,
 * float otherwise.  Works for in-core, host-resident and disk-backed
 * factors.  Errors: CT_ERR_ARG (NULL handle, ldv < M'), CT_ERR_IO (disk
 * tier), CT_ERR_CUDA. */
CT_API ct_status ct_factor_export(ct_factor f, void *VR, int64_t ldv, void *tau);

/* X = R^-1 (Q^T b~) for k sinograms (Sec. 2 Eq. 3: C = Q^T B, then R X = C;
 * Sec. 2.1 'dormqr' + 'dtrsm').  B: device, m x k (ray rows only; the
 * library appends the zero rows of b~), ldb >= m.  X: device, n x k,
 * ldx >= n.  Element type: float for a CT_FP32 factor, double otherwise.
 * For refining factors, FP64 iterative refinement follows the first solve:
 * each step computes the residual b~ - A~ x and A~^T of it in FP64 with the
 * sparse Siddon matrix, then adds a correction found by FP32 CGLS on the
 * problem preconditioned with R~ (the low-precision factor), until the
 * stopping quantity of opts->refine_tol is met or refine_max_iter steps.
 * opts may be NULL (factor's precision, defaults).  info may be NULL.  k = 0
 * does nothing (B and X may then be NULL).
 * Synchronises `stream` at the end (to read the convergence state).
 * B is scanned on the device for NaN/Inf (one read of B): a non-finite
 * sinogram makes the call return CT_ERR_NONFINITE (X then holds what the
 * arithmetic produced; a refining factor stops refining at the first
 * non-finite stopping measure, info->stop_measure = inf).
 * Errors: CT_ERR_ARG, CT_ERR_NOCONV (X still holds the best iterate),
 * CT_ERR_NONFINITE, CT_ERR_TIMEOUT, CT_ERR_OOM, CT_ERR_CUDA. */
CT_API ct_status ct_solve(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                   const ct_opts *opts, void *stream, ct_solve_info *info);

/* Sec. 2 Eq. 3 as ct_solve, but B and X are HOST buffers; the host-to-device copy of B
 * and the device-to-host copy of X are part of the call (staged through
 * library-owned pinned buffers).  Blocks until X is written.
 * Errors: as ct_solve. */
CT_API ct_status ct_solve_host(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                        const ct_opts *opts, void *stream, ct_solve_info *info);

/* Adjoint of the solve map of Sec. 2 Eq. 3, b -> x = R^-1 [Q^T b~]_{0:n}
 * (the paper has no adjoint; it serves differentiation through the solve):
 * gB = [Q [R^-T gX; 0]]_{0:m}  (the gradient of a loss L(x) with respect to
 * b, given gX = dL/dx).  gX: device, n x k, ldgx >= n; gB: device, m x k,
 * ldgb >= m; element type as ct_solve.  For refining factors the adjoint is
 * taken in FP64 arithmetic on the FP32 factors followed by the same FP64
 * refinement applied to the transposed problem.  gX is scanned for NaN/Inf
 * as ct_solve scans B (CT_ERR_NONFINITE).
 * Errors: as ct_solve. */
CT_API ct_status ct_solve_adjoint(ct_factor f, const void *gX, int64_t ldgx, int32_t k, void *gB,
                           int64_t ldgb, const ct_opts *opts, void *stream, ct_solve_info *info);

/* ---- Out-of-core factorisation (Sec. 2.2: the matrix does not fit the GPU) --
 *
 * As ct_build_system, but the dense A~ is assembled on the device a column
 * slab at a time (at most device_budget bytes) and kept in library-owned
 * pinned host memory; the sparse rows stay on the device.  Such a system is
 * factored with ct_qr_factor_ooc (ct_qr_factor refuses it).  The dense
 * values equal the in-core build's bit for bit.  Errors: as ct_build_system;
 * CT_ERR_ARG if device_budget is below one column; CT_ERR_HOSTMEM if the host
 * memory cannot be pinned. */
CT_API ct_status ct_build_system_host(const ct_geometry *geom, ct_precision storage,
                                      size_t device_budget, void *stream, ct_system *out);

/* Blocked Householder QR (Sec. 2 Eq. 2) of a host-resident system with a
 * bounded device working set, the paper's out-of-core setting (Sec. 2.2): left-looking superpanels of W columns (W a multiple of the
 * outer block, as wide as device_budget allows after two staging buffers of
 * one outer block of V each); each superpanel is copied in, updated by every
 * earlier block reflector (V streamed from host memory on a second stream,
 * overlapping the GEMMs), factored in core and copied back.  V and R end in
 * the system's host memory (taken over, as ct_qr_factor takes the device
 * copy); tau, T and the V tops stay on the device, plus a device copy of the
 * n x n triangle R (n * round_up(n,32) elements, not part of the budget) for
 * ct_solve, whose Q^T sweep then streams V from host memory.  The factor
 * works with ct_solve, ct_solve_host, ct_solve_adjoint, ct_factor_export and
 * ct_factor_save; ct_factor_device_ptrs returns CT_ERR_UNSUPPORTED.
 * Disk-backed systems (ct_build_system_disk) go through the same steps with
 * the file in place of host memory (see the disk tier below); their factor
 * is its own checkpoint, so ct_factor_save returns CT_ERR_UNSUPPORTED.
 * Errors: CT_ERR_ARG (no host matrix, budget below 2 staging buffers plus
 * one outer block of columns, disk file partly factored with another
 * precision or panel width), CT_ERR_OOM, CT_ERR_RANK (factor returned),
 * CT_ERR_INTERRUPTED (stop_after reached; no factor), CT_ERR_IO,
 * CT_ERR_TIMEOUT, CT_ERR_CUDA. */
CT_API ct_status ct_qr_factor_ooc(ct_system sys, const ct_opts *opts, size_t device_budget,
                                  void *stream, ct_factor *out);

/* ---- Disk tier (Sec. 2.2: the matrices live in secondary storage, part of
 * the main memory caches their blocks, and disk transfers overlap the GPU's
 * work) ----------------------------------------------------------------------
 *
 * A disk-backed system keeps A~ in one file of column blocks of block_cols
 * columns (rows [0, row_end) of each block only: the rows below are zero in
 * the structured lambda block), with a pinned host cache of
 * host_cache_bytes (at least three blocks) and background I/O threads.
 * ct_qr_factor_ooc factors it left-looking like a host-resident system, with
 * the outer block equal to block_cols; blocks move file -> cache -> device
 * and back, the next blocks are read ahead while the device works, and V
 * and R replace A~ in the file as superpanels finish.  The file records its
 * progress after every superpanel: a factorisation that stops (stop_after,
 * or a process that dies) resumes from the last finished superpanel when
 * ct_qr_factor_ooc is called again on the same or a reopened system (the
 * columns of the superpanel that was being written are rebuilt from the
 * sparse rows first), and a fully factored file yields its factor without
 * recomputation.  The factor takes over the file (ct_factor_free closes it;
 * the file stays on disk, the caller deletes it).  Its solves stream V from
 * the file through the cache; they run without CUDA graphs.
 *
 * Build the system and write A~ to `path` (created or truncated); the sparse
 * rows stay on the device.  block_cols: 0 = 1024 (FP32 storage) or 32 (FP64),
 * otherwise a positive multiple of 32.  The stored values equal the in-core
 * build's bit for bit.  Synchronous (returns when A~ is on disk).
 * Errors: as ct_build_system; CT_ERR_ARG (bad path or block_cols),
 * CT_ERR_HOSTMEM (cache cannot be pinned), CT_ERR_IO. */
CT_API ct_status ct_build_system_disk(const ct_geometry *geom, ct_precision storage,
                                      const char *path, int32_t block_cols,
                                      size_t host_cache_bytes, void *stream, ct_system *out);

/* Reopen a file written by ct_build_system_disk (the matrix in secondary
 * storage, Sec. 2.2) in any state (assembled,
 * partly or fully factored): header checked (magic, version, checksum), the
 * sparse rows rebuilt on the device from the stored geometry.
 * Errors: CT_ERR_ARG (missing or foreign file, checksum mismatch),
 * CT_ERR_HOSTMEM, CT_ERR_OOM, CT_ERR_CUDA. */
CT_API ct_status ct_system_open_disk(const char *path, size_t host_cache_bytes, void *stream,
                                     ct_system *out);

/* Progress of the out-of-core factorisation from disk (Sec. 2.2; the
 * resume records have no counterpart in the paper).  State of a
 * disk-backed system's file: *state 0 = A~ assembled, 1 =
 * factorisation in progress, 2 = factored; *done_cols = columns whose
 * factors are final on disk.  CT_ERR_STATE if the system has no file (or a
 * factor has taken it over). */
CT_API ct_status ct_disk_progress(ct_system sys, int32_t *state, int64_t *done_cols);

/* Process-wide counters of the disk tier (Sec. 2.2: the host cache of
 * blocks read from disk) since the last reset: bytes read and
 * written, cache hits (block resident), prefetched (read already in flight),
 * misses (read on demand), and the summed seconds of the I/O threads' reads
 * and writes.  reset != 0 zeroes them after reading.  Any pointer may be NULL.
 * Always returns CT_OK. */
CT_API ct_status ct_disk_stats(int32_t reset, int64_t *bytes_read, int64_t *bytes_written,
                               int64_t *hits, int64_t *prefetched, int64_t *misses,
                               double *read_s, double *write_s);

/* Host memory of the out-of-core tier (Sec. 2.2).  Pinned host blocks of
 * freed out-of-core systems and factors are kept (at most two) for reuse by
 * the next ct_build_system_host, since pinning tens of GB takes seconds;
 * this unpins and frees them.  Cannot fail (no return value). */
CT_API void ct_host_cache_release(void);

/* Checkpoint of a factorisation: the paper recomputes A = QR only when A
 * changes and reuses it for every sinogram of the same geometry (Sec. 2, text
 * after Eq. 3; Sec. 3.1.2), so a factor can be written to a file and read
 * back in another run.  The file holds the geometry, the precision and block
 * sizes, VR (M' x n), tau, and the per-block T and unit-lower V tops, with an
 * FNV-1a checksum of the payload.  Synchronous (staged through pinned host
 * memory).  Errors: CT_ERR_ARG (bad path), CT_ERR_HOSTMEM, CT_ERR_CUDA. */
CT_API ct_status ct_factor_save(ct_factor f, const char *path);

/* Read a factor written by ct_factor_save into *out (the reuse of A = QR
 * across runs, Sec. 2, text after Eq. 3).  `sys` must have been
 * built with the same geometry and storage precision; its sparse rows serve
 * the refinement, so it must outlive the factor.  Like ct_qr_factor, the
 * factor takes over the system's dense storage (overwritten by V and R); if
 * another factor already holds it, fresh storage is allocated.  On failure
 * the storage is handed back but its content is undefined.
 * Errors: CT_ERR_ARG (missing file, wrong magic/version, checksum mismatch,
 * geometry or precision mismatch), CT_ERR_OOM, CT_ERR_CUDA. */
CT_API ct_status ct_factor_load(ct_system sys, const char *path, void *stream, ct_factor *out);

/* Release a system or a factor and what the library allocated for it
 * (ownership of the library; the paper has no counterpart).  A
 * factor owns the dense storage it took over from its system (V and R); a
 * refining factor reads its system's sparse rows, so free a factor before
 * its system.  Pinned host blocks of out-of-core systems go to the reuse
 * cache (see ct_host_cache_release); a disk-backed file is closed and stays
 * on disk.  NULL is ignored.  Cannot fail (no return value). */
CT_API void ct_system_free(ct_system sys);
CT_API void ct_factor_free(ct_factor f);

/* Failure detection check.  Every device-side spin wait of the library
 * (grid meets of the cooperative panel kernels, mbarrier phases of the
 * tensor-core GEMMs) gives up after 4 s, records DEV_TIMEOUT and the site in
 * the device status word and lets its kernel return, so that a stalled
 * launch surfaces as CT_ERR_TIMEOUT instead of a hang.  This call runs the
 * panel kernels' grid meet on a grid that cannot complete it (one CTA
 * waiting for a second that is never launched) and returns what the next
 * synchronisation point reads: CT_ERR_TIMEOUT after about 4 s, with
 * ct_last_error naming site 90.  The status word is cleared on return and
 * the context stays usable.  The paper has no counterpart.
 * Errors: CT_ERR_TIMEOUT (expected), CT_ERR_CUDA, CT_ERR_OOM. */
CT_API ct_status ct_selftest_wait_timeout(void *stream);

/* Sanitizer substitute (a debugging aid; the paper has no counterpart).
 * enable != 0: every library scratch buffer allocated from now on (GEMM
 * operand copies and split-K partials, workspaces of the factorisation and
 * the solve) gets a 64 KiB guard band past its capacity, filled with the
 * byte 0xA5; enable == 0: buffers allocated later get none.  Buffers that
 * exist already keep their state.  Always returns CT_OK. */
CT_API ct_status ct_debug_canaries(int32_t enable);

/* Waits for the device, then reads the guard band of every live guarded
 * scratch buffer: *checked = buffers read, *corrupted = buffers whose band
 * no longer holds 0xA5 everywhere (a kernel wrote past the end of its
 * scratch).  corrupt_first != 0 first overwrites one byte of the first
 * band (inside that buffer's allocation) so that a test can see the check
 * fire.  The paper has no counterpart.
 * Errors: CT_ERR_ARG (NULL pointer), CT_ERR_CUDA. */
CT_API ct_status ct_debug_check_canaries(int32_t corrupt_first, int64_t *checked, int64_t *corrupted);

/* ---- Benchmark accounting (not part of the method) ---------------------- */

/* Benchmark accounting; the paper has no counterpart.  Zero the launch
 * counter; timing != 0 also brackets every tensor-core GEMM,
 * CUDA-core GEMM, panel, triangular-diagonal, sparse-product and Siddon launch
 * and every out-of-core host copy with CUDA events on its stream, recording
 * its algorithmic flops and bytes
 * (adds a little launch overhead; off by default).  Always returns CT_OK. */
CT_API ct_status ct_stats_reset(int32_t timing);

/* Benchmark accounting; the paper has no counterpart.  Synchronises the
 * device, then returns the number of kernels launched since
 * the last reset and, per class (14 entries each; classes: 0 tensor-core GEMM
 * with TF32 operands, 1 CUDA-core GEMM, 2 panel, 3 triangular diagonal
 * blocks, 4 sparse FP64 products, 5 Siddon, 6 other (split-K reductions),
 * 7 sparse FP32 products, 8 tensor-core GEMM with BF16 operands; out-of-core
 * host traffic: 9 V blocks streamed host to device, 10 superpanel columns
 * host to device, 11 factored columns device to host, 12 the compute
 * stream's waits for a streamed V block; 13 device-side operand
 * conversions, transposes and layout copies), the summed event time in ms,
 * algorithmic flops, algorithmic bytes (bytes copied for classes 9-11 and
 * 13) and launch count (copies for 9-11, waits for 12).  Any pointer may
 * be NULL.  Errors: CT_ERR_CUDA (the synchronisation or an event query failed). */
CT_API ct_status ct_stats_read(int64_t *launches, double *ms, double *flops, double *bytes,
                               int64_t *count);

/* Benchmark accounting; the paper has no counterpart.  Write one CSV line
 * per timed launch since the last ct_stats_reset(1): class, four shape
 * fields (GEMM: M, N, K, splits), ms, flops, bytes.
 * Errors: CT_ERR_ARG (NULL path or a file that cannot be written), CT_ERR_CUDA. */
CT_API ct_status ct_stats_dump(const char *path);

/* ---- Kernel-level entry points (used by the parity tests) --------------- */

/* GEMM engine behind the compact-WY trailing updates and the Q^T and R^-1
 * applications (Sec. 2.1, the BLAS-3 products inside 'dgeqrf', 'dormqr'
 * and 'dtrsm'): C = alpha * op(A) * op(B) + beta * C,
 * column-major, op = 'N' or 'T'.  kind: 0 = FP64 (DFMA), 1 = FP32 (FFMA),
 * 2 = TF32 tensor cores (tcgen05, FP32 accumulate), 3 = BF16 tensor cores,
 * 4 = TF32x3 and 5 = BF16x3 split-precision products on the tensor cores
 * (see ct_precision).  A, B, C are device pointers of double (kind 0) or
 * float (kinds 1-5).
 * Errors: CT_ERR_ARG, CT_ERR_TIMEOUT, CT_ERR_CUDA. */
CT_API ct_status ct_gemm(int32_t kind, char transa, char transb, int64_t M, int64_t N, int64_t K,
                  double alpha, const void *A, int64_t lda, const void *B, int64_t ldb,
                  double beta, void *C, int64_t ldc, void *stream);

/* ct_gemm for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 * ct_gemm keeps split-K partial products and K-major operand copies in
 * scratch the library allocates; a caller whose device memory all belongs to
 * its own pool, or that must not allocate at run time (cudaMalloc can fail
 * under memory pressure and synchronises the device), uses this variant
 * instead: same arguments, same kernels and tile choice, results equal
 * within rounding, and the scratch is one fixed 16 MiB array in the
 * library's static device memory, held by every GPU that loads the library
 * until the process exits.
 * kind: 0 = FP64, 1 = FP32, 2 = TF32 only; kinds 3 (BF16), 4 (TF32x3) and
 * 5 (BF16x3) are refused with CT_ERR_ARG (their operand copies are as large
 * as the operands).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and again after that
 * device's context has been re-created.
 * All calls share the array: calls that overlap on the GPU race.  A product
 * whose K-major operand copies would not fit in the array is refused with
 * CT_ERR_ARG (ct_last_error says how much it needs); the split-K depth of
 * ct_gemm's plan is reduced until the partial products fit.
 * Waits for `stream` before returning (it reads the call's device status).
 * Errors: CT_ERR_ARG, CT_ERR_TIMEOUT, CT_ERR_CUDA. */
CT_API ct_status ct_gemm_noalloc(int32_t kind, char transa, char transb, int64_t M, int64_t N,
                                 int64_t K, double alpha, const void *A, int64_t lda,
                                 const void *B, int64_t ldb, double beta, void *C, int64_t ldc,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CTQR_H */
