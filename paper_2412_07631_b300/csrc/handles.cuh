// handles.cuh -- the objects behind ct_system and ct_factor.
#pragma once

#include <algorithm>

#include "kernels.cuh"

namespace ctqr {
class DiskStore;
}

struct ct_system_s {
    ct_geometry geom{};
    bool fp64 = false;  // dense storage element type
    int64_t m = 0, n = 0, rows = 0, lda = 0, nnz = 0;
    void *dense = nullptr;  // column-major rows x n (NULL once consumed by a factor)
    void *host_dense = nullptr;  // out-of-core systems: the same matrix in pinned host memory
    size_t host_bytes = 0;       // size of that pinned block
    ctqr::DiskStore *store = nullptr;  // disk-backed systems: the file of A~ (owned)
    double *d_cs = nullptr;
    int32_t *row_nnz = nullptr;
    int64_t *row_ptr = nullptr;
    int32_t *col = nullptr;
    double *val = nullptr;
    int64_t *col_ptr = nullptr;
    int32_t *csc_row = nullptr;
    double *csc_val = nullptr;
    float *val32 = nullptr, *csc_val32 = nullptr;  // FP32 copies (inner refinement solves)
    ctqr::Scratch tmp, tmp2;
    ctqr::SparseSys sparse() const {
        return {m, n, nnz, geom.sqrt_lambda, row_ptr, col, val, col_ptr, csc_row, csc_val, val32, csc_val32,
                (int64_t)geom.n_bins, (int64_t)geom.n_side};
    }
};

// A captured CUDA graph for a repeated piece of the solve.  key identifies
// everything the graph bakes in (batch size, buffer addresses, scratch
// generations); a key seen once runs eagerly (sizing every scratch buffer),
// seen again it is captured, then replayed.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    uint64_t key = 0;      // key of exec
    uint64_t warm = 0;     // key of the last eager run
    int64_t kernels = 0;   // kernel launches inside the graph (for accounting)
};

struct ct_factor_s {
    ct_system sys = nullptr;  // borrowed (sparse rows for FP64 refinement)
    ct_precision prec = CT_FP64;
    bool fp64 = true;
    ctqr::GemmKind kind = ctqr::GEMM_F64;      // GEMMs of the solve, Gram and T
    ctqr::GemmKind upd_kind = ctqr::GEMM_F64;  // the two large trailing-update GEMMs of the QR
    int64_t M = 0, n = 0, m = 0, lda = 0;
    void *VR = nullptr;   // owned: R above the diagonal, V below
    void *tau = nullptr;  // owned: n scalars
    int NB = 0, nb = 0;   // outer block / panel widths
    int64_t nblocks = 0;
    void *Tall = nullptr;  // nblocks x (NB x NB), T_J of block J
    void *Vtop = nullptr;  // nblocks x (NB x NB), unit-lower top of V_J
    double rjj_min = 0, rjj_max = 0;
    // R for the triangular solves: VR itself (ld lda) for in-core factors, a
    // device copy of the top n rows (ld ldr) for out-of-core factors
    void *Rm = nullptr;
    int64_t ldr = 0;
    // out-of-core factors: V and R in pinned host memory (VR_host, ld lda,
    // owned); V blocks are streamed through `stage` for the Q^T sweep
    bool ooc = false;
    void *VR_host = nullptr;
    size_t host_bytes = 0;
    ctqr::DiskStore *store = nullptr;  // disk-backed factors: V and R in the file (owned)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // triangular-solve aids (built on first solve): inverse diagonal blocks of R
    // and their transposes (trsm_tb x trsm_tb each), R^T for the tensor-core path
    void *Rinv = nullptr, *RinvT = nullptr, *Rt = nullptr;
    int trsm_tb = 0;
    // tensor-core path: inverses of the trsm_sb x trsm_sb diagonal superblocks
    // (and their transposes), so each superblock is one GEMM
    void *RinvB = nullptr, *RinvTB = nullptr;
    int trsm_sb = 0;
    // solve plan (ct_opts.solve_block / solve_split of the latest solve call):
    // requested superblock rows (0: default) and least split-K depth of the
    // solve's GEMMs (0: the engine's default)
    int solve_sb_req = 0;
    int64_t solve_chunk = 0;
    int64_t ldrt = 0;
    // captured graphs of the solve, and the stream they run on
    GraphSlot g_direct, g_iter;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double *pinned = nullptr;  // host readback of per-slice scalars (pinned)
    size_t pinned_count = 0;
    bool graphs_enabled = true;
    bool gram_panel = true;  // FP32 panels from Gram matrices (else column by column)
    // work buffers
    ctqr::Scratch gemm_ws, W, W2, G, panel_ws, Bt, trsm_ws, refine_ws, host_pinned, misc, misc2;
    ctqr::Scratch V16;  // BF16 copies of a block reflector's V in both K-major layouts
    ctqr::Scratch W2h;  // BF16 copy of a narrow reflector's W2 (K-major), from the top-block kernel
    size_t es() const { return fp64 ? 8 : 4; }
    // One past the last row the reflectors of columns [0, col_end) can touch.
    // Below the ray rows, A~ holds sqrt(lambda) I: row m+i is untouched until
    // column i is reached, so reflectors up to column col_end-1 live in rows
    // [.., m + col_end) and every row beyond keeps its initial content.
    int64_t row_end(int64_t col_end) const { return M > m ? std::min(M, m + col_end) : M; }
};

namespace ctqr {
// Run body(stream) on `caller`, eagerly or through the captured graph of slot
// `g` (see GraphSlot).  body must not synchronise or read device data.
template <class Body>
ct_status run_graphed(ct_factor f, GraphSlot &g, uint64_t key, cudaStream_t caller, Body body);
uint64_t graph_key(ct_factor f, int64_t k, const void *extra);
// pinned host blocks of out-of-core matrices (cached across free/alloc)
ct_status pinned_acquire(size_t bytes, void **out, size_t *got);
void pinned_release(void *p, size_t bytes);
bool graphs_allowed(ct_factor f);
ct_status qr_factor_run(ct_factor f, cudaStream_t s);
ct_status qr_factor_range(ct_factor f, int64_t J0, int64_t J1, int64_t col_end, cudaStream_t s);
// C <- (I - V op(T) V^T) C for the block at column j (see qr.cu); vb/ldvb:
// V below the top block from a staging buffer instead of VR (nullptr: VR).
// v16r (BF16 updates of narrow blocks, w <= 32): the BF16 rounding of V below
// its top block, row-major with ld round_up(w, 64), already made by the
// panel kernel (nullptr: rounded here).
ct_status apply_block(ct_factor f, int64_t j, int w, const void *Vt, const void *T, bool qt, void *C,
                      int64_t ldc, int64_t ncols, cudaStream_t s, ctqr::GemmKind big, const void *vb,
                      int64_t ldvb, const void *v16r_made = nullptr);
ct_status stage_v_block(ct_factor f, int64_t J, void *dst, int64_t *ldd, cudaStream_t s);
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

// ---- graph slot implementation (header-only template) ----------------------
namespace ctqr {
int64_t launch_count();
bool timing_enabled();

template <class Body>
ct_status run_graphed(ct_factor f, GraphSlot &g, uint64_t key, cudaStream_t caller, Body body) {
    if (!graphs_allowed(f)) return body(caller);
    if (!f->side) {
        CT_CUDA(cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking));
        CT_CUDA(cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming));
        CT_CUDA(cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming));
    }
    if (!(g.exec && g.key == key)) {
        if (g.warm != key) {  // first sight of this key: eager run sizes every buffer
            g.warm = key;
            return body(caller);
        }
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        const int64_t before = launch_count();
        CT_CUDA(cudaStreamBeginCapture(f->side, cudaStreamCaptureModeThreadLocal));
        ct_status st = body(f->side);
        cudaError_t e = cudaStreamEndCapture(f->side, &graph);
        const int64_t kernels = launch_count() - before;
        count_launch((int)-kernels);  // nothing ran during capture
        if (st != CT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_status(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        g.key = key;
        g.kernels = kernels;
    }
    CT_CUDA(cudaEventRecord(f->ev_fork, caller));
    CT_CUDA(cudaStreamWaitEvent(f->side, f->ev_fork, 0));
    CT_CUDA(cudaGraphLaunch(g.exec, f->side));
    count_launch((int)g.kernels);
    CT_CUDA(cudaEventRecord(f->ev_join, f->side));
    CT_CUDA(cudaStreamWaitEvent(caller, f->ev_join, 0));
    return CT_OK;
}
}  // namespace ctqr
