// ooc.cu -- out-of-core variant of the system build and the factorisation:
// the dense A~ (and then V and R) lives in pinned host memory and the device
// holds a bounded working set, following the paper's out-of-core QR
// (Sec. 2.2: the matrix does not fit the GPU, tiles move between host and
// device around the factorisation tasks).
//
// Left-looking by superpanels.  Columns are taken W at a time (W a multiple
// of the outer block NB, as wide as the device budget allows).  For each
// superpanel [c0, c1):
//   1. copy its columns (rows that can be nonzero, < row_end(c1)) host -> device;
//   2. apply every earlier outer block J (columns < c0) to it, in order:
//      C <- (I - V_J T_J V_J^T)^T C, with T_J and V_J's top block kept on the
//      device and the rest of V_J streamed from host memory (double-buffered
//      on a copy stream, so the next block's copy overlaps this block's GEMMs);
//   3. factor it in core (panels, inner and trailing updates up to c1);
//   4. copy it back to host memory.
// The factor keeps tau, T_J and the V_J tops on the device, V and R in host
// memory, and a device copy of the n x n triangle R for the triangular
// solves.  Host-link traffic: each superpanel twice, plus, for superpanel s,
// the V of all earlier columns.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "handles.cuh"

namespace ctqr {

ct_status build_system_impl(const ct_geometry *geom, ct_precision storage, void *stream,
                            bool device_dense, ct_system *out);
ct_status rdiag_check(ct_factor f, cudaStream_t s);

namespace {

// One thread per ray row: the row's Siddon segments (CSR, walk order) merge
// into pixel runs as in the in-core fill (FP64 sums in walk order, one
// rounding to the storage type); runs whose pixel lies in [c0, c1) are added
// to the zeroed slab at column pix - c0, so the slab equals those columns of
// the in-core matrix bit for bit.
template <typename T>
__global__ void csr_slab_kernel(int64_t m, const int64_t *row_ptr, const int32_t *col,
                                const double *val, int64_t c0, int64_t c1, T *slab, int64_t lds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int run_pix = -1;
    double run = 0.0;
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
        const int pix = col[q];
        const double L = val[q];
        if (pix == run_pix) {
            run = __dadd_rn(run, L);
        } else {
            if (run_pix >= c0 && run_pix < c1) slab[i + (int64_t)(run_pix - c0) * lds] += (T)run;
            run_pix = pix;
            run = L;
        }
    }
    if (run_pix >= c0 && run_pix < c1) slab[i + (int64_t)(run_pix - c0) * lds] += (T)run;
}

template <typename T>
__global__ void lambda_slab_kernel(int64_t m, int64_t c0, int64_t c1, double sl, T *slab, int64_t lds) {
    const int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < c1) slab[(m + j) + (j - c0) * lds] = (T)sl;
}

// Pinned host blocks of out-of-core matrices are expensive to create (the
// pages are locked one by one: seconds for tens of GB), so freed blocks are
// kept and handed to the next request they fit, largest-fit last.  At most
// kMaxCached blocks are kept; ct_host_cache_release() unpins them.
constexpr int kMaxCached = 2;
std::mutex g_pin_mu;
std::vector<std::pair<void *, size_t>> g_pin_free;

struct Events {
    cudaEvent_t e[6] = {};
    ~Events() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
};

}  // namespace

// Pinned host block of at least `bytes` (from the cache when one fits).
ct_status pinned_acquire(size_t bytes, void **out, size_t *got) {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        int best = -1;
        for (int i = 0; i < (int)g_pin_free.size(); ++i)
            if (g_pin_free[i].second >= bytes && (best < 0 || g_pin_free[i].second < g_pin_free[best].second))
                best = i;
        if (best >= 0) {
            *out = g_pin_free[best].first;
            *got = g_pin_free[best].second;
            g_pin_free.erase(g_pin_free.begin() + best);
            return CT_OK;
        }
    }
    if (cudaMallocHost(out, bytes) != cudaSuccess) {
        cudaGetLastError();
        // release the cache and try once more
        ct_host_cache_release();
        if (cudaMallocHost(out, bytes) != cudaSuccess) {
            cudaGetLastError();
            *out = nullptr;
            return CT_ERR_HOSTMEM;
        }
    }
    *got = bytes;
    return CT_OK;
}

void pinned_release(void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if ((int)g_pin_free.size() >= kMaxCached) {  // drop the smallest
        auto it = std::min_element(g_pin_free.begin(), g_pin_free.end(),
                                   [](auto &a, auto &b) { return a.second < b.second; });
        if (it->second < bytes) {
            cudaFreeHost(it->first);
            g_pin_free.erase(it);
        } else {
            cudaFreeHost(p);
            return;
        }
    }
    g_pin_free.emplace_back(p, bytes);
}

}  // namespace ctqr

using namespace ctqr;

extern "C" void ct_host_cache_release(void) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (auto &b : g_pin_free) cudaFreeHost(b.first);
    g_pin_free.clear();
}

extern "C" ct_status ct_build_system_host(const ct_geometry *geom, ct_precision storage,
                                          size_t device_budget, void *stream, ct_system *out) {
    if (!out) return CT_ERR_ARG;
    *out = nullptr;
    ct_system sys = nullptr;
    CT_TRY(build_system_impl(geom, storage, stream, false, &sys));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = sys->fp64 ? 8 : 4;
    const size_t col_bytes = es * (size_t)sys->lda;
    int64_t ws = (int64_t)std::min<size_t>((size_t)sys->n, device_budget / col_bytes);
    if (ws < 1) {
        set_error("device budget %zu B is below one column (%zu B)", device_budget, col_bytes);
        ct_system_free(sys);
        return CT_ERR_ARG;
    }
    if (pinned_acquire(col_bytes * (size_t)sys->n, &sys->host_dense, &sys->host_bytes) != CT_OK) {
        sys->host_dense = nullptr;
        set_error("cannot pin %zu B of host memory for the dense matrix", col_bytes * (size_t)sys->n);
        ct_system_free(sys);
        return CT_ERR_HOSTMEM;
    }
    void *slab = nullptr;
    if (cudaMalloc(&slab, col_bytes * (size_t)ws) != cudaSuccess) {
        cudaGetLastError();
        ct_system_free(sys);
        return CT_ERR_OOM;
    }
    ct_status st = CT_OK;
    for (int64_t c0 = 0; c0 < sys->n && st == CT_OK; c0 += ws) {
        const int64_t c1 = std::min<int64_t>(sys->n, c0 + ws);
        if (cudaMemsetAsync(slab, 0, col_bytes * (size_t)(c1 - c0), s) != cudaSuccess) { st = CT_ERR_CUDA; break; }
        const unsigned g = (unsigned)ceil_div(std::max<int64_t>(sys->m, 1), 256);
        const unsigned gl = (unsigned)ceil_div(c1 - c0, 256);
        if (sys->fp64) {
            csr_slab_kernel<double><<<g, 256, 0, s>>>(sys->m, sys->row_ptr, sys->col, sys->val, c0, c1,
                                                      (double *)slab, sys->lda);
            if (sys->geom.sqrt_lambda > 0)
                lambda_slab_kernel<double><<<gl, 256, 0, s>>>(sys->m, c0, c1, sys->geom.sqrt_lambda,
                                                              (double *)slab, sys->lda);
        } else {
            csr_slab_kernel<float><<<g, 256, 0, s>>>(sys->m, sys->row_ptr, sys->col, sys->val, c0, c1,
                                                     (float *)slab, sys->lda);
            if (sys->geom.sqrt_lambda > 0)
                lambda_slab_kernel<float><<<gl, 256, 0, s>>>(sys->m, c0, c1, sys->geom.sqrt_lambda,
                                                             (float *)slab, sys->lda);
        }
        count_launch(sys->geom.sqrt_lambda > 0 ? 2 : 1);
        if (cudaGetLastError() != cudaSuccess) { st = CT_ERR_CUDA; break; }
        if (cudaMemcpyAsync((char *)sys->host_dense + col_bytes * (size_t)c0, slab, col_bytes * (size_t)(c1 - c0),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess) { st = CT_ERR_CUDA; break; }
    }
    if (st == CT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = CT_ERR_CUDA;
    cudaFree(slab);
    if (st == CT_OK) st = check_device_status(s);
    if (st != CT_OK) {
        ct_system_free(sys);
        return st;
    }
    *out = sys;
    return CT_OK;
}

extern "C" ct_status ct_qr_factor_ooc(ct_system sys, const ct_opts *opts, size_t device_budget,
                                      void *stream, ct_factor *out) {
    if (!sys || !out) return CT_ERR_ARG;
    *out = nullptr;
    if (!sys->host_dense) {
        set_error("the system has no host-resident dense matrix (build it with ct_build_system_host)");
        return CT_ERR_ARG;
    }
    ct_opts o{};
    o.precision = CT_TF32_REFINE;
    if (opts) o = *opts;
    if (o.precision < CT_FP64 || o.precision > CT_BF16_REFINE) return CT_ERR_ARG;
    if ((o.precision == CT_FP64) != sys->fp64) {
        set_error("factor precision does not match the system's storage");
        return CT_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    ct_factor f = new (std::nothrow) ct_factor_s;
    if (!f) return CT_ERR_HOSTMEM;
    f->sys = sys;
    f->prec = o.precision;
    f->fp64 = o.precision == CT_FP64;
    f->kind = f->fp64 ? GEMM_F64 : (o.precision == CT_FP32 ? GEMM_F32 : GEMM_TF32);
    f->upd_kind = o.precision == CT_BF16_REFINE ? GEMM_BF16 : f->kind;
    f->M = sys->rows;
    f->n = sys->n;
    f->m = sys->m;
    f->lda = sys->lda;
    int nb = o.nb_inner > 0 ? o.nb_inner : (f->fp64 ? 16 : 32);
    nb = std::min(nb, 32);
    int NB = o.nb_outer > 0 ? o.nb_outer : (f->fp64 ? 32 : (f->kind == GEMM_F32 ? 128 : (f->upd_kind == GEMM_BF16 ? 1280 : 1024)));
    NB = (int)round_up(std::max(NB, nb), nb);
    if (NB % 32) NB = (int)round_up(NB, 32);
    f->nb = nb;
    f->NB = NB;
    f->nblocks = ceil_div(f->n, NB);
    f->ooc = true;
    const size_t es = f->es();
    const size_t col_bytes = es * (size_t)f->lda;
    // device budget: two staging buffers for V blocks + the superpanel
    const size_t stage_bytes = es * (size_t)round_up(f->M, 32) * NB;
    int64_t W = 0;
    if (device_budget > 2 * stage_bytes) W = (int64_t)((device_budget - 2 * stage_bytes) / col_bytes) / NB * NB;
    W = std::min<int64_t>(W, round_up(f->n, NB));
    if (W < NB) {
        set_error("device budget %zu B too small: needs 2 x %zu B of staging plus %zu B per %d columns",
                  device_budget, stage_bytes, col_bytes * NB, NB);
        delete f;
        return CT_ERR_ARG;
    }
    f->VR_host = sys->host_dense;  // factored in place, as ct_qr_factor does with the device copy
    f->host_bytes = sys->host_bytes;
    sys->host_dense = nullptr;
    void *sp = nullptr, *stg[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    Events ev;  // ready[0..1], free[0..1], host_ready
    auto fail = [&](ct_status st) {
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        cudaStreamSynchronize(s);
        cudaFree(sp);
        if (stg[1]) cudaFree(stg[1]);
        // the host storage goes back to the system (its content is no longer A~)
        sys->host_dense = f->VR_host;
        sys->host_bytes = f->host_bytes;
        f->VR_host = nullptr;
        f->VR = nullptr;  // the superpanel alias, freed above
        f->stage = stg[0];
        ct_factor_free(f);
        return st;
    };
    if (cudaMalloc(&f->tau, es * (size_t)f->n) != cudaSuccess ||
        cudaMalloc(&f->Tall, es * (size_t)f->nblocks * NB * NB) != cudaSuccess ||
        cudaMalloc(&f->Vtop, es * (size_t)f->nblocks * NB * NB) != cudaSuccess ||
        cudaMalloc(&stg[0], stage_bytes) != cudaSuccess || cudaMalloc(&stg[1], stage_bytes) != cudaSuccess ||
        cudaMalloc(&sp, col_bytes * (size_t)W) != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_OOM);
    }
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(CT_ERR_CUDA);
    for (auto &e : ev.e)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(CT_ERR_CUDA);
    cudaEvent_t *ready = ev.e, *freed = ev.e + 2, host_ready = ev.e[4];
    // both staging buffers start free; no host block is pending
    for (int b = 0; b < 2; ++b)
        if (cudaEventRecord(freed[b], s) != cudaSuccess) return fail(CT_ERR_CUDA);
    if (cudaEventRecord(host_ready, s) != cudaSuccess) return fail(CT_ERR_CUDA);
    ct_status st = CT_OK;
    for (int64_t c0 = 0; c0 < f->n; c0 += W) {
        const int64_t c1 = std::min<int64_t>(f->n, c0 + W);
        const int64_t J0 = c0 / NB, J1 = ceil_div(c1, NB);
        const int64_t rows = f->row_end(c1);  // rows of these columns that can be nonzero
        if (cudaMemcpy2DAsync(sp, col_bytes, (char *)f->VR_host + col_bytes * (size_t)c0, col_bytes,
                              es * (size_t)rows, c1 - c0, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(CT_ERR_CUDA);
        // global column c of the superpanel sits at sp + (c - c0) columns
        f->VR = (char *)sp - col_bytes * (size_t)c0;
        // 2. the earlier outer blocks, V streamed through two staging buffers
        int64_t ldv[2] = {0, 0};
        auto prefetch = [&](int64_t J) -> ct_status {
            const int b = (int)(J & 1);
            CT_CUDA(cudaStreamWaitEvent(cs, freed[b], 0));
            CT_CUDA(cudaStreamWaitEvent(cs, host_ready, 0));
            CT_TRY(stage_v_block(f, J, stg[b], &ldv[b], cs));
            CT_CUDA(cudaEventRecord(ready[b], cs));
            return CT_OK;
        };
        if (J0 > 0 && (st = prefetch(0)) != CT_OK) return fail(st);
        for (int64_t J = 0; J < J0; ++J) {
            const int b = (int)(J & 1);
            if (J + 1 < J0 && (st = prefetch(J + 1)) != CT_OK) return fail(st);
            if (cudaStreamWaitEvent(s, ready[b], 0) != cudaSuccess) return fail(CT_ERR_CUDA);
            const int64_t j = J * NB;
            const int w = (int)std::min<int64_t>(NB, f->n - j);
            const void *VtJ = (char *)f->Vtop + es * (size_t)J * NB * NB;
            const void *TJ = (char *)f->Tall + es * (size_t)J * NB * NB;
            st = apply_block(f, j, w, VtJ, TJ, true, (char *)sp + es * (size_t)j, f->lda, c1 - c0, s,
                             f->upd_kind, stg[b], ldv[b]);
            if (st != CT_OK) return fail(st);
            if (cudaEventRecord(freed[b], s) != cudaSuccess) return fail(CT_ERR_CUDA);
        }
        // 3. this superpanel in core
        if ((st = qr_factor_range(f, J0, J1, c1, s)) != CT_OK) return fail(st);
        // 4. back to host memory
        if (cudaMemcpy2DAsync((char *)f->VR_host + col_bytes * (size_t)c0, col_bytes, sp, col_bytes,
                              es * (size_t)rows, c1 - c0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return fail(CT_ERR_CUDA);
        if (cudaEventRecord(host_ready, s) != cudaSuccess) return fail(CT_ERR_CUDA);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess)
        return fail(CT_ERR_CUDA);
    cudaStreamDestroy(cs);
    cs = nullptr;
    cudaFree(sp);
    sp = nullptr;
    cudaFree(stg[1]);
    stg[1] = nullptr;
    f->stage = stg[0];
    f->stage_bytes = stage_bytes;
    f->VR = nullptr;
    // R (the top n rows) on the device for the triangular solves
    f->ldr = round_up(f->n, 32);
    if (cudaMalloc(&f->Rm, es * (size_t)f->ldr * f->n) != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_OOM);
    }
    if (cudaMemcpy2DAsync(f->Rm, es * f->ldr, f->VR_host, col_bytes, es * (size_t)f->n, f->n,
                          cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(CT_ERR_CUDA);
    st = rdiag_check(f, s);
    if (st != CT_OK && st != CT_ERR_RANK) return fail(st);
    *out = f;
    return st;
}
