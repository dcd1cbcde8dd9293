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
// solves (collected from each superpanel while it is on the device).
// Host-link traffic: each superpanel twice, plus, for superpanel s, the V of
// all earlier columns.
//
// Disk tier: the same steps with a file (DiskStore: column blocks of NB
// columns, a pinned block cache, background I/O threads) in place of host
// memory.  Blocks are read ahead while the device works; the write-back of
// superpanel s is made durable while superpanel s+1 is factored.  Before a
// superpanel's write-back the file's header records [done, dirty) = the
// finished columns and the columns about to be rewritten, so a run that
// stops anywhere resumes at `done` after rebuilding [done, dirty) from the
// sparse rows (left-looking: every column past `done` is then A~ again).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "diskstore.cuh"
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

namespace ctqr {
namespace {

// Columns [c0, c1) of A~ into the zeroed device slab (leading dimension lds,
// which must cover every row these columns can touch: lds >= row_end(c1)).
void assemble_slab(ct_system sys, int64_t c0, int64_t c1, void *slab, int64_t lds, cudaStream_t s) {
    const unsigned g = (unsigned)ceil_div(std::max<int64_t>(sys->m, 1), 256);
    const unsigned gl = (unsigned)ceil_div(c1 - c0, 256);
    if (sys->fp64) {
        csr_slab_kernel<double><<<g, 256, 0, s>>>(sys->m, sys->row_ptr, sys->col, sys->val, c0, c1,
                                                  (double *)slab, lds);
        if (sys->geom.sqrt_lambda > 0)
            lambda_slab_kernel<double><<<gl, 256, 0, s>>>(sys->m, c0, c1, sys->geom.sqrt_lambda,
                                                          (double *)slab, lds);
    } else {
        csr_slab_kernel<float><<<g, 256, 0, s>>>(sys->m, sys->row_ptr, sys->col, sys->val, c0, c1,
                                                 (float *)slab, lds);
        if (sys->geom.sqrt_lambda > 0)
            lambda_slab_kernel<float><<<gl, 256, 0, s>>>(sys->m, c0, c1, sys->geom.sqrt_lambda,
                                                         (float *)slab, lds);
    }
    count_launch(sys->geom.sqrt_lambda > 0 ? 2 : 1);
}

// Blocks [b0, b1) of the file rebuilt from the sparse rows (the disk build,
// and the repair of a write-back that an interrupted run left half done).
ct_status assemble_blocks(ct_system sys, DiskStore *d, int64_t b0, int64_t b1, cudaStream_t s) {
    if (b0 >= b1) return CT_OK;
    const size_t es = sys->fp64 ? 8 : 4;
    size_t slab_bytes = 0;
    for (int64_t b = b0; b < b1; ++b) slab_bytes = std::max(slab_bytes, es * d->block_rows(b) * d->block_w(b));
    void *slab = nullptr;
    if (cudaMalloc(&slab, slab_bytes) != cudaSuccess) {
        cudaGetLastError();
        return CT_ERR_OOM;
    }
    ct_status st = CT_OK;
    for (int64_t b = b0; b < b1 && st == CT_OK; ++b) {
        const int64_t rb = d->block_rows(b), w = d->block_w(b), c0 = d->block_c0(b);
        if (cudaMemsetAsync(slab, 0, es * rb * w, s) != cudaSuccess) { st = CT_ERR_CUDA; break; }
        assemble_slab(sys, c0, c0 + w, slab, rb, s);
        if (cudaGetLastError() != cudaSuccess) { st = CT_ERR_CUDA; break; }
        int slot = -1;
        if ((st = d->acquire_write(b, s, &slot)) != CT_OK) break;
        if (cudaMemcpyAsync(d->slot_ptr(slot), slab, es * rb * w, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = CT_ERR_CUDA;
        const ct_status st2 = d->commit(slot, s);
        if (st == CT_OK) st = st2;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && st == CT_OK) st = CT_ERR_CUDA;
    cudaFree(slab);
    if (st == CT_OK) st = check_device_status(s);
    if (st == CT_OK) st = d->flush();
    return st;
}

// Page-aligned host buffer (direct I/O of the per-block records).
struct HostBuf {
    void *p = nullptr;
    explicit HostBuf(size_t n) {
        if (posix_memalign(&p, 4096, std::max<size_t>(n, 4096)) != 0) p = nullptr;
        if (p) memset(p, 0, std::max<size_t>(n, 4096));
    }
    ~HostBuf() { free(p); }
};

// tau, T_J and the V_J top of blocks [J0, J1) from the device to the file.
ct_status write_block_records(ct_factor f, int64_t J0, int64_t J1, cudaStream_t s) {
    DiskStore *d = f->store;
    const size_t es = f->es(), stride = d->aux_stride(), NB = f->NB;
    HostBuf h(stride * (size_t)(J1 - J0));
    if (!h.p) return CT_ERR_HOSTMEM;
    for (int64_t J = J0; J < J1; ++J) {
        char *rec = (char *)h.p + stride * (size_t)(J - J0);
        const int64_t w = std::min<int64_t>(NB, f->n - J * NB);
        CT_CUDA(cudaMemcpyAsync(rec, (char *)f->tau + es * J * NB, es * w, cudaMemcpyDeviceToHost, s));
        CT_CUDA(cudaMemcpyAsync(rec + es * NB, (char *)f->Tall + es * J * NB * NB, es * NB * NB,
                                cudaMemcpyDeviceToHost, s));
        CT_CUDA(cudaMemcpyAsync(rec + es * (NB + NB * NB), (char *)f->Vtop + es * J * NB * NB, es * NB * NB,
                                cudaMemcpyDeviceToHost, s));
    }
    CT_CUDA(cudaStreamSynchronize(s));
    return d->write_aux(J0, J1, h.p);
}

// The records of blocks [J0, J1) from the file to the device (resume).
ct_status read_block_records(ct_factor f, int64_t J0, int64_t J1, cudaStream_t s) {
    if (J0 >= J1) return CT_OK;
    DiskStore *d = f->store;
    const size_t es = f->es(), stride = d->aux_stride(), NB = f->NB;
    HostBuf h(stride * (size_t)(J1 - J0));
    if (!h.p) return CT_ERR_HOSTMEM;
    CT_TRY(d->read_aux(J0, J1, h.p));
    for (int64_t J = J0; J < J1; ++J) {
        const char *rec = (const char *)h.p + stride * (size_t)(J - J0);
        const int64_t w = std::min<int64_t>(NB, f->n - J * NB);
        CT_CUDA(cudaMemcpyAsync((char *)f->tau + es * J * NB, rec, es * w, cudaMemcpyHostToDevice, s));
        CT_CUDA(cudaMemcpyAsync((char *)f->Tall + es * J * NB * NB, rec + es * NB, es * NB * NB,
                                cudaMemcpyHostToDevice, s));
        CT_CUDA(cudaMemcpyAsync((char *)f->Vtop + es * J * NB * NB, rec + es * (NB + NB * NB), es * NB * NB,
                                cudaMemcpyHostToDevice, s));
    }
    CT_CUDA(cudaStreamSynchronize(s));  // the host buffer goes away
    return CT_OK;
}

// Columns [c0, c1) (rows [0, rows)) from the host copy or the file into the
// device superpanel sp (leading dimension lda).  File blocks hold only their
// own rows; the rows below, up to `rows`, are zero.
ct_status load_cols(ct_factor f, int64_t c0, int64_t c1, int64_t rows, void *sp, cudaStream_t s) {
    const size_t es = f->es();
    const size_t col_bytes = es * (size_t)f->lda;
    DiskStore *d = f->store;
    ProfScope prof(PROF_H2D_COLS, s, 0.0, (double)es * rows * (c1 - c0));
    if (!d) {
        CT_CUDA(cudaMemcpy2DAsync(sp, col_bytes, (char *)f->VR_host + col_bytes * (size_t)c0, col_bytes,
                                  es * (size_t)rows, c1 - c0, cudaMemcpyHostToDevice, s));
        return CT_OK;
    }
    const int64_t b0 = c0 / f->NB, b1 = ceil_div(c1, f->NB);
    const int ahead = std::max(1, d->nslots() / 2 - 1);
    for (int64_t b = b0; b < std::min<int64_t>(b1, b0 + ahead); ++b) d->prefetch(b);
    for (int64_t b = b0; b < b1; ++b) {
        if (b + ahead < b1) d->prefetch(b + ahead);
        int slot = -1;
        CT_TRY(d->acquire(b, s, &slot));
        const int64_t rb = d->block_rows(b), w = d->block_w(b);
        char *dst = (char *)sp + col_bytes * (size_t)(d->block_c0(b) - c0);
        const cudaError_t e = cudaMemcpy2DAsync(dst, col_bytes, d->slot_ptr(slot), es * rb, es * rb, w,
                                                cudaMemcpyHostToDevice, s);
        CT_TRY(d->release(slot, s));
        CT_CUDA(e);
        if (rows > rb) CT_CUDA(cudaMemset2DAsync(dst + es * rb, col_bytes, 0, es * (rows - rb), w, s));
    }
    return CT_OK;
}

// The factored superpanel back to the host copy or the file.
ct_status store_cols(ct_factor f, int64_t c0, int64_t c1, int64_t rows, const void *sp, cudaStream_t s) {
    const size_t es = f->es();
    const size_t col_bytes = es * (size_t)f->lda;
    DiskStore *d = f->store;
    ProfScope prof(PROF_D2H_COLS, s, 0.0, (double)es * rows * (c1 - c0));
    if (!d) {
        CT_CUDA(cudaMemcpy2DAsync((char *)f->VR_host + col_bytes * (size_t)c0, col_bytes, sp, col_bytes,
                                  es * (size_t)rows, c1 - c0, cudaMemcpyDeviceToHost, s));
        return CT_OK;
    }
    for (int64_t b = c0 / f->NB; b < ceil_div(c1, f->NB); ++b) {
        int slot = -1;
        CT_TRY(d->acquire_write(b, s, &slot));
        const int64_t rb = d->block_rows(b), w = d->block_w(b);
        const cudaError_t e = cudaMemcpy2DAsync(d->slot_ptr(slot), es * rb,
                                                (const char *)sp + col_bytes * (size_t)(d->block_c0(b) - c0),
                                                col_bytes, es * rb, w, cudaMemcpyDeviceToHost, s);
        CT_TRY(d->commit(slot, s));
        CT_CUDA(e);
    }
    return CT_OK;
}

// R's columns [c0, c1) (rows above the diagonal block's end) from the file
// into the device copy Rm (a resumed factorisation's finished columns).
ct_status load_r_cols(ct_factor f, int64_t c0, int64_t c1, cudaStream_t s) {
    DiskStore *d = f->store;
    const size_t es = f->es();
    const int ahead = std::max(1, d->nslots() / 2 - 1);
    const int64_t b0 = c0 / f->NB, b1 = ceil_div(c1, f->NB);
    for (int64_t b = b0; b < std::min<int64_t>(b1, b0 + ahead); ++b) d->prefetch(b);
    for (int64_t b = b0; b < b1; ++b) {
        if (b + ahead < b1) d->prefetch(b + ahead);
        int slot = -1;
        CT_TRY(d->acquire(b, s, &slot));
        const int64_t rb = d->block_rows(b), w = d->block_w(b), cb = d->block_c0(b);
        const int64_t r = std::min<int64_t>({f->n, rb, cb + w});
        const cudaError_t e = cudaMemcpy2DAsync((char *)f->Rm + es * (size_t)cb * f->ldr, es * f->ldr,
                                                d->slot_ptr(slot), es * rb, es * r, w,
                                                cudaMemcpyHostToDevice, s);
        CT_TRY(d->release(slot, s));
        CT_CUDA(e);
    }
    return CT_OK;
}

}  // namespace
}  // namespace ctqr

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
        assemble_slab(sys, c0, c1, slab, sys->lda, s);
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

extern "C" ct_status ct_build_system_disk(const ct_geometry *geom, ct_precision storage, const char *path,
                                          int32_t block_cols, size_t host_cache_bytes, void *stream,
                                          ct_system *out) {
    if (!out || !path || !*path) return CT_ERR_ARG;
    *out = nullptr;
    if (block_cols < 0 || block_cols % 32) {
        set_error("block_cols must be 0 or a positive multiple of 32 (got %d)", block_cols);
        return CT_ERR_ARG;
    }
    ct_system sys = nullptr;
    CT_TRY(build_system_impl(geom, storage, stream, false, &sys));
    const int bw = block_cols > 0 ? block_cols : (sys->fp64 ? 32 : 1024);
    DiskStore *d = nullptr;
    ct_status st = DiskStore::create(path, sys->geom, sys->fp64, sys->m, sys->n, sys->rows, sys->lda, bw,
                                     host_cache_bytes, &d);
    if (st == CT_OK) st = assemble_blocks(sys, d, 0, d->nblocks(), (cudaStream_t)stream);
    if (st != CT_OK) {
        delete d;
        ct_system_free(sys);
        return st;
    }
    sys->store = d;
    *out = sys;
    return CT_OK;
}

extern "C" ct_status ct_system_open_disk(const char *path, size_t host_cache_bytes, void *stream,
                                         ct_system *out) {
    if (!out || !path) return CT_ERR_ARG;
    *out = nullptr;
    DiskStore *d = nullptr;
    CT_TRY(DiskStore::open(path, host_cache_bytes, &d));
    const DiskHeader &h = d->header();
    ct_system sys = nullptr;
    ct_status st = build_system_impl(&h.geom, h.es == 8 ? CT_FP64 : CT_FP32, stream, false, &sys);
    if (st == CT_OK && (sys->m != h.m || sys->n != h.n || sys->rows != h.rows || sys->lda != h.lda)) {
        set_error("'%s' does not match the system its geometry builds", path);
        st = CT_ERR_ARG;
    }
    if (st != CT_OK) {
        delete d;
        ct_system_free(sys);
        return st;
    }
    sys->store = d;
    *out = sys;
    return CT_OK;
}

extern "C" ct_status ct_disk_progress(ct_system sys, int32_t *state, int64_t *done_cols) {
    if (!sys) return CT_ERR_ARG;
    if (!sys->store) return CT_ERR_STATE;
    if (state) *state = sys->store->header().state;
    if (done_cols) *done_cols = sys->store->header().done_cols;
    return CT_OK;
}

extern "C" ct_status ct_qr_factor_ooc(ct_system sys, const ct_opts *opts, size_t device_budget,
                                      void *stream, ct_factor *out) {
    if (!sys || !out) return CT_ERR_ARG;
    *out = nullptr;
    DiskStore *d = sys->store;
    if (!sys->host_dense && !d) {
        set_error("the system has no host-resident or disk-resident dense matrix "
                  "(build it with ct_build_system_host or ct_build_system_disk)");
        return CT_ERR_ARG;
    }
    ct_opts o{};
    o.precision = CT_TF32_REFINE;
    if (opts) o = *opts;
    if (o.precision < CT_FP64 || o.precision > CT_BF16X3_REFINE || o.stop_after < 0) return CT_ERR_ARG;
    if ((o.precision == CT_FP64) != sys->fp64) {
        set_error("factor precision does not match the system's storage");
        return CT_ERR_ARG;
    }
    int nb = o.nb_inner > 0 ? o.nb_inner : (sys->fp64 ? 16 : 32);
    nb = std::min(nb, 32);
    if (d) {
        const DiskHeader &h = d->header();
        if (o.nb_outer > 0 && o.nb_outer != h.bw) {
            set_error("the file's blocks are %d columns wide; the outer block must match (got %d)", h.bw,
                      o.nb_outer);
            return CT_ERR_ARG;
        }
        if (h.state != DISK_ASSEMBLED) {
            if (h.prec != (int32_t)o.precision || (o.nb_inner > 0 && std::min(o.nb_inner, 32) != h.nb_inner)) {
                set_error("'%s' holds a factorisation in precision %d, panels of %d: resume it with those",
                          "the file", h.prec, h.nb_inner);
                return CT_ERR_ARG;
            }
            nb = h.nb_inner;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    ct_factor f = new (std::nothrow) ct_factor_s;
    if (!f) return CT_ERR_HOSTMEM;
    f->sys = sys;
    f->prec = o.precision;
    f->fp64 = o.precision == CT_FP64;
    f->kind = solve_kind(o.precision);
    f->upd_kind = update_kind(o.precision);
    f->gram_panel = !(o.flags & CT_OPT_COLUMN_PANEL);
    f->M = sys->rows;
    f->n = sys->n;
    f->m = sys->m;
    f->lda = sys->lda;
    int NB = o.nb_outer > 0 ? o.nb_outer : (f->fp64 ? 32 : (f->kind == GEMM_F32 ? 128 : (f->upd_kind == GEMM_BF16 ? 2048 : 1536)));
    if (d) NB = d->bw();
    NB = (int)round_up(std::max(NB, nb), nb);
    if (NB % 32) NB = (int)round_up(NB, 32);
    if (d && NB != d->bw()) {
        set_error("panel width %d does not divide the file's %d-column blocks", nb, d->bw());
        delete f;
        return CT_ERR_ARG;
    }
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
    // the factor takes over the host storage or the file
    if (d) {
        f->store = d;
        sys->store = nullptr;
    } else {
        f->VR_host = sys->host_dense;  // factored in place, as ct_qr_factor does with the device copy
        f->host_bytes = sys->host_bytes;
        sys->host_dense = nullptr;
    }
    void *sp = nullptr, *stg[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    Events ev;  // ready[0..1], free[0..1], host_ready
    // Host tier: a superpanel's write-back (device to host) and the next
    // superpanel's load (host to device) run in kPipe column chunks on two
    // copy streams, each load chunk after the store of the same part of the
    // device buffer, so the two directions of the link overlap.
    constexpr int kPipe = 4;
    const bool piped = d == nullptr;
    cudaStream_t ss = nullptr, ls = nullptr;  // store stream, load stream
    cudaEvent_t stored[kPipe] = {}, loaded = nullptr, computed = nullptr;
    auto fail = [&](ct_status st) {
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        for (cudaStream_t x : {ss, ls})
            if (x) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
        for (cudaEvent_t x : stored)
            if (x) cudaEventDestroy(x);
        if (loaded) cudaEventDestroy(loaded);
        if (computed) cudaEventDestroy(computed);
        cudaStreamSynchronize(s);
        cudaFree(sp);
        if (stg[1]) cudaFree(stg[1]);
        // the storage goes back to the system (host memory: its content is no
        // longer A~; the file: resumable from its recorded progress)
        sys->host_dense = f->VR_host;
        sys->host_bytes = f->host_bytes;
        sys->store = f->store;
        f->VR_host = nullptr;
        f->store = nullptr;
        f->VR = nullptr;  // the superpanel alias, freed above
        f->stage = stg[0];
        ct_factor_free(f);
        return st;
    };
    f->ldr = round_up(f->n, 32);
    if (cudaMalloc(&f->tau, es * (size_t)f->n) != cudaSuccess ||
        cudaMalloc(&f->Tall, es * (size_t)f->nblocks * NB * NB) != cudaSuccess ||
        cudaMalloc(&f->Vtop, es * (size_t)f->nblocks * NB * NB) != cudaSuccess ||
        cudaMalloc(&f->Rm, es * (size_t)f->ldr * f->n) != cudaSuccess ||
        cudaMalloc(&stg[0], stage_bytes) != cudaSuccess || cudaMalloc(&stg[1], stage_bytes) != cudaSuccess ||
        cudaMalloc(&sp, col_bytes * (size_t)W) != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_OOM);
    }
    // R (the top n rows, upper triangle) is collected on the device as
    // superpanels finish; the rest of Rm is never read but kept finite
    if (cudaMemsetAsync(f->Rm, 0, es * (size_t)f->ldr * f->n, s) != cudaSuccess) return fail(CT_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(CT_ERR_CUDA);
    for (auto &e : ev.e)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(CT_ERR_CUDA);
    if (piped) {
        if (cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&loaded, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&computed, cudaEventDisableTiming) != cudaSuccess)
            return fail(CT_ERR_CUDA);
        for (auto &e : stored)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(CT_ERR_CUDA);
    }
    const int64_t chunk = ceil_div(W, kPipe);  // columns per pipelined copy
    int prev_chunks = 0;                       // store chunks of the previous superpanel in flight
    cudaEvent_t *ready = ev.e, *freed = ev.e + 2, host_ready = ev.e[4];
    // both staging buffers start free; no host block is pending
    for (int b = 0; b < 2; ++b)
        if (cudaEventRecord(freed[b], s) != cudaSuccess) return fail(CT_ERR_CUDA);
    if (cudaEventRecord(host_ready, s) != cudaSuccess) return fail(CT_ERR_CUDA);
    ct_status st = CT_OK;
    int64_t start = 0;
    if (d) {  // resume where the file's recorded progress ends
        const DiskHeader h = d->header();
        if (h.state == DISK_ASSEMBLED) {
            if ((st = d->set_progress(DISK_FACTORING, 0, 0, (int32_t)o.precision, nb, 0, 0)) != CT_OK)
                return fail(st);
        } else {
            start = h.done_cols;
            // columns of a write-back the last run may have left half done: rebuilt as A~
            if (h.dirty_cols > start &&
                (st = assemble_blocks(sys, d, start / NB, ceil_div(h.dirty_cols, NB), s)) != CT_OK)
                return fail(st);
            if ((st = read_block_records(f, 0, ceil_div(start, NB), s)) != CT_OK) return fail(st);
            if (start > 0 && (st = load_r_cols(f, 0, start, s)) != CT_OK) return fail(st);
        }
    }
    int done_panels = 0;
    for (int64_t c0 = start; c0 < f->n; c0 += W) {
        const int64_t c1 = std::min<int64_t>(f->n, c0 + W);
        const int64_t J0 = c0 / NB, J1 = ceil_div(c1, NB);
        const int64_t rows = f->row_end(c1);  // rows of these columns that can be nonzero
        // 1. the superpanel's columns
        if (piped) {
            int q = 0;
            for (int64_t a = c0; a < c1; a += chunk, ++q) {
                const int64_t b = std::min(c1, a + chunk);
                // the same part of the buffer held the previous superpanel's chunk q
                if (q < prev_chunks && cudaStreamWaitEvent(ls, stored[q], 0) != cudaSuccess)
                    return fail(CT_ERR_CUDA);
                ProfScope prof(PROF_H2D_COLS, ls, 0.0, (double)es * rows * (b - a));
                if (cudaMemcpy2DAsync((char *)sp + col_bytes * (size_t)(a - c0), col_bytes,
                                      (char *)f->VR_host + col_bytes * (size_t)a, col_bytes, es * (size_t)rows,
                                      b - a, cudaMemcpyHostToDevice, ls) != cudaSuccess)
                    return fail(CT_ERR_CUDA);
            }
            if (cudaEventRecord(loaded, ls) != cudaSuccess || cudaStreamWaitEvent(s, loaded, 0) != cudaSuccess)
                return fail(CT_ERR_CUDA);
        } else if ((st = load_cols(f, c0, c1, rows, sp, s)) != CT_OK) {
            return fail(st);
        }
        // global column c of the superpanel sits at sp + (c - c0) columns
        f->VR = (char *)sp - col_bytes * (size_t)c0;
        // 2. the earlier outer blocks, V streamed through two staging buffers
        int64_t ldv[2] = {0, 0};
        const int ahead = d ? std::max(1, d->nslots() / 2 - 1) : 0;
        auto prefetch = [&](int64_t J) -> ct_status {
            const int b = (int)(J & 1);
            for (int64_t q = J + 1; d && q <= std::min<int64_t>(J + ahead, J0 - 1); ++q) d->prefetch(q);
            CT_CUDA(cudaStreamWaitEvent(cs, freed[b], 0));
            CT_CUDA(cudaStreamWaitEvent(cs, host_ready, 0));
            CT_TRY(stage_v_block(f, J, stg[b], &ldv[b], cs));
            CT_CUDA(cudaEventRecord(ready[b], cs));
            return CT_OK;
        };
        if (J0 > 0 && (st = prefetch(0)) != CT_OK) return fail(st);
        for (int64_t J = 0; J < J0; ++J) {
            const int b = (int)(J & 1);
            {
                // timed (when accounting is on) from before to after the wait:
                // the stall of the compute stream on this block's copy
                ProfScope stall(PROF_COPY_WAIT, s, 0.0, 0.0);
                if (cudaStreamWaitEvent(s, ready[b], 0) != cudaSuccess) return fail(CT_ERR_CUDA);
            }
            const int64_t j = J * NB;
            const int w = (int)std::min<int64_t>(NB, f->n - j);
            const void *VtJ = (char *)f->Vtop + es * (size_t)J * NB * NB;
            const void *TJ = (char *)f->Tall + es * (size_t)J * NB * NB;
            st = apply_block(f, j, w, VtJ, TJ, true, (char *)sp + es * (size_t)j, f->lda, c1 - c0, s,
                             f->upd_kind, stg[b], ldv[b]);
            if (st != CT_OK) return fail(st);
            if (cudaEventRecord(freed[b], s) != cudaSuccess) return fail(CT_ERR_CUDA);
            // the next block's copy (the file read may block this thread while
            // the device works on block J)
            if (J + 1 < J0 && (st = prefetch(J + 1)) != CT_OK) return fail(st);
        }
        // 3. this superpanel in core; its R part into the device copy
        if ((st = qr_factor_range(f, J0, J1, c1, s)) != CT_OK) return fail(st);
        if (cudaMemcpy2DAsync((char *)f->Rm + es * (size_t)c0 * f->ldr, es * f->ldr, sp, col_bytes,
                              es * (size_t)std::min<int64_t>(f->n, c1), c1 - c0, cudaMemcpyDeviceToDevice,
                              s) != cudaSuccess)
            return fail(CT_ERR_CUDA);
        // 4. back to host memory / the file.  For the file: the previous
        // superpanel's writes are made durable and recorded first (while the
        // device factors this one), then these columns are marked as being
        // rewritten, then written back.
        if (d) {
            if ((st = d->flush()) != CT_OK ||
                (st = d->set_progress(DISK_FACTORING, c0, c1, (int32_t)o.precision, nb, 0, 0)) != CT_OK)
                return fail(st);
        }
        if (piped) {
            // write-back on the store stream once this superpanel's work is done
            if (cudaEventRecord(computed, s) != cudaSuccess || cudaStreamWaitEvent(ss, computed, 0) != cudaSuccess)
                return fail(CT_ERR_CUDA);
            int q = 0;
            for (int64_t a = c0; a < c1; a += chunk, ++q) {
                const int64_t b = std::min(c1, a + chunk);
                {
                    ProfScope prof(PROF_D2H_COLS, ss, 0.0, (double)es * rows * (b - a));
                    if (cudaMemcpy2DAsync((char *)f->VR_host + col_bytes * (size_t)a, col_bytes,
                                          (char *)sp + col_bytes * (size_t)(a - c0), col_bytes,
                                          es * (size_t)rows, b - a, cudaMemcpyDeviceToHost, ss) != cudaSuccess)
                        return fail(CT_ERR_CUDA);
                }
                if (cudaEventRecord(stored[q], ss) != cudaSuccess) return fail(CT_ERR_CUDA);
            }
            prev_chunks = q;
            // the next superpanel streams these V blocks back from host memory
            if (cudaEventRecord(host_ready, ss) != cudaSuccess) return fail(CT_ERR_CUDA);
        } else {
            if ((st = store_cols(f, c0, c1, rows, sp, s)) != CT_OK) return fail(st);
            if (d && (st = write_block_records(f, J0, J1, s)) != CT_OK) return fail(st);
            if (cudaEventRecord(host_ready, s) != cudaSuccess) return fail(CT_ERR_CUDA);
        }
        if (d && o.stop_after > 0 && ++done_panels >= o.stop_after && c1 < f->n) {
            if ((st = d->flush()) != CT_OK ||
                (st = d->set_progress(DISK_FACTORING, c1, c1, (int32_t)o.precision, nb, 0, 0)) != CT_OK)
                return fail(st);
            set_error("stopped after %d superpanel(s) at column %lld of %lld", done_panels, (long long)c1,
                      (long long)f->n);
            return fail(CT_ERR_INTERRUPTED);
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess ||
        (ss && cudaStreamSynchronize(ss) != cudaSuccess) || (ls && cudaStreamSynchronize(ls) != cudaSuccess))
        return fail(CT_ERR_CUDA);
    cudaStreamDestroy(cs);
    cs = nullptr;
    for (cudaStream_t *x : {&ss, &ls})
        if (*x) {
            cudaStreamDestroy(*x);
            *x = nullptr;
        }
    for (auto &x : stored)
        if (x) {
            cudaEventDestroy(x);
            x = nullptr;
        }
    if (loaded) cudaEventDestroy(loaded);
    if (computed) cudaEventDestroy(computed);
    loaded = computed = nullptr;
    cudaFree(sp);
    sp = nullptr;
    cudaFree(stg[1]);
    stg[1] = nullptr;
    f->stage = stg[0];
    f->stage_bytes = stage_bytes;
    f->VR = nullptr;
    st = rdiag_check(f, s);
    if (st != CT_OK && st != CT_ERR_RANK) return fail(st);
    if (d) {
        const ct_status st2 = d->flush();
        const ct_status st3 = st2 == CT_OK ? d->set_progress(DISK_FACTORED, f->n, f->n, (int32_t)o.precision, nb,
                                                             f->rjj_min, f->rjj_max)
                                           : st2;
        if (st3 != CT_OK) return fail(st3);
    }
    *out = f;
    return st;
}
