// api.cu -- the extern "C" entry points declared in include/ctqr.h.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "diskstore.cuh"
#include "handles.cuh"

namespace ctqr {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ct_status cuda_status(cudaError_t e, const char *what, const char *file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) return CT_ERR_OOM;
    return CT_ERR_CUDA;
}

unsigned long long current_context_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr, *q = nullptr;
        cudaDriverEntryPointQueryResult r1, r2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) ==
                cudaSuccess && r1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) ==
                cudaSuccess && r2 == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrentFn)p;
            get_id = (GetIdFn)q;
        }
    });
    if (!get_current) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int num_sms() {
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (sms[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        sms[dev] = v;
    }
    return sms[dev];
}

DevStatus *device_status() {
    static DevStatus *st[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!st[dev]) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(DevStatus)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(DevStatus));
        cudaDeviceSynchronize();
        st[dev] = (DevStatus *)p;
    }
    return st[dev];
}

ct_status check_device_status(cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    DevStatus h{};
    DevStatus *d = device_status();
    if (!d) return CT_ERR_OOM;
    CT_CUDA(cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.code == DEV_OK) return CT_OK;
    CT_CUDA(cudaMemset(d, 0, sizeof(DevStatus)));
    set_error("device status %d at site %d (aux %d)", h.code, h.where, h.aux);
    switch (h.code) {
        case DEV_TIMEOUT: return CT_ERR_TIMEOUT;
        case DEV_NONFINITE: return CT_ERR_NONFINITE;
        default: return CT_ERR_ARG;
    }
}

// ---- benchmark accounting ---------------------------------------------------
namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_timing{false};
struct ProfRec {
    int cls;
    double flops, bytes;
    int64_t d[4];
    cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;
size_t g_prof_used = 0;
}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
bool timing_enabled() { return g_timing.load(std::memory_order_relaxed); }

// Graphs are used unless the caller turned them off or per-launch timing is on
// (timed launches must run one by one to be measured).
// Disk-backed factors read blocks on the host during the Q sweep, so they
// always run eagerly.
bool graphs_allowed(ct_factor f) { return f->graphs_enabled && !timing_enabled() && !f->store; }

uint64_t graph_key(ct_factor f, int64_t k, const void *extra) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    mix((uint64_t)k);
    mix((uint64_t)(uintptr_t)extra);
    mix((uint64_t)f->solve_sb_req);
    mix((uint64_t)f->solve_chunk);
    mix((uint64_t)(uintptr_t)f->RinvB);
    const Scratch *all[] = {&f->gemm_ws, &f->W, &f->W2, &f->G, &f->Bt, &f->trsm_ws,
                            &f->refine_ws, &f->misc, &f->misc2};
    for (const Scratch *sc : all) {
        mix((uint64_t)(uintptr_t)sc->ptr);
        mix(sc->gen);
    }
    return h | 1ull;  // never 0 (0 = empty slot)
}

ProfScope::ProfScope(int c, cudaStream_t st, double f, double b, int64_t d0, int64_t d1,
                     int64_t d2, int64_t d3)
    : cls(c), s(st), flops(f), bytes(b), slot(-1) {
    if (!g_timing.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_used == g_prof.size()) {
        ProfRec r{};
        if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) return;
        g_prof.push_back(r);
    }
    slot = (int)g_prof_used++;
    ProfRec &r = g_prof[slot];
    r.cls = c;
    r.flops = f;
    r.bytes = b;
    r.d[0] = d0;
    r.d[1] = d1;
    r.d[2] = d2;
    r.d[3] = d3;
    cudaEventRecord(r.e0, s);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[slot].e1, s);
}

namespace {
std::atomic<bool> g_canaries{false};
std::mutex g_scratch_mu;
std::vector<Scratch *> g_scratches;  // live buffers (registration order)
}  // namespace

Scratch::Scratch() {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    g_scratches.push_back(this);
}

ct_status Scratch::ensure(size_t need) {
    if (need <= bytes) return CT_OK;
    if (ptr) {
        cudaError_t e = cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        guarded = false;
        if (e != cudaSuccess) return cuda_status(e, "cudaFree", __FILE__, __LINE__);
    }
    size_t sz = (need + (2u << 20) - 1) & ~(size_t)((2u << 20) - 1);
    const bool guard = g_canaries.load();
    cudaError_t e = cudaMalloc(&ptr, sz + (guard ? kGuardBytes : 0));
    if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_status(e, "cudaMalloc(scratch)", __FILE__, __LINE__);
    }
    if (guard) {
        e = cudaMemset((char *)ptr + sz, kGuardByte, kGuardBytes);
        if (e != cudaSuccess) return cuda_status(e, "cudaMemset(guard)", __FILE__, __LINE__);
    }
    bytes = sz;
    guarded = guard;
    ++gen;
    return CT_OK;
}

Scratch::~Scratch() {
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        for (size_t i = 0; i < g_scratches.size(); ++i)
            if (g_scratches[i] == this) {
                g_scratches.erase(g_scratches.begin() + (long)i);
                break;
            }
    }
    if (ptr) cudaFree(ptr);
}

}  // namespace ctqr

using namespace ctqr;

namespace {

void free_system_storage(ct_system s) {
    cudaFree(s->dense);
    if (s->host_dense) pinned_release(s->host_dense, s->host_bytes);
    delete s->store;
    cudaFree(s->d_cs);
    cudaFree(s->row_nnz);
    cudaFree(s->row_ptr);
    cudaFree(s->col);
    cudaFree(s->val);
    cudaFree(s->col_ptr);
    cudaFree(s->csc_row);
    cudaFree(s->csc_val);
    cudaFree(s->val32);
    cudaFree(s->csc_val32);
}

template <typename T>
ct_status dmalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) return cuda_status(e, "cudaMalloc", __FILE__, __LINE__);
    return CT_OK;
}

bool is_refine(ct_precision p) { return is_refine_prec(p); }

}  // namespace

namespace ctqr {
ct_status rdiag_check(ct_factor f, cudaStream_t s);
// The system without (device_dense = false) or with its dense device matrix.
ct_status build_system_impl(const ct_geometry *geom, ct_precision storage, void *stream,
                            bool device_dense, ct_system *out);
}  // namespace ctqr

extern "C" {

const char *ct_status_str(ct_status s) {
    switch (s) {
        case CT_OK: return "CT_OK";
        case CT_ERR_ARG: return "CT_ERR_ARG";
        case CT_ERR_OOM: return "CT_ERR_OOM";
        case CT_ERR_CUDA: return "CT_ERR_CUDA";
        case CT_ERR_RANK: return "CT_ERR_RANK";
        case CT_ERR_NOCONV: return "CT_ERR_NOCONV";
        case CT_ERR_TIMEOUT: return "CT_ERR_TIMEOUT";
        case CT_ERR_NONFINITE: return "CT_ERR_NONFINITE";
        case CT_ERR_HOSTMEM: return "CT_ERR_HOSTMEM";
        case CT_ERR_STATE: return "CT_ERR_STATE";
        case CT_ERR_UNSUPPORTED: return "CT_ERR_UNSUPPORTED";
        case CT_ERR_IO: return "CT_ERR_IO";
        case CT_ERR_INTERRUPTED: return "CT_ERR_INTERRUPTED";
    }
    return "CT_ERR_UNKNOWN";
}

const char *ct_last_error(void) { return g_err; }

ct_status ct_stats_reset(int32_t timing) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches.store(0);
    g_prof_used = 0;
    g_timing.store(timing != 0);
    return CT_OK;
}

ct_status ct_stats_dump(const char *path) {
    if (!path) return CT_ERR_ARG;
    CT_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    FILE *fp = fopen(path, "w");
    if (!fp) return CT_ERR_ARG;
    fprintf(fp, "class,d0,d1,d2,d3,ms,flops,bytes\n");
    for (size_t i = 0; i < g_prof_used; ++i) {
        const ProfRec &r = g_prof[i];
        float t = 0.f;
        cudaEventElapsedTime(&t, r.e0, r.e1);
        fprintf(fp, "%d,%lld,%lld,%lld,%lld,%.6f,%.6g,%.6g\n", r.cls, (long long)r.d[0],
                (long long)r.d[1], (long long)r.d[2], (long long)r.d[3], t, r.flops, r.bytes);
    }
    fclose(fp);
    return CT_OK;
}

ct_status ct_stats_read(int64_t *launches, double *ms, double *flops, double *bytes,
                        int64_t *count) {
    CT_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (launches) *launches = g_launches.load();
    for (int c = 0; c < PROF_NCLASS; ++c) {
        if (ms) ms[c] = 0;
        if (flops) flops[c] = 0;
        if (bytes) bytes[c] = 0;
        if (count) count[c] = 0;
    }
    for (size_t i = 0; i < g_prof_used; ++i) {
        const ProfRec &r = g_prof[i];
        float t = 0.f;
        CT_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
        if (ms) ms[r.cls] += t;
        if (flops) flops[r.cls] += r.flops;
        if (bytes) bytes[r.cls] += r.bytes;
        if (count) count[r.cls] += 1;
    }
    return CT_OK;
}

ct_status ct_build_system(const ct_geometry *geom, ct_precision storage, void *stream,
                          ct_system *out) {
    return build_system_impl(geom, storage, stream, true, out);
}

}  // extern "C"

ct_status ctqr::build_system_impl(const ct_geometry *geom, ct_precision storage, void *stream,
                                  bool device_dense, ct_system *out) {
    if (!geom || !out) return CT_ERR_ARG;
    *out = nullptr;
    const ct_geometry g = *geom;
    if (g.n_side < 1 || g.n_views < 1 || g.n_bins < 1 || !(g.pixel_width > 0) ||
        !(g.bin_width > 0) || !(g.arc_deg > 0) || !(g.sqrt_lambda >= 0) ||
        !std::isfinite(g.sqrt_lambda) || g.n_side > 46340 ||
        (g.kind != CT_GEOM_PARALLEL && g.kind != CT_GEOM_FAN) ||
        (g.projector != CT_PROJ_SIDDON && g.projector != CT_PROJ_JOSEPH)) {
        set_error("invalid geometry");
        return CT_ERR_ARG;
    }
    if (g.kind == CT_GEOM_FAN &&
        (g.n_bins < 2 || !(g.fan_deg > 0 && g.fan_deg < 180) ||
         !(g.source_dist > 0.7071067811865476 * g.n_side * g.pixel_width) || !std::isfinite(g.source_dist))) {
        set_error("invalid fan-beam geometry: needs n_bins >= 2, 0 < fan_deg < 180 and the source "
                  "outside the image (source_dist > half-diagonal)");
        return CT_ERR_ARG;
    }
    if ((int64_t)g.n_views * g.n_bins > INT32_MAX) {
        set_error("too many rays");
        return CT_ERR_ARG;
    }
    if (storage < CT_FP64 || storage > CT_BF16X3_REFINE) return CT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ct_system sys = new (std::nothrow) ct_system_s;
    if (!sys) return CT_ERR_HOSTMEM;
    sys->geom = g;
    sys->fp64 = storage == CT_FP64;
    sys->m = (int64_t)g.n_views * g.n_bins;
    sys->n = (int64_t)g.n_side * g.n_side;
    sys->rows = sys->m + (g.sqrt_lambda > 0 ? sys->n : 0);
    if (sys->rows < sys->n) {
        set_error("fewer rows (%lld) than unknowns (%lld): add views/bins or sqrt_lambda > 0",
                  (long long)sys->rows, (long long)sys->n);
        delete sys;
        return CT_ERR_ARG;
    }
    sys->lda = round_up(sys->rows, 32);
    auto fail = [&](ct_status st) {
        free_system_storage(sys);
        delete sys;
        return st;
    };
    // Ray geometry on the host in FP64 (libm cos/sin), exact axis values.
    // Parallel: per-view (cos, sin), theta_v = v * arc / n_views degrees.
    // Fan: per-ray (c, s, t) of the line from source v through detector d:
    // theta = beta_v + gamma_d + 90 degrees, t = -source_dist * sin(gamma_d).
    auto snap = [](double &c, double &sn) {
        if (std::fabs(c) < 1e-15) { c = 0.0; sn = (sn > 0.0) ? 1.0 : -1.0; }
        if (std::fabs(sn) < 1e-15) { sn = 0.0; c = (c > 0.0) ? 1.0 : -1.0; }
    };
    std::vector<double> cs;
    if (g.kind == CT_GEOM_FAN) {
        cs.resize(3 * (size_t)sys->m);
        for (int v = 0; v < g.n_views; ++v) {
            const double beta = ((double)v * g.arc_deg / (double)g.n_views) * (M_PI / 180.0);
            for (int d = 0; d < g.n_bins; ++d) {
                const double gamma =
                    (((double)d - 0.5 * (double)(g.n_bins - 1)) * (g.fan_deg / (double)(g.n_bins - 1))) *
                    (M_PI / 180.0);
                const double theta = (beta + gamma) + 0.5 * M_PI;
                double c = std::cos(theta), sn = std::sin(theta);
                snap(c, sn);
                const size_t r = (size_t)v * g.n_bins + d;
                cs[3 * r] = c;
                cs[3 * r + 1] = sn;
                cs[3 * r + 2] = -(g.source_dist * std::sin(gamma));
            }
        }
    } else {
        cs.resize(2 * (size_t)g.n_views);
        for (int v = 0; v < g.n_views; ++v) {
            double theta = ((double)v * g.arc_deg / (double)g.n_views) * (M_PI / 180.0);
            double c = std::cos(theta), sn = std::sin(theta);
            snap(c, sn);
            cs[2 * v] = c;
            cs[2 * v + 1] = sn;
        }
    }
    ct_status st;
    if ((st = dmalloc(&sys->d_cs, cs.size())) != CT_OK) return fail(st);
    if (cudaMemcpyAsync(sys->d_cs, cs.data(), sizeof(double) * cs.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(CT_ERR_CUDA);
    if ((st = dmalloc(&sys->row_nnz, sys->m)) != CT_OK) return fail(st);
    if ((st = dmalloc(&sys->row_ptr, sys->m + 1)) != CT_OK) return fail(st);
    SiddonArgs a{g.n_side, g.n_views, g.n_bins, g.pixel_width, g.bin_width, g.sqrt_lambda,
                 sys->d_cs, g.kind, g.projector, sys->row_nnz, sys->row_ptr, nullptr, nullptr, &sys->tmp};
    if ((st = siddon_build(a, s)) != CT_OK) return fail(st);
    int64_t nnz = 0;
    if (cudaMemcpyAsync(&nnz, sys->row_ptr + sys->m, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(CT_ERR_CUDA);
    sys->nnz = nnz;
    if ((st = dmalloc(&sys->col, nnz)) != CT_OK) return fail(st);
    if ((st = dmalloc(&sys->val, nnz)) != CT_OK) return fail(st);
    const size_t es = sys->fp64 ? 8 : 4;
    if (device_dense) {
        cudaError_t e = cudaMalloc(&sys->dense, es * (size_t)sys->lda * sys->n);
        if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc(dense A)", __FILE__, __LINE__));
        e = cudaMemsetAsync(sys->dense, 0, es * (size_t)sys->lda * sys->n, s);
        if (e != cudaSuccess) return fail(CT_ERR_CUDA);
    }
    a.d_col = sys->col;
    a.d_val = sys->val;
    if ((st = siddon_fill(a, sys->dense, sys->fp64, sys->lda, s)) != CT_OK) return fail(st);
    if ((st = dmalloc(&sys->col_ptr, sys->n + 1)) != CT_OK) return fail(st);
    if ((st = dmalloc(&sys->csc_row, nnz)) != CT_OK) return fail(st);
    if ((st = dmalloc(&sys->csc_val, nnz)) != CT_OK) return fail(st);
    if ((st = build_csc(sys->m, sys->n, nnz, sys->row_ptr, sys->col, sys->val, sys->col_ptr,
                        sys->csc_row, sys->csc_val, sys->tmp, sys->tmp2, s)) != CT_OK)
        return fail(st);
    if ((st = check_device_status(s)) != CT_OK) return fail(st);
    *out = sys;
    return CT_OK;
}

extern "C" {

ct_status ct_system_info(ct_system sys, int64_t *m_rays, int64_t *n_pixels, int64_t *rows,
                         int64_t *lda, int64_t *nnz) {
    if (!sys) return CT_ERR_ARG;
    if (m_rays) *m_rays = sys->m;
    if (n_pixels) *n_pixels = sys->n;
    if (rows) *rows = sys->rows;
    if (lda) *lda = sys->lda;
    if (nnz) *nnz = sys->nnz;
    return CT_OK;
}

ct_status ct_system_device_ptrs(ct_system sys, void **dense, const int64_t **row_ptr,
                                const int32_t **col_idx, const double **val) {
    if (!sys) return CT_ERR_ARG;
    if (dense) *dense = sys->dense;
    if (row_ptr) *row_ptr = sys->row_ptr;
    if (col_idx) *col_idx = sys->col;
    if (val) *val = sys->val;
    return CT_OK;
}

ct_status ct_system_export(ct_system sys, int64_t *row_ptr, int32_t *col_idx, double *val,
                           void *dense, int64_t ldd) {
    if (!sys) return CT_ERR_ARG;
    const void *dsrc = sys->dense ? sys->dense : sys->host_dense;
    if (dense && !dsrc && sys->store) {  // disk: only while the file still holds A~
        if (sys->store->header().state != DISK_ASSEMBLED) return CT_ERR_STATE;
    } else if (dense && !dsrc) {
        return CT_ERR_STATE;
    }
    if (dense && ldd < sys->rows) return CT_ERR_ARG;
    if (row_ptr) CT_CUDA(cudaMemcpy(row_ptr, sys->row_ptr, sizeof(int64_t) * (sys->m + 1), cudaMemcpyDeviceToHost));
    if (col_idx && sys->nnz) CT_CUDA(cudaMemcpy(col_idx, sys->col, sizeof(int32_t) * sys->nnz, cudaMemcpyDeviceToHost));
    if (val && sys->nnz) CT_CUDA(cudaMemcpy(val, sys->val, sizeof(double) * sys->nnz, cudaMemcpyDeviceToHost));
    if (dense && dsrc) {
        const size_t es = sys->fp64 ? 8 : 4;
        CT_CUDA(cudaMemcpy2D(dense, es * ldd, dsrc, es * sys->lda, es * sys->rows, sys->n,
                             cudaMemcpyDefault));
    } else if (dense) {
        CT_TRY(disk_export(sys->store, sys->rows, dense, ldd));
    }
    return CT_OK;
}

ct_status ct_factor_export(ct_factor f, void *VR, int64_t ldv, void *tau) {
    if (!f) return CT_ERR_ARG;
    const size_t es = f->es();
    if (VR) {
        if (ldv < f->M) return CT_ERR_ARG;
        if (f->store) {
            CT_TRY(disk_export(f->store, f->M, VR, ldv));
        } else {
            CT_CUDA(cudaMemcpy2D(VR, es * ldv, f->ooc ? f->VR_host : f->VR, es * f->lda, es * f->M, f->n,
                                 cudaMemcpyDefault));
        }
    }
    if (tau) CT_CUDA(cudaMemcpy(tau, f->tau, es * f->n, cudaMemcpyDeviceToHost));
    return CT_OK;
}

ct_status ct_selftest_wait_timeout(void *stream) { return wait_selftest((cudaStream_t)stream); }

ct_status ct_debug_canaries(int32_t enable) {
    g_canaries.store(enable != 0);
    return CT_OK;
}

ct_status ct_debug_check_canaries(int32_t corrupt_first, int64_t *checked, int64_t *corrupted) {
    if (!checked || !corrupted) return CT_ERR_ARG;
    *checked = 0;
    *corrupted = 0;
    CT_CUDA(cudaDeviceSynchronize());
    std::vector<unsigned char> host(kGuardBytes);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    bool injected = false;
    for (Scratch *sc : g_scratches) {
        if (!sc->guarded || !sc->ptr) continue;
        char *guard = (char *)sc->ptr + sc->bytes;
        if (corrupt_first && !injected) {  // inside the allocation: the guard band itself
            CT_CUDA(cudaMemset(guard, 0, 1));
            injected = true;
        }
        CT_CUDA(cudaMemcpy(host.data(), guard, kGuardBytes, cudaMemcpyDeviceToHost));
        ++*checked;
        for (size_t i = 0; i < kGuardBytes; ++i)
            if (host[i] != kGuardByte) {
                ++*corrupted;
                break;
            }
    }
    return CT_OK;
}

ct_status ct_forward_project(ct_system sys, const double *X, int64_t ldx, int32_t k, double *P,
                             int64_t ldp, void *stream) {
    if (!sys || k < 0 || ldx < sys->n || ldp < sys->m) return CT_ERR_ARG;
    if (k == 0) return CT_OK;
    if (!X || !P) return CT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // column-major in, column-major out: go through slice-fastest staging.
    double *xr = nullptr, *pr = nullptr;
    CT_CUDA(cudaMallocAsync((void **)&xr, sizeof(double) * sys->n * k, s));
    CT_CUDA(cudaMallocAsync((void **)&pr, sizeof(double) * sys->m * k, s));
    ct_status st = transpose_d(X, ldx, xr, k, sys->n, k, s);  // (n x k, ld ldx) -> row-major
    SparseSys S = sys->sparse();
    S.sqrt_lambda = 0.0;
    if (st == CT_OK) st = spmm_ax(S, k, xr, 0.0, nullptr, 1.0, pr, s);
    if (st == CT_OK) st = transpose_d(pr, k, P, ldp, k, sys->m, s);  // row-major (m x k) -> col-major
    cudaFreeAsync(xr, s);
    cudaFreeAsync(pr, s);
    if (st != CT_OK) return st;
    return check_device_status(s);
}

ct_status ct_qr_factor(ct_system sys, const ct_opts *opts, void *stream, ct_factor *out) {
    if (!sys || !out) return CT_ERR_ARG;
    *out = nullptr;
    if (!sys->dense) {
        set_error("system matrix already consumed by a factorisation");
        return CT_ERR_STATE;
    }
    ct_opts o{};
    o.precision = sys->fp64 ? CT_FP64 : CT_TF32_REFINE;
    if (opts) o = *opts;
    if (o.precision < CT_FP64 || o.precision > CT_BF16X3_REFINE) return CT_ERR_ARG;
    if ((o.precision == CT_FP64) != sys->fp64) {
        set_error("precision does not match the system's storage");
        return CT_ERR_ARG;
    }
    if (!sys->dense) {
        set_error(sys->host_dense ? "the dense matrix is in host memory: use ct_qr_factor_ooc"
                  : sys->store    ? "the dense matrix is on disk: use ct_qr_factor_ooc"
                                  : "the system's dense storage was already consumed by a factor");
        return CT_ERR_ARG;
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
    int nb = o.nb_inner > 0 ? o.nb_inner : (f->fp64 ? 16 : 32);
    nb = std::min(nb, 32);
    int NB = o.nb_outer > 0 ? o.nb_outer : (f->fp64 ? 32 : (f->kind == GEMM_F32 ? 128 : (f->upd_kind == GEMM_BF16 ? 2048 : 1536)));
    NB = (int)round_up(std::max(NB, nb), nb);
    if (NB % 32) NB = (int)round_up(NB, 32);
    f->nb = nb;
    f->NB = NB;
    f->nblocks = ceil_div(f->n, NB);
    const size_t es = f->es();
    auto fail = [&](ct_status st) {
        // the dense storage stays consumed only on success
        if (f->VR && !sys->dense) sys->dense = f->VR;
        cudaFree(f->tau);
        cudaFree(f->Tall);
        cudaFree(f->Vtop);
        delete f;
        return st;
    };
    if (cudaMalloc(&f->tau, es * (size_t)f->n) != cudaSuccess) return fail(CT_ERR_OOM);
    if (cudaMalloc(&f->Tall, es * (size_t)f->nblocks * NB * NB) != cudaSuccess) return fail(CT_ERR_OOM);
    if (cudaMalloc(&f->Vtop, es * (size_t)f->nblocks * NB * NB) != cudaSuccess) return fail(CT_ERR_OOM);
    f->VR = sys->dense;
    sys->dense = nullptr;
    f->Rm = f->VR;
    f->ldr = f->lda;
    ct_status st = qr_factor_run(f, s);
    if (st != CT_OK) return fail(st);
    st = rdiag_check(f, s);
    if (st == CT_ERR_RANK) {  // keep the factor: the caller may still inspect it
        *out = f;
        return CT_ERR_RANK;
    }
    if (st != CT_OK) return fail(st);
    *out = f;
    return CT_OK;
}

}  // extern "C"

// min/max |R_jj| into the factor, and the rank test |R_jj| >= n u max|R_jj|.
ct_status ctqr::rdiag_check(ct_factor f, cudaStream_t s) {
    double *dmm = nullptr;
    if (cudaMallocAsync((void **)&dmm, 2 * sizeof(double), s) != cudaSuccess) return CT_ERR_OOM;
    ct_status st = rdiag_minmax(f->fp64, f->Rm, f->ldr, f->n, dmm, s);
    double hmm[2] = {0, 0};
    if (st == CT_OK && cudaMemcpyAsync(hmm, dmm, sizeof(hmm), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = CT_ERR_CUDA;
    cudaFreeAsync(dmm, s);
    if (st == CT_OK) st = check_device_status(s);
    if (st != CT_OK) return st;
    f->rjj_min = hmm[0];
    f->rjj_max = hmm[1];
    const double u = f->fp64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
    if (!(f->rjj_min >= (double)f->n * u * f->rjj_max)) {
        set_error("rank deficient: min|R_jj| = %g, max|R_jj| = %g", f->rjj_min, f->rjj_max);
        return CT_ERR_RANK;
    }
    return CT_OK;
}

extern "C" {

ct_status ct_factor_device_ptrs(ct_factor f, void **VR, int64_t *lda, void **tau) {
    if (!f) return CT_ERR_ARG;
    if (f->ooc) {
        set_error("out-of-core factor: V and R are in host memory");
        return CT_ERR_UNSUPPORTED;
    }
    if (VR) *VR = f->VR;
    if (lda) *lda = f->lda;
    if (tau) *tau = f->tau;
    return CT_OK;
}

}  // extern "C"

// The solve plan of ct_opts (superblock rows of the triangular solve, least
// split-K depth of the solve's GEMMs): validated and recorded in the factor;
// a new superblock size drops the stored superblock inverses, which the next
// triangular solve rebuilds.
static ct_status apply_solve_plan(ct_factor f, const ct_opts *o) {
    const int sb = o ? o->solve_block : 0;
    const int chunk = o ? o->solve_split : 0;
    if (sb != 0) {
        const int q = sb / 128;
        if (sb < 128 || sb > 16384 || sb % 128 != 0 || (q & (q - 1)) != 0) {
            set_error("solve_block %d: 0, or 128 times a power of two up to 16384", sb);
            return CT_ERR_ARG;
        }
    }
    if (chunk != 0 && (chunk < 32 || chunk % 32 != 0)) {
        set_error("solve_split %d: 0, or a multiple of 32", chunk);
        return CT_ERR_ARG;
    }
    f->solve_chunk = chunk;
    if (sb != f->solve_sb_req) {
        if (f->RinvB) {  // cudaFree waits for the device, so no solve still reads them
            CT_CUDA(cudaFree(f->RinvB));
            CT_CUDA(cudaFree(f->RinvTB));
            f->RinvB = f->RinvTB = nullptr;
            f->trsm_sb = 0;
        }
        f->solve_sb_req = sb;
    }
    return CT_OK;
}

extern "C" {

ct_status ct_solve(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                   const ct_opts *opts, void *stream, ct_solve_info *info) {
    if (!f || k < 0 || ldb < f->m || ldx < f->n) return CT_ERR_ARG;
    CT_TRY(apply_solve_plan(f, opts));
    f->graphs_enabled = !(opts && (opts->flags & CT_OPT_NO_GRAPHS));
    if (k == 0) return CT_OK;
    if (!B || !X) return CT_ERR_ARG;
    if (is_refine(f->prec) && !f->sys) return CT_ERR_STATE;
    return solve_run(f, B, ldb, k, X, ldx, opts, (cudaStream_t)stream, info);
}

ct_status ct_solve_host(ct_factor f, const void *B, int64_t ldb, int32_t k, void *X, int64_t ldx,
                        const ct_opts *opts, void *stream, ct_solve_info *info) {
    if (!f || k < 0 || ldb < f->m || ldx < f->n) return CT_ERR_ARG;
    CT_TRY(apply_solve_plan(f, opts));
    if (k == 0) return CT_OK;
    if (!B || !X) return CT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    f->graphs_enabled = !(opts && (opts->flags & CT_OPT_NO_GRAPHS));
    const size_t ies = f->prec == CT_FP32 ? 4 : 8;
    const size_t bbytes = ies * (size_t)f->m * k, xbytes = ies * (size_t)f->n * k;
    CT_TRY(f->host_pinned.ensure(bbytes + xbytes + 256));
    void *dB = f->host_pinned.ptr;
    void *dX = (char *)f->host_pinned.ptr + ((bbytes + 255) & ~(size_t)255);
    CT_CUDA(cudaMemcpy2DAsync(dB, ies * f->m, B, ies * ldb, ies * f->m, k, cudaMemcpyHostToDevice, s));
    ct_status st = solve_run(f, dB, f->m, k, dX, f->n, opts, s, info);
    if (st != CT_OK && st != CT_ERR_NOCONV) return st;
    CT_CUDA(cudaMemcpy2DAsync(X, ies * ldx, dX, ies * f->n, ies * f->n, k, cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaStreamSynchronize(s));
    return st;
}

ct_status ct_solve_adjoint(ct_factor f, const void *gX, int64_t ldgx, int32_t k, void *gB,
                           int64_t ldgb, const ct_opts *opts, void *stream, ct_solve_info *info) {
    if (!f || k < 0 || ldgx < f->n || ldgb < f->m) return CT_ERR_ARG;
    CT_TRY(apply_solve_plan(f, opts));
    f->graphs_enabled = !(opts && (opts->flags & CT_OPT_NO_GRAPHS));
    if (k == 0) return CT_OK;
    if (!gX || !gB) return CT_ERR_ARG;
    return adjoint_run(f, gX, ldgx, k, gB, ldgb, opts, (cudaStream_t)stream, info);
}

void ct_system_free(ct_system sys) {
    if (!sys) return;
    free_system_storage(sys);
    delete sys;
}

void ct_factor_free(ct_factor f) {
    if (!f) return;
    if (f->g_direct.exec) cudaGraphExecDestroy(f->g_direct.exec);
    if (f->g_iter.exec) cudaGraphExecDestroy(f->g_iter.exec);
    if (f->side) cudaStreamDestroy(f->side);
    if (f->ev_fork) cudaEventDestroy(f->ev_fork);
    if (f->ev_join) cudaEventDestroy(f->ev_join);
    if (f->pinned) cudaFreeHost(f->pinned);
    cudaFree(f->Rinv);
    cudaFree(f->RinvT);
    cudaFree(f->Rt);
    if (f->ooc) {
        cudaFree(f->Rm);
        cudaFree(f->stage);
        if (f->VR_host) pinned_release(f->VR_host, f->host_bytes);
        delete f->store;
    }
    cudaFree(f->RinvB);
    cudaFree(f->RinvTB);
    cudaFree(f->VR);
    cudaFree(f->tau);
    cudaFree(f->Tall);
    cudaFree(f->Vtop);
    delete f;
}

ct_status ct_gemm(int32_t kind, char transa, char transb, int64_t M, int64_t N, int64_t K,
                  double alpha, const void *A, int64_t lda, const void *B, int64_t ldb, double beta,
                  void *C, int64_t ldc, void *stream) {
    if (kind < 0 || kind > 5) return CT_ERR_ARG;
    const bool ta = transa == 'T' || transa == 't';
    const bool tb = transb == 'T' || transb == 't';
    if ((!ta && transa != 'N' && transa != 'n') || (!tb && transb != 'N' && transb != 'n'))
        return CT_ERR_ARG;
    if (M < 0 || N < 0 || K < 0) return CT_ERR_ARG;
    if (ldc < std::max<int64_t>(1, M)) return CT_ERR_ARG;
    if (lda < std::max<int64_t>(1, ta ? K : M) || ldb < std::max<int64_t>(1, tb ? N : K))
        return CT_ERR_ARG;
    static Scratch ws;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    GemmArgs g{(GemmKind)kind, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc};
    cudaStream_t s = (cudaStream_t)stream;
    CT_TRY(gemm(g, ws, s));
    return check_device_status(s);
}

}  // extern "C"
