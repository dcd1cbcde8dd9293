// diskstore.cu -- block file, pinned block cache and I/O threads of the disk
// tier (see diskstore.cuh).
#include <errno.h>
#include <stddef.h>
#include <fcntl.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <new>

#include "diskstore.cuh"
#include "handles.cuh"

namespace ctqr {
namespace {

constexpr char kDiskMagic[8] = {'C', 'T', 'Q', 'R', 'D', 'S', 'K', '1'};
constexpr uint32_t kDiskVersion = 1;
constexpr size_t kPage = 4096;
constexpr int kIoThreads = 4;
constexpr double kWaitLimitS = 900.0;  // host-side wait on a block before giving up

static_assert(sizeof(DiskHeader) <= kPage, "disk header must fit one page");

size_t page_up(size_t b) { return (b + kPage - 1) / kPage * kPage; }

uint64_t fnv1a(const void *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

// pread / pwrite the whole range (short transfers and EINTR retried).
bool full_io(bool rd, int fd, void *buf, size_t bytes, int64_t off) {
    char *p = (char *)buf;
    while (bytes > 0) {
        const ssize_t r = rd ? pread(fd, p, bytes, off) : pwrite(fd, p, bytes, off);
        if (r < 0 && errno == EINTR) continue;
        if (r <= 0) return false;
        p += r;
        bytes -= (size_t)r;
        off += r;
    }
    return true;
}

// An aligned host buffer for O_DIRECT transfers outside the cache.
struct AlignedBuf {
    void *p = nullptr;
    explicit AlignedBuf(size_t n) {
        if (posix_memalign(&p, kPage, page_up(std::max<size_t>(n, 1))) != 0) p = nullptr;
    }
    ~AlignedBuf() { free(p); }
};

std::mutex g_stats_mu;
int64_t g_rd = 0, g_wr = 0, g_hit = 0, g_pre = 0, g_miss = 0;
double g_rd_s = 0, g_wr_s = 0;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void disk_stats_add(int64_t rd, int64_t wr, double rd_s, double wr_s, int hit, int pre, int miss) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_rd += rd;
    g_wr += wr;
    g_rd_s += rd_s;
    g_wr_s += wr_s;
    g_hit += hit;
    g_pre += pre;
    g_miss += miss;
}

int64_t DiskStore::block_rows(int64_t b) const {
    const int64_t c1 = std::min<int64_t>(hdr_.n, (b + 1) * (int64_t)hdr_.bw);
    return hdr_.rows > hdr_.m ? std::min<int64_t>(hdr_.rows, hdr_.m + c1) : hdr_.rows;
}

static ct_status open_file(const char *path, bool create, int *fd, bool *direct) {
    const int base = O_RDWR | (create ? (O_CREAT | O_TRUNC) : 0);
    *direct = true;
    *fd = open(path, base | O_DIRECT, 0644);
    if (*fd < 0 && errno == EINVAL) {  // file systems without direct I/O (tmpfs)
        *direct = false;
        *fd = open(path, base, 0644);
    }
    if (*fd < 0) {
        set_error("cannot open '%s': %s", path, strerror(errno));
        return CT_ERR_ARG;
    }
    return CT_OK;
}

ct_status DiskStore::create(const char *path, const ct_geometry &g, bool fp64, int64_t m, int64_t n,
                            int64_t rows, int64_t lda, int bw, size_t cache_bytes, DiskStore **out) {
    *out = nullptr;
    if (!path || !*path || bw <= 0 || n <= 0) return CT_ERR_ARG;
    DiskStore *d = new (std::nothrow) DiskStore;
    if (!d) return CT_ERR_HOSTMEM;
    memcpy(d->hdr_.magic, kDiskMagic, 8);
    d->hdr_.version = kDiskVersion;
    d->hdr_.es = fp64 ? 8 : 4;
    d->hdr_.geom = g;
    d->hdr_.m = m;
    d->hdr_.n = n;
    d->hdr_.rows = rows;
    d->hdr_.lda = lda;
    d->hdr_.bw = bw;
    d->hdr_.nblocks = (int32_t)ceil_div(n, bw);
    d->hdr_.state = DISK_ASSEMBLED;
    d->hdr_.prec = -1;
    d->path_ = path;
    ct_status st = open_file(path, true, &d->fd_, &d->direct_);
    if (st == CT_OK) st = d->init_cache(cache_bytes);
    if (st == CT_OK && ftruncate(d->fd_, d->off_.back() + (int64_t)(d->aux_stride_ * d->hdr_.nblocks)) != 0) {
        set_error("cannot size '%s': %s", path, strerror(errno));
        st = CT_ERR_IO;
    }
    if (st == CT_OK) st = d->write_header();
    if (st != CT_OK) {
        delete d;
        return st;
    }
    *out = d;
    return CT_OK;
}

ct_status DiskStore::open(const char *path, size_t cache_bytes, DiskStore **out) {
    *out = nullptr;
    if (!path || !*path) return CT_ERR_ARG;
    DiskStore *d = new (std::nothrow) DiskStore;
    if (!d) return CT_ERR_HOSTMEM;
    d->path_ = path;
    ct_status st = open_file(path, false, &d->fd_, &d->direct_);
    if (st == CT_OK) {
        AlignedBuf h(kPage);
        if (!h.p || !full_io(true, d->fd_, h.p, kPage, 0)) {
            set_error("cannot read the header of '%s'", path);
            st = CT_ERR_ARG;
        } else {
            memcpy(&d->hdr_, h.p, sizeof(DiskHeader));
            const DiskHeader &x = d->hdr_;
            if (memcmp(x.magic, kDiskMagic, 8) != 0 || x.version != kDiskVersion) {
                set_error("'%s' is not a version-%u disk matrix file", path, kDiskVersion);
                st = CT_ERR_ARG;
            } else if (x.checksum != fnv1a(&x, offsetof(DiskHeader, checksum))) {
                set_error("header checksum mismatch in '%s'", path);
                st = CT_ERR_ARG;
            } else if ((x.es != 4 && x.es != 8) || x.bw <= 0 || x.n <= 0 || x.rows < x.n ||
                       x.nblocks != ceil_div(x.n, x.bw) || x.done_cols < 0 || x.done_cols > x.n ||
                       x.dirty_cols < x.done_cols || x.dirty_cols > x.n) {
                set_error("inconsistent header in '%s'", path);
                st = CT_ERR_ARG;
            }
        }
    }
    if (st == CT_OK) st = d->init_cache(cache_bytes);
    if (st != CT_OK) {
        delete d;
        return st;
    }
    *out = d;
    return CT_OK;
}

ct_status DiskStore::init_cache(size_t cache_bytes) {
    const size_t es = hdr_.es;
    off_.assign(hdr_.nblocks + 1, 0);
    off_[0] = kPage;
    slot_bytes_ = 0;
    for (int64_t b = 0; b < hdr_.nblocks; ++b) {
        const size_t bytes = page_up(es * (size_t)block_rows(b) * (size_t)block_w(b));
        off_[b + 1] = off_[b] + (int64_t)bytes;
        slot_bytes_ = std::max(slot_bytes_, bytes);
    }
    aux_stride_ = page_up(es * ((size_t)hdr_.bw + 2 * (size_t)hdr_.bw * hdr_.bw));
    const int n = (int)std::max<size_t>(3, cache_bytes / slot_bytes_);
    const int nslots = (int)std::min<int64_t>(n, std::max<int64_t>(3, hdr_.nblocks));
    size_t got = 0;
    void *p = nullptr;
    if (pinned_acquire(slot_bytes_ * nslots, &p, &got) != CT_OK) {
        set_error("cannot pin %zu B for the block cache", slot_bytes_ * nslots);
        return CT_ERR_HOSTMEM;
    }
    pool_ = (char *)p;
    pool_bytes_ = got;
    if (direct_ && ((uintptr_t)pool_ % kPage) != 0) {  // direct I/O needs page-aligned buffers
        ::close(fd_);
        fd_ = ::open(path_.c_str(), O_RDWR);
        direct_ = false;
        if (fd_ < 0) {
            set_error("cannot reopen '%s': %s", path_.c_str(), strerror(errno));
            return CT_ERR_IO;
        }
    }
    slots_.resize(nslots);
    for (auto &s : slots_)
        CT_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming | cudaEventBlockingSync));
    CT_CUDA(cudaGetDevice(&device_));
    for (int i = 0; i < kIoThreads; ++i) workers_.emplace_back([this] { worker(); });
    return CT_OK;
}

DiskStore::~DiskStore() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    qcv_.notify_all();
    for (auto &t : workers_) t.join();  // queued writes finish first
    if (fd_ >= 0) ::close(fd_);
    for (auto &s : slots_)
        if (s.ev) cudaEventDestroy(s.ev);
    if (pool_) pinned_release(pool_, pool_bytes_);
}

void DiskStore::worker() {
    cudaSetDevice(device_);
    for (;;) {
        std::unique_lock<std::mutex> lk(mu_);
        qcv_.wait(lk, [&] { return stop_ || !queue_.empty(); });
        if (queue_.empty()) return;
        const int i = queue_.front();
        queue_.pop_front();
        Slot &sl = slots_[i];
        const bool rd = sl.state == S_READING;
        if (!rd) sl.state = S_WRITING;
        const int64_t b = sl.block;
        cudaEvent_t ev = sl.ev;
        lk.unlock();
        // the device's last use of the buffer: the copy out of the old
        // content (read) or the copy that filled it (write)
        const cudaError_t ce = cudaEventSynchronize(ev);
        const size_t bytes = (size_t)(off_[b + 1] - off_[b]);
        const double t0 = now_s();
        const bool ok = ce == cudaSuccess && full_io(rd, fd_, slot_ptr(i), bytes, off_[b]);
        const double dt = now_s() - t0;
        const int err = errno;
        lk.lock();
        if (!ok && io_status_ == CT_OK) {
            io_status_ = ce != cudaSuccess ? CT_ERR_CUDA : CT_ERR_IO;
            io_error_ = std::string(rd ? "read" : "write") + " of block " + std::to_string(b) + " of '" +
                        path_ + "' failed: " + (ce != cudaSuccess ? cudaGetErrorString(ce) : strerror(err));
        }
        if (rd) {
            sl.state = ok ? S_READY : S_FREE;
            if (!ok) sl.block = -1;
        } else {
            sl.state = S_READY;
        }
        disk_stats_add(rd && ok ? (int64_t)bytes : 0, !rd && ok ? (int64_t)bytes : 0, rd ? dt : 0,
                       rd ? 0 : dt, 0, 0, 0);
        cv_.notify_all();
    }
}

int DiskStore::find(int64_t b) const {
    for (int i = 0; i < (int)slots_.size(); ++i)
        if (slots_[i].block == b && slots_[i].state != S_FREE) return i;
    return -1;
}

// A slot that can take a new block now: free first, else the least recently
// used clean one that nobody holds.
int DiskStore::victim() const {
    int best = -1;
    for (int i = 0; i < (int)slots_.size(); ++i) {
        const Slot &s = slots_[i];
        if (s.pins > 0) continue;
        if (s.state == S_FREE) return i;
        if (s.state == S_READY && (best < 0 || s.lru < slots_[best].lru)) best = i;
    }
    return best;
}

ct_status DiskStore::wait_locked(std::unique_lock<std::mutex> &lk, const char *what,
                                 const std::function<bool()> &ready) {
    const double t0 = now_s();
    while (!ready()) {
        if (io_status_ != CT_OK) {
            set_error("%s", io_error_.c_str());
            return io_status_;
        }
        bool all_pinned = true;
        for (auto &s : slots_) all_pinned = all_pinned && s.pins > 0;
        if (all_pinned) {
            set_error("block cache of %d slots is fully held while waiting for %s", nslots(), what);
            return CT_ERR_STATE;
        }
        if (now_s() - t0 > kWaitLimitS) {
            set_error("gave up after %.0f s waiting for %s of '%s'", kWaitLimitS, what, path_.c_str());
            return CT_ERR_TIMEOUT;
        }
        cv_.wait_for(lk, std::chrono::milliseconds(200));
    }
    if (io_status_ != CT_OK) {
        set_error("%s", io_error_.c_str());
        return io_status_;
    }
    return CT_OK;
}

ct_status DiskStore::acquire(int64_t b, cudaStream_t s, int *slot) {
    if (b < 0 || b >= hdr_.nblocks) return CT_ERR_ARG;
    std::unique_lock<std::mutex> lk(mu_);
    int i = find(b);
    int hit = 0, pre = 0, miss = 0;
    if (i >= 0 && slots_[i].state == S_FILLING) {
        set_error("block %lld is being rewritten", (long long)b);
        return CT_ERR_STATE;
    }
    if (i >= 0) {
        (slots_[i].state == S_READING ? pre : hit) = 1;
    } else {
        miss = 1;
        CT_TRY(wait_locked(lk, "a free cache slot", [&] { return victim() >= 0; }));
        i = victim();
        slots_[i].block = b;
        slots_[i].state = S_READING;
        queue_.push_back(i);
        qcv_.notify_one();
    }
    slots_[i].pins++;  // held while waiting, so it cannot be chosen as a victim
    ct_status st = wait_locked(lk, "a block read", [&] { return slots_[i].state != S_READING; });
    if (st == CT_OK && slots_[i].block != b) st = CT_ERR_IO;
    if (st != CT_OK) {
        slots_[i].pins--;
        return st;
    }
    slots_[i].lru = ++clock_;
    lk.unlock();
    disk_stats_add(0, 0, 0, 0, hit, pre, miss);
    *slot = i;
    CT_CUDA(cudaStreamWaitEvent(s, slots_[i].ev, 0));
    return CT_OK;
}

ct_status DiskStore::acquire_write(int64_t b, cudaStream_t s, int *slot) {
    if (b < 0 || b >= hdr_.nblocks) return CT_ERR_ARG;
    std::unique_lock<std::mutex> lk(mu_);
    int i = find(b);
    if (i >= 0) {  // reuse its slot once no read, write or holder is pending
        CT_TRY(wait_locked(lk, "a pending transfer", [&] {
            const Slot &x = slots_[i];
            return x.block != b || (x.pins == 0 && (x.state == S_READY || x.state == S_FREE));
        }));
        if (slots_[i].block != b) i = -1;
    }
    if (i < 0) {
        CT_TRY(wait_locked(lk, "a free cache slot", [&] { return victim() >= 0; }));
        i = victim();
    }
    slots_[i].block = b;
    slots_[i].state = S_FILLING;
    slots_[i].pins = 1;
    slots_[i].lru = ++clock_;
    lk.unlock();
    *slot = i;
    CT_CUDA(cudaStreamWaitEvent(s, slots_[i].ev, 0));
    return CT_OK;
}

ct_status DiskStore::release(int slot, cudaStream_t s) {
    CT_CUDA(cudaEventRecord(slots_[slot].ev, s));
    std::lock_guard<std::mutex> lk(mu_);
    slots_[slot].pins--;
    cv_.notify_all();
    return CT_OK;
}

ct_status DiskStore::commit(int slot, cudaStream_t s) {
    CT_CUDA(cudaEventRecord(slots_[slot].ev, s));
    std::lock_guard<std::mutex> lk(mu_);
    slots_[slot].pins--;
    slots_[slot].state = S_DIRTY;
    queue_.push_back(slot);
    qcv_.notify_one();
    cv_.notify_all();
    return CT_OK;
}

void DiskStore::prefetch(int64_t b) {
    if (b < 0 || b >= hdr_.nblocks) return;
    std::lock_guard<std::mutex> lk(mu_);
    if (io_status_ != CT_OK || find(b) >= 0) return;
    const int i = victim();
    if (i < 0) return;
    slots_[i].block = b;
    slots_[i].state = S_READING;
    slots_[i].lru = ++clock_;
    queue_.push_back(i);
    qcv_.notify_one();
}

ct_status DiskStore::flush() {
    {
        std::unique_lock<std::mutex> lk(mu_);
        CT_TRY(wait_locked(lk, "the write-back", [&] {
            for (auto &x : slots_)
                if (x.state == S_DIRTY || x.state == S_WRITING) return false;
            return true;
        }));
    }
    if (fdatasync(fd_) != 0) {
        set_error("fdatasync of '%s' failed: %s", path_.c_str(), strerror(errno));
        return CT_ERR_IO;
    }
    return CT_OK;
}

ct_status DiskStore::write_aux(int64_t b0, int64_t b1, const void *host) {
    if (b0 < 0 || b1 > hdr_.nblocks || b0 >= b1) return CT_OK;
    const size_t bytes = aux_stride_ * (size_t)(b1 - b0);
    const double t0 = now_s();
    if (!full_io(false, fd_, (void *)host, bytes, off_.back() + (int64_t)(aux_stride_ * b0))) {
        set_error("write of the block records of '%s' failed: %s", path_.c_str(), strerror(errno));
        return CT_ERR_IO;
    }
    disk_stats_add(0, (int64_t)bytes, 0, now_s() - t0, 0, 0, 0);
    return CT_OK;
}

ct_status DiskStore::read_aux(int64_t b0, int64_t b1, void *host) {
    if (b0 < 0 || b1 > hdr_.nblocks || b0 >= b1) return CT_OK;
    const size_t bytes = aux_stride_ * (size_t)(b1 - b0);
    const double t0 = now_s();
    if (!full_io(true, fd_, host, bytes, off_.back() + (int64_t)(aux_stride_ * b0))) {
        set_error("read of the block records of '%s' failed: %s", path_.c_str(), strerror(errno));
        return CT_ERR_IO;
    }
    disk_stats_add((int64_t)bytes, 0, now_s() - t0, 0, 0, 0, 0);
    return CT_OK;
}

ct_status DiskStore::write_header() {
    hdr_.checksum = fnv1a(&hdr_, offsetof(DiskHeader, checksum));
    AlignedBuf h(kPage);
    if (!h.p) return CT_ERR_HOSTMEM;
    memset(h.p, 0, kPage);
    memcpy(h.p, &hdr_, sizeof(DiskHeader));
    if (!full_io(false, fd_, h.p, kPage, 0) || fdatasync(fd_) != 0) {
        set_error("write of the header of '%s' failed: %s", path_.c_str(), strerror(errno));
        return CT_ERR_IO;
    }
    return CT_OK;
}

ct_status DiskStore::set_progress(int32_t state, int64_t done_cols, int64_t dirty_cols, int32_t prec,
                                  int32_t nb_inner, double rjj_min, double rjj_max) {
    hdr_.state = state;
    hdr_.done_cols = done_cols;
    hdr_.dirty_cols = dirty_cols;
    hdr_.prec = prec;
    hdr_.nb_inner = nb_inner;
    hdr_.rjj_min = rjj_min;
    hdr_.rjj_max = rjj_max;
    return write_header();
}

ct_status disk_export(DiskStore *d, int64_t rows, void *dst, int64_t ldd) {
    const size_t es = d->header().es;
    cudaPointerAttributes pa{};
    const bool on_device = cudaPointerGetAttributes(&pa, dst) == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    cudaStream_t s = nullptr;
    CT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ct_status st = CT_OK;
    for (int64_t b = 0; b < d->nblocks() && st == CT_OK; ++b) {
        int slot = -1;
        if ((st = d->acquire(b, s, &slot)) != CT_OK) break;
        const int64_t rb = d->block_rows(b), w = d->block_w(b);
        char *out = (char *)dst + es * (size_t)d->block_c0(b) * ldd;
        if (cudaMemcpy2DAsync(out, es * ldd, d->slot_ptr(slot), es * rb, es * rb, w, cudaMemcpyDefault, s) !=
            cudaSuccess)
            st = CT_ERR_CUDA;
        const ct_status st2 = d->release(slot, s);
        if (st == CT_OK) st = st2;
        if (st == CT_OK && rows > rb) {
            if (on_device) {
                if (cudaMemset2DAsync(out + es * rb, es * ldd, 0, es * (rows - rb), w, s) != cudaSuccess)
                    st = CT_ERR_CUDA;
            } else {
                for (int64_t c = 0; c < w; ++c) memset(out + es * (c * ldd + rb), 0, es * (rows - rb));
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess && st == CT_OK) st = CT_ERR_CUDA;
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return st;
}

}  // namespace ctqr

extern "C" ct_status ct_disk_stats(int32_t reset, int64_t *bytes_read, int64_t *bytes_written,
                                   int64_t *hits, int64_t *prefetched, int64_t *misses,
                                   double *read_s, double *write_s) {
    using namespace ctqr;
    std::lock_guard<std::mutex> lk(g_stats_mu);
    if (bytes_read) *bytes_read = g_rd;
    if (bytes_written) *bytes_written = g_wr;
    if (hits) *hits = g_hit;
    if (prefetched) *prefetched = g_pre;
    if (misses) *misses = g_miss;
    if (read_s) *read_s = g_rd_s;
    if (write_s) *write_s = g_wr_s;
    if (reset) {
        g_rd = g_wr = g_hit = g_pre = g_miss = 0;
        g_rd_s = g_wr_s = 0;
    }
    return CT_OK;
}
