// diskstore.cuh -- the disk tier of the out-of-core factorisation.
//
// The paper's out-of-core solver (Sec. 2.2) keeps the matrices in secondary
// storage, uses part of the main memory as a cache of their blocks, and
// overlaps the GPU's tasks with the disk transfers of the next tasks'
// operands.  DiskStore is that layer for the left-looking factorisation of
// ooc.cu: the dense A~ (later V and R) lives in one file as column blocks,
// a fixed pool of pinned host slots caches blocks (least recently used
// first out, dirty blocks written back before reuse), and a few I/O threads
// serve reads and writes in the background so that the caller can prefetch
// the blocks of the next tasks while the device works on the current ones.
//
// File layout: a 4096-byte header; then block b (columns [b*bw, c1_b)), the
// rows [0, row_end(c1_b)) of its columns stored column-major with leading
// dimension row_end(c1_b) (rows beyond are zero in A~ and stay zero in V;
// row_end as in the structured lambda block), each block padded to 4096
// bytes; then one auxiliary record per block (tau, T_J, unit-lower top of
// V_J, bw + 2 bw^2 elements, padded to 4096) written as the factorisation
// completes the block.  The header records how far the factorisation got,
// so an interrupted run resumes at the first unfinished superpanel.
#pragma once

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace ctqr {

enum DiskState : int32_t { DISK_ASSEMBLED = 0, DISK_FACTORING = 1, DISK_FACTORED = 2 };

struct DiskHeader {
    char magic[8];
    uint32_t version;
    uint32_t es;  // element size: 4 (float) or 8 (double)
    ct_geometry geom;
    int64_t m, n, rows, lda;  // rays, pixels, M', device leading dimension
    int32_t bw;               // columns per block
    int32_t nblocks;
    int32_t state;            // DiskState
    int32_t prec;             // factor precision once factoring started, else -1
    int32_t nb_inner;         // panel width of that factorisation
    int32_t pad0;
    int64_t done_cols;        // columns whose V, R, tau, T are final on disk
    int64_t dirty_cols;       // columns [done_cols, dirty_cols) may be partly rewritten
    double rjj_min, rjj_max;  // |R_jj| extremes once factored
    uint64_t checksum;        // FNV-1a of every byte before this field
};

class DiskStore {
   public:
    // New file at `path` (truncated) for an M' x n matrix in blocks of bw
    // columns; cache_bytes of pinned host memory for the block cache (at
    // least three blocks are always kept).
    static ct_status create(const char *path, const ct_geometry &g, bool fp64, int64_t m, int64_t n,
                            int64_t rows, int64_t lda, int bw, size_t cache_bytes, DiskStore **out);
    // Existing file: header checked (magic, version, checksum).
    static ct_status open(const char *path, size_t cache_bytes, DiskStore **out);
    ~DiskStore();

    const DiskHeader &header() const { return hdr_; }
    int64_t nblocks() const { return hdr_.nblocks; }
    int bw() const { return hdr_.bw; }
    int64_t block_c0(int64_t b) const { return b * hdr_.bw; }
    int64_t block_w(int64_t b) const { return std::min<int64_t>(hdr_.bw, hdr_.n - b * hdr_.bw); }
    // rows stored for block b = its leading dimension in the file and in a slot
    int64_t block_rows(int64_t b) const;

    // Block b resident in a slot, pinned for the caller; `s` is made to wait
    // for earlier device use of the slot.  Release with release(slot, s) after
    // enqueuing the copies out of the slot on s.
    ct_status acquire(int64_t b, cudaStream_t s, int *slot);
    // A slot to receive block b's new content (no read), pinned; `s` waits
    // for earlier device use of the slot.  Hand it back with commit(slot, s)
    // after enqueuing the copy into the slot on s: written to disk in the
    // background once that copy completes.
    ct_status acquire_write(int64_t b, cudaStream_t s, int *slot);
    ct_status release(int slot, cudaStream_t s);
    ct_status commit(int slot, cudaStream_t s);
    // Start reading block b into a free slot if it is not resident (no wait).
    void prefetch(int64_t b);
    void *slot_ptr(int slot) const { return pool_ + slot_bytes_ * (size_t)slot; }
    int nslots() const { return (int)slots_.size(); }

    // Every write issued so far is on disk (fdatasync).
    ct_status flush();
    // Auxiliary records of blocks [b0, b1): host buffer of (b1-b0) records,
    // record r at r * aux_stride(); tau, T, V top in that order.
    size_t aux_stride() const { return aux_stride_; }
    ct_status write_aux(int64_t b0, int64_t b1, const void *host);
    ct_status read_aux(int64_t b0, int64_t b1, void *host);
    // Header fields updated and written (fdatasync).
    ct_status set_progress(int32_t state, int64_t done_cols, int64_t dirty_cols, int32_t prec,
                           int32_t nb_inner, double rjj_min, double rjj_max);

   private:
    enum SlotState : int { S_FREE = 0, S_READING, S_READY, S_FILLING, S_DIRTY, S_WRITING };
    struct Slot {
        int64_t block = -1;
        int state = S_FREE;
        int pins = 0;
        uint64_t lru = 0;
        cudaEvent_t ev = nullptr;  // last device use of the slot's buffer
    };
    DiskStore() = default;
    ct_status init_cache(size_t cache_bytes);
    int find(int64_t b) const;
    int victim() const;
    ct_status wait_locked(std::unique_lock<std::mutex> &lk, const char *what,
                          const std::function<bool()> &ready);
    void worker();
    ct_status write_header();

    DiskHeader hdr_{};
    std::string path_;
    int fd_ = -1;
    bool direct_ = false;
    std::vector<int64_t> off_;  // file offset of each block (+1: end of the block region)
    size_t aux_stride_ = 0;
    char *pool_ = nullptr;
    size_t pool_bytes_ = 0, slot_bytes_ = 0;
    std::vector<Slot> slots_;
    uint64_t clock_ = 0;
    std::deque<int> queue_;
    std::vector<std::thread> workers_;
    std::mutex mu_;
    std::condition_variable cv_;   // slot state changes
    std::condition_variable qcv_;  // queue
    bool stop_ = false;
    ct_status io_status_ = CT_OK;
    std::string io_error_;
    int device_ = 0;
};

// Every block of the file into dst (host or device memory, leading dimension
// ldd >= rows), rows a block does not store set to zero.  Synchronous.
ct_status disk_export(DiskStore *d, int64_t rows, void *dst, int64_t ldd);

// Process-wide I/O accounting of the disk tier (ct_disk_stats).
void disk_stats_add(int64_t rd, int64_t wr, double rd_s, double wr_s, int hit, int pre, int miss);

}  // namespace ctqr
