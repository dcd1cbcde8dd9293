// common.cuh -- internal helpers of libctqr: status handling, bounded waits,
// device status word, small PTX wrappers (mbarrier, TMA, tcgen05).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "../../include/ctqr.h"

namespace ctqr {

// ---------------------------------------------------------------------------
// Host-side error plumbing.
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
ct_status cuda_status(cudaError_t e, const char *what, const char *file, int line);

#define CT_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) return ctqr::cuda_status(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define CT_TRY(expr)                         \
    do {                                     \
        ct_status _s = (expr);               \
        if (_s != CT_OK) return _s;          \
    } while (0)

// Device status word codes (written by kernels, read by the host at sync points).
enum DevCode : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NONFINITE = 2, DEV_BADARG = 3 };

struct DevStatus {
    int code;    // first error code raised (DevCode)
    int where;   // kernel-specific location tag
    int aux;     // kernel-specific detail
    int pad;
};

// Per-process device status word (one per device ordinal, allocated lazily).
DevStatus *device_status();
// Reads, clears and converts the device status word (synchronises `stream`).
ct_status check_device_status(cudaStream_t stream);

// Bounded wait budget for device spin loops (nanoseconds of %globaltimer).
constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void raise_status(DevStatus *st, int code, int where, int aux) {
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->where = where;
        st->aux = aux;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on the phase with the given parity.  Returns false (and raises
// DEV_TIMEOUT) if the wait did not end within kWaitLimitNs, or if another
// thread of the grid already raised an error (so that all roles drain fast).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, DevStatus *st, int where) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    uint32_t spins = 0;
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((++spins & 63u) == 0) {
            if (*((volatile int *)&st->code) != 0) return false;
            if (globaltimer_ns() - t0 > kWaitLimitNs) {
                raise_status(st, DEV_TIMEOUT, where, 0);
                return false;
            }
        }
    }
}

// ---- TMA ----------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int32_t x,
                                            int32_t y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- tcgen05 --------------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Whole warp: allocate ncols TMEM columns, address written to *dst (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
// D(tmem) (+)= A(smem desc) * B(smem desc), kind::tf32 or kind::f16 by template.
template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}
// Arrive on an mbarrier once all previously issued tcgen05.mma of this thread complete.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
// 32 lanes x 32 columns of 32-bit TMEM data into 32 registers per thread.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%"
        "14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Small host utilities.
// ---------------------------------------------------------------------------
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

int num_sms();

// Process-unique identity of the calling thread's current CUDA context (0 if
// the driver cannot report one).  State that a context owns -- the device
// addresses of static device arrays, kernel attributes -- is keyed on it, so
// that a context created anew (after cudaDeviceReset) is set up again
// instead of being handed stale addresses or settings.
unsigned long long current_context_id();

// Runs a set-up step once per device and context: the first time it is
// asked for with a device current, and again once that device's context has
// been replaced.  The step's error is returned to every caller until it is
// retried under a new context.
struct PerContextOnce {
    std::mutex mu;
    unsigned long long ctx[64] = {};
    cudaError_t err[64] = {};
    template <class F>
    cudaError_t run(F set_up) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        const unsigned long long id = current_context_id();
        std::lock_guard<std::mutex> lk(mu);
        if (id == 0 || ctx[dev] != id) {
            err[dev] = set_up();
            ctx[dev] = id;
        }
        return err[dev];
    }
};

// ---- benchmark accounting (not part of the method) -------------------------------
// Every kernel launch of the library increments a process-wide counter; when
// timing is enabled, launches of the classes below are bracketed by CUDA
// events on their stream and their algorithmic flops/bytes are recorded.
enum ProfClass : int {
    PROF_TC_GEMM = 0, PROF_SIMT_GEMM = 1, PROF_PANEL = 2, PROF_TRSM_DIAG = 3, PROF_SPMM = 4,
    PROF_SIDDON = 5, PROF_OTHER = 6, PROF_SPMM32 = 7, PROF_TC_GEMM_BF16 = 8,
    // out-of-core host traffic (bytes = bytes copied): V blocks streamed to
    // the device, superpanel columns loaded, factored columns written back,
    // and the compute stream's stalls waiting for a streamed V block
    PROF_H2D_V = 9, PROF_H2D_COLS = 10, PROF_D2H_COLS = 11, PROF_COPY_WAIT = 12,
    // device-side operand conversions, transposes and layout copies
    PROF_COPY = 13, PROF_NCLASS = 14
};
void count_launch(int n = 1);
struct ProfScope {
    int cls;
    cudaStream_t s;
    double flops, bytes;
    int slot;
    ProfScope(int cls, cudaStream_t s, double flops, double bytes, int64_t d0 = 0, int64_t d1 = 0,
              int64_t d2 = 0, int64_t d3 = 0);
    ~ProfScope();
};

// Device scratch buffer owned by the library (grown on demand, never
// shrunk).  With guard bands on (ct_debug_canaries), a buffer allocated
// gets kGuardBytes of the byte kGuardByte past its capacity; every live
// buffer is registered so that ct_debug_check_canaries can verify them.
constexpr size_t kGuardBytes = (size_t)64 << 10;
constexpr unsigned char kGuardByte = 0xA5;
// 32 FP32 values rounded to BF16 (nearest) and stored as four 16-byte
// words at dst (16-byte aligned): one row of a row-major BF16 copy.
__device__ __forceinline__ void store_bf16_row32(void *dst, const float (&x)[32]) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(x[8 * q + 2 * h], x[8 * q + 2 * h + 1]);
            w[h] = *reinterpret_cast<const uint32_t *>(&p);
        }
        d[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
    uint64_t gen = 0;      // bumped whenever the buffer moves (captured graphs key on it)
    bool guarded = false;  // a guard band follows the capacity
    ct_status ensure(size_t need);
    Scratch();
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch();
};

}  // namespace ctqr
