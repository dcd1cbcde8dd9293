// gemm_noalloc.cu -- ct_gemm_noalloc: the library's GEMM engine for callers
// that cannot allocate device memory.
//
// ct_gemm (and every GEMM inside the factorisation) keeps two kinds of
// scratch in device memory the library allocates on demand: the partial
// products of a split-K launch, summed afterwards in a fixed order, and the
// K-major copies of operands the tensor cores cannot read in place.  Some
// callers cannot let a library call cudaMalloc: code that has handed all
// device memory to its own pool or arena, and code running under a rule of
// no runtime allocation (cudaMalloc can fail under memory pressure and
// synchronises the device).  This entry point serves them: the same kernels,
// with the scratch in one file-scope device array of fixed size, so the call
// allocates nothing.
//
// The array (kScratchBytes) and a status word live in this module's static
// device memory: every GPU that loads the library holds them until the
// process exits.  Host code cannot pass the array's name to a kernel (in host
// code it is a host-side stand-in, not a device address), so the first call
// on each device -- with that device current -- looks up the device addresses
// with cudaGetSymbolAddress and keeps them for that device's context (a
// context created anew, after cudaDeviceReset, is looked up again).
//
// Accepted kinds: 0 (FP64), 1 (FP32) and 2 (TF32); the BF16 and split
// products (kinds 3-5) need operand copies as large as the operands and are
// refused.  Split-K follows the allocating engine's plan, with the depth
// reduced until the partial products fit in the room the copies leave.
//
// All calls share the array and keep the last call's contents; calls that
// overlap on the GPU (two streams, two threads) race on it.  The status word
// is cleared at the start of each call; the partial-product area is fully
// overwritten by each split-K launch before it is read, so it needs no
// clearing.  Each call waits for its stream before returning, to read the
// status word back.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) DevStatus g_status;

struct NoAllocPtrs {
    unsigned char *scratch = nullptr;
    DevStatus *status = nullptr;
};

ct_status noalloc_setup(NoAllocPtrs *out) {
    static NoAllocPtrs per_dev[64];
    static PerContextOnce once;
    int dev = 0;
    CT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CT_ERR_ARG;
    CT_CUDA(once.run([dev]() -> cudaError_t {
        void *p = nullptr, *q = nullptr;
        per_dev[dev] = NoAllocPtrs{};
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_status);
        if (e == cudaSuccess) per_dev[dev] = NoAllocPtrs{(unsigned char *)p, (DevStatus *)q};
        return e;
    }));
    *out = per_dev[dev];
    return CT_OK;
}

ct_status too_big(size_t need) {
    set_error("ct_gemm_noalloc: this product needs %zu bytes of scratch, the fixed limit is %zu",
              need, kScratchBytes);
    return CT_ERR_ARG;
}

}  // namespace

}  // namespace ctqr

using namespace ctqr;

extern "C" ct_status ct_gemm_noalloc(int32_t kind, char transa, char transb, int64_t M, int64_t N,
                                     int64_t K, double alpha, const void *A, int64_t lda,
                                     const void *B, int64_t ldb, double beta, void *C,
                                     int64_t ldc, void *stream) {
    if (kind < 0 || kind > 2) return CT_ERR_ARG;
    const bool ta = transa == 'T' || transa == 't';
    const bool tb = transb == 'T' || transb == 't';
    if ((!ta && transa != 'N' && transa != 'n') || (!tb && transb != 'N' && transb != 'n'))
        return CT_ERR_ARG;
    if (M < 0 || N < 0 || K < 0) return CT_ERR_ARG;
    if (ldc < std::max<int64_t>(1, M)) return CT_ERR_ARG;
    if (lda < std::max<int64_t>(1, ta ? K : M) || ldb < std::max<int64_t>(1, tb ? N : K))
        return CT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocPtrs P;
    CT_TRY(noalloc_setup(&P));
    CT_CUDA(cudaMemsetAsync(P.status, 0, sizeof(DevStatus), s));
    if (M == 0 || N == 0) return CT_OK;

    GemmArgs g{(GemmKind)kind, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc};
    const bool fp64 = g.kind == GEMM_F64;
    const size_t es = fp64 ? 8 : 4;
    if (g.kind == GEMM_TF32 &&
        (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15) || (g.lda & 3) || (g.ldb & 3)))
        g.kind = GEMM_F32;  // tiles must start on 16-byte boundaries; CUDA cores otherwise
    const bool tc = g.kind == GEMM_TF32;
    size_t used = 0;
    if (K == 0) {
        if (g.beta != 1.0) CT_TRY(splitk_reduce(fp64, M, N, 0, nullptr, 0.0, g.beta, C, ldc, s));
    } else {
        if (tc && (!g.ta || g.tb)) {
            // K-major copies of operands stored the other way round, in the array
            const int64_t ldt = round_up(K, 32);
            const size_t abytes = !g.ta ? (size_t)round_up(4 * ldt * M, 256) : 0;
            const size_t bbytes = g.tb ? (size_t)round_up(4 * ldt * N, 256) : 0;
            if (abytes + bbytes > kScratchBytes) return too_big(abytes + bbytes);
            if (!g.ta) {
                CT_TRY(transpose_any(0, g.A, g.lda, 0, P.scratch, ldt, M, K, s));
                g.A = P.scratch;
                g.lda = ldt;
                g.ta = true;
            }
            if (g.tb) {
                CT_TRY(transpose_any(0, g.B, g.ldb, 0, P.scratch + abytes, ldt, N, K, s));
                g.B = P.scratch + abytes;
                g.ldb = ldt;
                g.tb = false;
            }
            used = abytes + bbytes;
        }
        // split-K as planned by the allocating engine, then made shallower
        // until the partial products fit in the room left in the array
        const int64_t BM = tc ? 128 : (fp64 ? 64 : 128);
        const int64_t BN = tc ? 256 : (fp64 ? 64 : 128);
        const int64_t align = tc ? 32 : 16;
        int64_t splits, kchunk;
        plan_splits(ceil_div(M, BM) * ceil_div(N, BN), K, tc ? 256 : 128, align, &splits, &kchunk);
        const size_t room = kScratchBytes - used;
        if (splits > 1 && es * (size_t)(M * N * splits) > room) {
            splits = std::max<int64_t>(1, (int64_t)(room / (es * (size_t)(M * N))));
            kchunk = round_up(ceil_div(K, splits), align);
            splits = ceil_div(K, kchunk);
        }
        if (splits <= 1) {
            CT_TRY(tc ? gemm_tc_launch_status(g, 1, K, 0, P.status, s)
                      : gemm_simt_launch(g, 1, K, 0, s));
        } else {
            void *part = P.scratch + used;
            GemmArgs p = g;
            p.alpha = 1.0;
            p.beta = 0.0;
            p.C = part;
            p.ldc = M;
            CT_TRY(tc ? gemm_tc_launch_status(p, (int)splits, kchunk, M * N, P.status, s)
                      : gemm_simt_launch(p, (int)splits, kchunk, M * N, s));
            CT_TRY(splitk_reduce(fp64, M, N, (int)splits, part, g.alpha, g.beta, C, ldc, s));
        }
    }
    DevStatus h{};
    CT_CUDA(cudaMemcpyAsync(&h, P.status, sizeof(h), cudaMemcpyDeviceToHost, s));
    CT_CUDA(cudaStreamSynchronize(s));
    if (h.code == DEV_OK) return CT_OK;
    set_error("ct_gemm_noalloc: device status %d at site %d", h.code, h.where);
    return h.code == DEV_TIMEOUT ? CT_ERR_TIMEOUT : CT_ERR_CUDA;
}
