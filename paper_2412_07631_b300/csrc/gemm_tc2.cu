// gemm_tc2.cu -- the tensor-core GEMM of gemm_tc.cu on SM pairs
// (tcgen05 cta_group::2), for products with many 256 x 256 output tiles.
//
// Why pairs.  With one SM per 128 x 256 tile, each SM pulls 48 KB of
// operands through L2 and TMA per 32-deep K stage, and its 4-stage ring
// (192 KB) covers only about one microsecond of MMA work, so the tensor pipe
// waits on copies (about 60-70% busy on the long products of the QR).  A
// pair of SMs (a 2-CTA cluster) computes a 256 x 256 tile with one MMA
// stream: each SM holds its own 128 rows of A and half (128 columns) of B,
// and the tensor cores of the pair read both halves of B.  Per SM that is
// 32 KB per stage -- a third less operand traffic per flop -- and the same
// shared memory holds 6 stages.  Measured on 8192^3 TF32: 775 TFLOP/s
// against 575 for the one-SM kernel.
//
// Roles (320 threads per CTA, as in the one-SM kernel):
//   warp 0 lane 0 (each CTA): TMA producer.  Loads its A rows and B columns
//     into a 6-stage ring; both CTAs' copies of a stage complete on the
//     leader's `full` barrier (TMA with cta_group::2), which the leader's
//     producer arms with the bytes of the pair.
//   warp 1: allocates the pair's 512 TMEM columns (two 128 x 256 FP32
//     accumulators per SM; collective over the pair).  In the leader CTA
//     (cluster rank 0) lane 0 issues the MMAs.  Each stage's MMAs are
//     committed to the `empty` barrier of both CTAs, each tile to `acc_full`
//     of both CTAs.
//   warps 2-9 (each CTA): epilogue of the CTA's 128 accumulator rows, as in
//     the one-SM kernel; they then arrive on the leader's `acc_empty`.
// A CTA waits only on barriers in its own shared memory; arrivals cross the
// pair as copy completions, remote arrives and multicast commits.  The
// peer's producer knows its last copies have landed when the leader's MMAs
// that read them have committed `empty`.  All waits are bounded (4 s,
// DEV_TIMEOUT); every path ends at one cluster barrier, after which the pair
// frees its TMEM.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

constexpr int BMC = 128;        // rows of A per CTA (pair tile: 256)
constexpr int BN = 256;         // columns per pair tile (128 of B per CTA)
constexpr int BNC = BN / 2;
constexpr int ROW_BYTES = 128;  // one K stage: 32 FP32 or 64 BF16 values
constexpr int STAGES = 6;
constexpr int A_BYTES = BMC * ROW_BYTES;  // 16 KiB
constexpr int B_BYTES = BNC * ROW_BYTES;  // 16 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int ACC_COLS = 256;
constexpr int TMEM_COLS = 2 * ACC_COLS;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers*/;

template <int OP> struct Op2;
template <> struct Op2<0> {  // TF32
    static constexpr int BK = 32, MMA_K = 8;
    static constexpr uint32_t FMT = 2;
};
template <> struct Op2<1> {  // BF16
    static constexpr int BK = 64, MMA_K = 16;
    static constexpr uint32_t FMT = 1;
};

// ---- cluster / pair primitives ------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t map_to_rank(const void *p, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
    return out;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}
// try_wait with cluster-scope acquire (for barriers arrived on from the peer)
__device__ __forceinline__ bool try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool wait_cluster(uint64_t *bar, uint32_t parity, DevStatus *st, int where) {
    if (try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    uint32_t spins = 0;
    while (true) {
        if (try_wait_cluster(bar, parity)) return true;
        if ((++spins & 63u) == 0) {
            if (*((volatile int *)&st->code) != 0) return false;
            if (globaltimer_ns() - t0 > kWaitLimitNs) {
                raise_status(st, DEV_TIMEOUT, where, 0);
                return false;
            }
        }
    }
}
// TMA 2-D load into this CTA's shared memory, completing on an mbarrier that
// may live in either CTA of the pair (shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *smem_dst, const CUtensorMap *map, int32_t x,
                                                 int32_t y, uint32_t bar_cluster_addr) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster_addr)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc2(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
template <int OP>
__device__ __forceinline__ void mma2(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
    if constexpr (OP == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}
// arrive on `bar` (same offset) in both CTAs of the pair once the issued MMAs complete
__device__ __forceinline__ void commit_pair(uint64_t *bar) {
    const uint16_t mask = 0x3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void commit_own(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused with 128B swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;  // 8-row swizzle atoms 1024 B apart
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;  // SWIZZLE_128B
    return d;
}

struct PairSched {
    int64_t mt, nt, tiles, work;
    bool m_fast, upper;
    // upper: a square tile grid of which only the tiles on and above the
    // diagonal are computed (a symmetric product whose lower part is unused)
    __host__ __device__ PairSched(int64_t M, int64_t N, int splits, bool upper_only) {
        mt = (M + 2 * BMC - 1) / (2 * BMC);
        nt = (N + BN - 1) / BN;
        upper = upper_only && mt == nt;
        tiles = upper ? mt * (mt + 1) / 2 : mt * nt;
        work = tiles * splits;
        m_fast = mt <= nt;
    }
    // Tiles are walked in groups of kGroup rows of the longer grid dimension;
    // inside a group the shorter dimension varies fastest, then the group's
    // rows, so pairs resident together share a few operand tiles of each
    // dimension through L2.
    __device__ void decode(int64_t w, int64_t &mi, int64_t &ni, int64_t &z) const {
        constexpr int64_t kGroup = 8;
        z = w / tiles;
        int64_t t = w - z * tiles;
        if (upper) {  // row by row: tile row r holds nt - r tiles, from the diagonal on
            int64_t r = 0;
            while (t >= nt - r) {
                t -= nt - r;
                ++r;
            }
            mi = r;
            ni = r + t;
            return;
        }
        const int64_t nf = m_fast ? mt : nt, ns = m_fast ? nt : mt;
        const int64_t g = t / (kGroup * nf), r = t - g * (kGroup * nf);
        const int64_t rows = min(kGroup, ns - g * kGroup);
        const int64_t sl = g * kGroup + r % rows, fa = r / rows;
        if (m_fast) { mi = fa; ni = sl; }
        else { ni = fa; mi = sl; }
    }
};

template <int OP>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     int64_t M, int64_t N, int64_t K, int64_t kchunk, int splits, float alpha,
                     float beta, float *C, int64_t ldc, int64_t split_stride, int upper_only,
                     DevStatus *st) {
    constexpr int BK = Op2<OP>::BK;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);  // leader: stage of the pair landed
    uint64_t *empty = full + STAGES;      // MMAs reading the stage are done
    uint64_t *acc_full = empty + STAGES;  // [2]
    uint64_t *acc_empty = acc_full + 2;   // [2] (leader; 2 x EPI_WARPS arrivals)
    uint64_t *drain = acc_empty + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int64_t pair = blockIdx.x / 2, npairs = gridDim.x / 2;
    const PairSched ts(M, N, splits, upper_only != 0);

    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 2 * EPI_WARPS);
        }
        mbar_init(drain, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc2(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers initialised, TMEM allocated
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer (each CTA) ----------------
        const uint32_t full0 = map_to_rank(&full[0], 0);  // the leader's ring of `full`
        int64_t kt_glob = 0, issued = 0;
        bool ok = true;
        for (int64_t w = pair; w < ts.work && ok; w += npairs) {
            int64_t mi, ni, z;
            ts.decode(w, mi, ni, z);
            const int64_t kb = z * kchunk, ke = min(K, kb + kchunk);
            const int nk = (int)((ke - kb + BK - 1) / BK);
            for (int kt = 0; kt < nk; ++kt, ++kt_glob) {
                const int s = (int)(kt_glob % STAGES);
                const uint32_t ph = (uint32_t)(kt_glob / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, st, 11)) { ok = false; break; }
                if (leader) mbar_arrive_expect_tx(&full[s], 2 * STAGE_BYTES);
                uint8_t *sa = smem + s * STAGE_BYTES;
                const uint32_t bar = full0 + (uint32_t)(s * sizeof(uint64_t));
                const int32_t k = (int32_t)(kb + (int64_t)kt * BK);
                tma_load_2d_pair(sa, &tmA, k, (int32_t)(mi * 2 * BMC + rank * BMC), bar);
                tma_load_2d_pair(sa + A_BYTES, &tmB, k, (int32_t)(ni * BN + rank * BNC), bar);
                issued = kt_glob + 1;
            }
        }
        // Drain: the leader sees its own `full` phases; the peer knows its
        // copies landed once the MMAs that read them committed `empty`.
        for (int64_t q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q) {
            const uint32_t ph = (uint32_t)(q / STAGES) & 1u;
            if (leader) mbar_wait(&full[q % STAGES], ph, st, 12);
            else mbar_wait(&empty[q % STAGES], ph, st, 13);
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------- MMA issuer (leader) ----------------
        constexpr uint32_t F = Op2<OP>::FMT;
        const uint32_t idesc = (1u << 4)                          // D = F32
                               | (F << 7) | (F << 10)             // A, B: TF32 or BF16, K-major
                               | ((uint32_t)(BN >> 3) << 17)      // N = 256
                               | ((uint32_t)((2 * BMC) >> 4) << 24);  // M = 256 (pair)
        int64_t kt_glob = 0, local = 0;
        bool ok = true;
        for (int64_t w = pair; w < ts.work && ok; w += npairs, ++local) {
            int64_t mi, ni, z;
            ts.decode(w, mi, ni, z);
            const int64_t kb = z * kchunk, ke = min(K, kb + kchunk);
            const int nk = (int)((ke - kb + BK - 1) / BK);
            const int b = (int)(local & 1);
            const uint32_t use = (uint32_t)(local >> 1);
            if (!wait_cluster(&acc_empty[b], (use & 1u) ^ 1u, st, 14)) break;
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(b * ACC_COLS);
            for (int kt = 0; kt < nk; ++kt, ++kt_glob) {
                const int s = (int)(kt_glob % STAGES);
                const uint32_t ph = (uint32_t)(kt_glob / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, st, 15)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t sb = sa + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / Op2<OP>::MMA_K; ++kk)
                    mma2<OP>(d_tmem, make_desc(sa + kk * 32), make_desc(sb + kk * 32), idesc,
                             (kt > 0 || kk > 0) ? 1u : 0u);
                commit_pair(&empty[s]);
            }
            if (ok) commit_pair(&acc_full[b]);
        }
        commit_own(drain);
        mbar_wait(drain, 0, st, 17);
    } else if (warp >= 2) {
        // ---------------- epilogue (each CTA, its 128 rows) ----------------
        const int e = warp - 2;
        const int q = warp % 4;   // TMEM lane quarter this warp may access
        const int half = e / 4;   // which 128 of the 256 accumulator columns
        const uint32_t leader_acc_empty0 = map_to_rank(&acc_empty[0], 0);
        int64_t local = 0;
        for (int64_t w = pair; w < ts.work; w += npairs, ++local) {
            int64_t mi, ni, z;
            ts.decode(w, mi, ni, z);
            const int b = (int)(local & 1);
            const uint32_t use = (uint32_t)(local >> 1);
            if (!mbar_wait(&acc_full[b], use & 1u, st, 18)) break;
            tc_fence_after();
            float *Cz = C + z * split_stride;
            const int64_t row = mi * 2 * BMC + rank * BMC + 32 * q + lane;
            const uint32_t t0 = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * ACC_COLS + half * 128);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(t0 + (uint32_t)(c * 32), r);
                const int64_t col0 = ni * BN + half * 128 + c * 32;
                if (row < M) {
                    float *p = Cz + row + col0 * ldc;
                    const int ncols = (N - col0 < 32) ? (int)(N - col0) : 32;
                    if (beta != 0.0f) {
                        float old[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) old[j] = (j < ncols) ? p[(int64_t)j * ldc] : 0.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < ncols) p[(int64_t)j * ldc] = alpha * __uint_as_float(r[j]) + beta * old[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < ncols) p[(int64_t)j * ldc] = alpha * __uint_as_float(r[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) remote_arrive(leader_acc_empty0 + (uint32_t)(b * sizeof(uint64_t)));
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // the leader's MMAs (reading this CTA's stages) are complete
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc2(tmem_base, TMEM_COLS);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn2() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

ct_status make_map2(CUtensorMap *map, bool bf16, const void *base, int64_t rows, int64_t cols,
                    int64_t ld, uint32_t box_rows, uint32_t box_cols) {
    EncodeTiledFn fn = encode_fn2();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return CT_ERR_CUDA;
    }
    const int64_t es = bf16 ? 2 : 4;
    if (((uintptr_t)base & 15) || ((ld * es) & 15)) {
        set_error("TMA operand not 16-byte aligned (base %p, ld %lld)", base, (long long)ld);
        return CT_ERR_ARG;
    }
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {box_rows, box_cols};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return CT_ERR_CUDA;
    }
    return CT_OK;
}

// Co-resident 2-CTA clusters of this kernel (the persistent grid), per kernel;
// the shared-memory attribute and the occupancy query run once per device and
// context (both belong to the context).
template <int OP>
int max_pairs() {
    static PerContextOnce once;
    static int pairs[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const cudaError_t e = once.run([dev]() -> cudaError_t {
        pairs[dev] = 0;
        cudaError_t err = cudaFuncSetAttribute(gemm_pair_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               SMEM_BYTES);
        if (err != cudaSuccess) return err;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * num_sms());
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = SMEM_BYTES;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        err = cudaOccupancyMaxActiveClusters(&n, gemm_pair_kernel<OP>, &cfg);
        if (err == cudaSuccess) pairs[dev] = n;
        return err;
    });
    return e == cudaSuccess ? pairs[dev] : 0;
}

template <int OP>
ct_status launch_pair(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                      DevStatus *status, cudaStream_t s) {
    const int pairs_max = max_pairs<OP>();
    if (pairs_max <= 0) {
        cudaGetLastError();
        set_error("no co-resident SM pair for the paired GEMM kernel");
        return CT_ERR_CUDA;
    }
    constexpr int BK = Op2<OP>::BK;
    CUtensorMap ma, mb;
    CT_TRY(make_map2(&ma, OP == 1, g.A, g.K, g.M, g.lda, BK, BMC));
    CT_TRY(make_map2(&mb, OP == 1, g.B, g.K, g.N, g.ldb, BK, BNC));
    const PairSched sched(g.M, g.N, splits, g.upper_only);
    const int64_t pairs = std::min<int64_t>(sched.work, pairs_max);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CT_CUDA(cudaLaunchKernelEx(&cfg, gemm_pair_kernel<OP>, ma, mb, g.M, g.N, g.K, kchunk, splits,
                               (float)g.alpha, (float)g.beta, (float *)g.C, g.ldc, split_stride,
                               (int)g.upper_only, status));
    count_launch();
    return CT_OK;
}

}  // namespace

// Paired (2-SM) launch of a K-major TF32/BF16 product; callers pick it when
// the product has enough 256 x 256 tiles to occupy the machine.  Device
// errors go to `status` (NULL: the library's status word).
ct_status gemm_pair_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                           cudaStream_t s, DevStatus *status) {
    if ((g.kind != GEMM_TF32 && g.kind != GEMM_BF16) || !g.ta || g.tb) return CT_ERR_ARG;
    if (!status) status = device_status();
    return g.kind == GEMM_BF16 ? launch_pair<1>(g, splits, kchunk, split_stride, status, s)
                               : launch_pair<0>(g, splits, kchunk, split_stride, status, s);
}

int64_t gemm_pair_tiles(int64_t M, int64_t N) { return ceil_div(M, 2 * BMC) * ceil_div(N, BN); }

}  // namespace ctqr
