// gemm_tc.cu -- tensor-core GEMM for the WY trailing update and the Q^T
// application (the dense contractions of the hot path), on sm_103a tcgen05.
//
// C = alpha * op(A) * op(B) + beta * C, column-major FP32 C, FP32
// accumulation in tensor memory.  Two operand forms:
//   TF32: operands are FP32 in memory; the tensor core reads the FP32 bit
//         pattern and uses its TF32 part (kind::tf32, K = 8 per MMA).
//   BF16: operands are bfloat16 copies made by the dispatcher (kind::f16
//         with BF16 inputs, K = 16 per MMA).
// Either way one shared-memory stage row is 128 bytes of K (32 FP32 or 64
// BF16 values), so the swizzled tile layout, the descriptors and the TMA
// boxes are the same bytes; only the element count per row differs.
//
// Operand layouts: op(A) = A^T of a column-major A is "K-major" (each output
// row's K values contiguous).  Operands must be K-major (the transposed,
// MN-major operand form yields zeros for 32-bit types on this hardware, as a
// layout probe showed), so the dispatcher hands this kernel K-major operands
// only ('T','N' in column-major terms), transposing the other forms first.
// A K-major tile is one TMA box of 128 B x rows: 8-row swizzle atoms 1024 B
// apart.
//
// Persistent kernel: one CTA per SM walks the output tiles (128 x 256, K in
// 128-byte stages) of its share of the work list.  Warp 0 issues TMA loads
// into a 4-stage shared-memory ring; warp 1 allocates 512 TMEM columns (two
// 128 x 256 FP32 accumulators) and one of its threads issues the MMAs (UMMA
// M=128, N=256, or N = the tile's columns inside C rounded up to 16 for a
// narrow last tile, so a product of 32-224 columns, such as a panel's V^T C,
// does not pay for 256); warps 2-9 drain an accumulator with tcgen05.ld and write C
// while the MMAs of the next tile fill the other accumulator.  The tile order
// puts the grid dimension with fewer tiles fastest, so CTAs resident at the
// same time share the operand tile of the longer dimension through L2.
//
// Epilogue forms.  With beta = 0 (a plain product or a split-K partial) the
// scaled accumulator is staged in shared memory and written by TMA tensor
// stores.  With beta = 1 and a short K (the rank-32 panel updates, bound by
// the C traffic) it is staged the same way and added to C by TMA reduce-add
// stores, so C is read and written by the copy engine and the L2.
// fl(c + alpha*acc) is the same rounding either way.  Other cases, or a C
// that is not 16-byte aligned, use the thread epilogue (C loaded, scaled and
// stored by threads): for deep products it measured faster than the staged
// forms, whose shared-memory traffic competes with the MMA operand reads.
// Each epilogue warp owns two 32 x 16 staging buffers and reuses one only
// after the copy engine has finished reading it.
//
// Every mbarrier wait is bounded (4 s); on expiry the kernel records
// DEV_TIMEOUT in the device status word, drains and returns.
#include <algorithm>
#include <mutex>

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

constexpr int BM = 128, BN = 256, ROW_BYTES = 128, STAGES = 4;
constexpr int A_BYTES = BM * ROW_BYTES;  // 16 KiB
constexpr int B_BYTES = BN * ROW_BYTES;  // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int ACC_COLS = 256;
constexpr int TMEM_COLS = 2 * ACC_COLS;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
// epilogue staging: per warp two 32-row x 16-column FP32 boxes
constexpr int STG_ROWS = 32, STG_COLS = 16;
constexpr int STG_FLOATS = STG_ROWS * STG_COLS;
constexpr int STG_BYTES = EPI_WARPS * 2 * STG_FLOATS * 4;  // 32 KiB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STG_BYTES + 1024 /*align*/ + 256 /*barriers*/;

// K elements per 128-byte stage row and per MMA, by operand form.
template <int OP> struct OpTraits;
template <> struct OpTraits<0> {  // TF32
    static constexpr int BK = 32, MMA_K = 8;
    static constexpr uint32_t FMT = 2;
};
template <> struct OpTraits<1> {  // BF16
    static constexpr int BK = 64, MMA_K = 16;
    static constexpr uint32_t FMT = 1;
};

enum EpiMode : int { EPI_THREADS = 0, EPI_TMA_STORE = 1, EPI_TMA_ADD = 2 };


// ---- TMA stores from shared memory (bulk async-groups of the issuing thread) ----
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int32_t x,
                                             int32_t y, int32_t z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void tma_add_3d(const CUtensorMap *map, const void *src, int32_t x,
                                           int32_t y, int32_t z) {
    asm volatile(
        "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one committed group of this thread still reading shared memory
__device__ __forceinline__ void bulk_wait_read_1() {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading/stride
// byte offsets (16-byte units), version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;  // SWIZZLE_128B
    return d;
}

// Descriptor of the kk-th MMA slice of a K-major stage tile (8 TF32 or 16
// BF16 values = 32 bytes): the slice starts kk*32 bytes into each 128-byte
// row; 8-row swizzle atoms are 1024 B apart.
__device__ __forceinline__ uint64_t slice_desc(uint32_t tile, int kk) {
    return make_desc(tile + kk * 32, 16, 1024);
}

struct TileSched {
    int64_t mt, nt, tiles, work;
    bool m_fast;
    __device__ TileSched(int64_t M, int64_t N, int splits) {
        mt = (M + BM - 1) / BM;
        nt = (N + BN - 1) / BN;
        tiles = mt * nt;
        work = tiles * splits;
        m_fast = mt <= nt;
    }
    // work item w -> (m tile, n tile, split)
    // Tiles are walked in groups of kGroup rows of the longer grid dimension;
    // inside a group the shorter dimension varies fastest, then the group's
    // rows.  CTAs resident together then share a few operand tiles of each
    // dimension, so neither operand is streamed from DRAM once per row of
    // the other when it does not fit L2 (the short-K trailing updates).
    __device__ void decode(int64_t w, int64_t &mi, int64_t &ni, int64_t &z) const {
        constexpr int64_t kGroup = 8;
        z = w / tiles;
        const int64_t t = w - z * tiles;
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
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, int epi,
                   int64_t M, int64_t N, int64_t K, int64_t kchunk, int splits,
                   float alpha, float beta, float *C, int64_t ldc, int64_t split_stride,
                   DevStatus *st) {
    constexpr int BK = OpTraits<OP>::BK;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *stage_out = (float *)(smem + STAGES * STAGE_BYTES);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES + STG_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;   // [2] MMA -> epilogue
    uint64_t *acc_empty = acc_full + 2;    // [2] epilogue -> MMA
    uint64_t *drain = acc_empty + 2;       // MMA completion before TMEM release
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const TileSched ts(M, N, splits);

    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        if (epi != EPI_THREADS) tma_prefetch_desc(&tmC);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
        mbar_init(drain, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int64_t kt_glob = 0, issued = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < ts.work && ok; w += gridDim.x) {
            int64_t mi, ni, z;
            ts.decode(w, mi, ni, z);
            const int64_t kb = z * kchunk, ke = min(K, kb + kchunk);
            const int nk = (int)((ke - kb + BK - 1) / BK);
            for (int kt = 0; kt < nk; ++kt, ++kt_glob) {
                const int s = (int)(kt_glob % STAGES);
                const uint32_t ph = (uint32_t)(kt_glob / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, st, 1)) { ok = false; break; }
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                uint8_t *sa = smem + s * STAGE_BYTES;
                const int32_t k = (int32_t)(kb + (int64_t)kt * BK);
                tma_load_2d(sa, &tmA, k, (int32_t)(mi * BM), &full[s]);
                tma_load_2d(sa + A_BYTES, &tmB, k, (int32_t)(ni * BN), &full[s]);
                issued = kt_glob + 1;
            }
        }
        // Drain: every issued copy must have landed before the CTA may exit.
        for (int64_t q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q)
            mbar_wait(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, st, 2);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t F = OpTraits<OP>::FMT;
        const uint32_t idesc0 = (1u << 4)                       // D = F32
                                | (F << 7) | (F << 10)          // A, B = TF32 or BF16, K-major
                                | ((uint32_t)(BM >> 4) << 24);  // M
        int64_t kt_glob = 0, local = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < ts.work && ok; w += gridDim.x, ++local) {
            int64_t mi, ni, z;
            ts.decode(w, mi, ni, z);
            const int64_t kb = z * kchunk, ke = min(K, kb + kchunk);
            const int nk = (int)((ke - kb + BK - 1) / BK);
            // MMA width: the tile's columns inside C, rounded up to 16 (M = 128
            // takes N = 16 .. 256 in steps of 16); B's rows beyond N are the
            // copy engine's zero fill, and the epilogue stores no column >= N
            const int64_t nvalid = min((int64_t)BN, N - ni * BN);
            const uint32_t idesc = idesc0 | ((uint32_t)(((nvalid + 15) / 16 * 16) >> 3) << 17);
            const int b = (int)(local & 1);
            const uint32_t use = (uint32_t)(local >> 1);
            if (!mbar_wait(&acc_empty[b], (use & 1u) ^ 1u, st, 5)) break;
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(b * ACC_COLS);
            for (int kt = 0; kt < nk; ++kt, ++kt_glob) {
                const int s = (int)(kt_glob % STAGES);
                const uint32_t ph = (uint32_t)(kt_glob / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, st, 3)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t sb = sa + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / OpTraits<OP>::MMA_K; ++kk)
                    tc_mma<OP>(d_tmem, slice_desc(sa, kk), slice_desc(sb, kk), idesc,
                              (kt > 0 || kk > 0) ? 1u : 0u);
                tc_commit(&empty[s]);
            }
            tc_commit(&acc_full[b]);
        }
        // all issued MMAs must complete before TMEM is released
        tc_commit(drain);
        mbar_wait(drain, 0, st, 6);
    } else if (warp >= 2) {
        // ---------------- epilogue (8 warps) ----------------
        const int e = warp - 2;
        const int q = warp % 4;            // TMEM lane quarter this warp may access
        const int half = e / 4;            // which 128 of the 256 accumulator columns
        int64_t local = 0;
        uint32_t nbox = 0;                 // staged boxes issued by this warp
        for (int64_t w = blockIdx.x; w < ts.work; w += gridDim.x, ++local) {
            int64_t mi, ni, z;
            ts.decode(w, mi, ni, z);
            const int b = (int)(local & 1);
            const uint32_t use = (uint32_t)(local >> 1);
            if (!mbar_wait(&acc_full[b], use & 1u, st, 4)) break;
            tc_fence_after();
            const int64_t row = mi * BM + 32 * q + lane;
            float *Cz = C + z * split_stride;
            const uint32_t t0 = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * ACC_COLS + half * 128);
            if (epi != EPI_THREADS) {
                // stage 32 x 16 boxes in shared memory; the copy engine stores or adds them
                float *stg = stage_out + e * 2 * STG_FLOATS;
                const int64_t row0 = mi * BM + 32 * q;
                // buffers alternate by boxes issued, so the one group that
                // wait_group.read 1 may leave in flight is the other buffer's
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(t0 + (uint32_t)(c * 32), r);
#pragma unroll
                    for (int hc = 0; hc < 2; ++hc) {
                        const int64_t col0 = ni * BN + half * 128 + c * 32 + hc * STG_COLS;
                        if (row0 >= M || col0 >= N) continue;  // box wholly outside C
                        float *buf = stg + (nbox++ & 1) * STG_FLOATS;
                        if (lane == 0) bulk_wait_read_1();
                        __syncwarp();
#pragma unroll
                        for (int j = 0; j < STG_COLS; ++j)
                            buf[j * STG_ROWS + lane] = alpha * __uint_as_float(r[hc * STG_COLS + j]);
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            if (epi == EPI_TMA_ADD) tma_add_3d(&tmC, buf, (int32_t)row0, (int32_t)col0, (int32_t)z);
                            else tma_store_3d(&tmC, buf, (int32_t)row0, (int32_t)col0, (int32_t)z);
                            bulk_commit();
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
                continue;
            }
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
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        // the staged boxes must be written out (and their buffers read) before exit
        if (epi != EPI_THREADS && lane == 0) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---- host: tensor maps ---------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

// 2-D tensor map over a column-major rows x cols matrix (ld elements) of
// FP32 or BF16, box = box_rows (contiguous dim) x box_cols, 128-byte swizzle.
ct_status make_map(CUtensorMap *map, bool bf16, const void *base, int64_t rows, int64_t cols,
                   int64_t ld, uint32_t box_rows, uint32_t box_cols) {
    EncodeTiledFn fn = encode_fn();
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
        set_error("cuTensorMapEncodeTiled failed (%d) rows=%lld cols=%lld ld=%lld", (int)r,
                  (long long)rows, (long long)cols, (long long)ld);
        return CT_ERR_CUDA;
    }
    return CT_OK;
}

// 3-D FP32 map over C (M x N, ld ldc) and its split-K copies (split_stride
// apart), box 32 x 16 x 1 unswizzled: the epilogue's staging layout.
ct_status make_map_c(CUtensorMap *map, const void *C, int64_t M, int64_t N, int64_t ldc,
                     int splits, int64_t split_stride) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return CT_ERR_CUDA;
    }
    const int64_t s2 = splits > 1 ? split_stride : round_up(ldc * N, 4);
    cuuint64_t dims[3] = {(cuuint64_t)M, (cuuint64_t)N, (cuuint64_t)std::max(splits, 1)};
    cuuint64_t strides[2] = {(cuuint64_t)(ldc * 4), (cuuint64_t)(s2 * 4)};
    cuuint32_t box[3] = {STG_ROWS, STG_COLS, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(C), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (C) failed (%d)", (int)r);
        return CT_ERR_CUDA;
    }
    return CT_OK;
}

constexpr int64_t kTmaAddMaxK = 64;

// Epilogue form for this call (see the file comment).
int pick_epilogue(const GemmArgs &g, int splits, int64_t split_stride) {
    const bool aligned = ((uintptr_t)g.C & 15) == 0 && (g.ldc & 3) == 0 &&
                         (splits <= 1 || (split_stride & 3) == 0) && g.M < (1LL << 31) &&
                         g.N < (1LL << 31);
    if (!aligned) return EPI_THREADS;
    if (g.beta == 0.0) return EPI_TMA_STORE;
    // Reduce-add pays for short products (rank-32 panel updates), where C
    // traffic dominates; for deep ones the thread epilogue measured faster.
    if (g.beta == 1.0 && splits <= 1 && g.K <= kTmaAddMaxK) return EPI_TMA_ADD;
    return EPI_THREADS;
}

template <int OP>
ct_status launch_tc(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                    DevStatus *status, cudaStream_t s) {
    static PerContextOnce once;  // the attribute belongs to each device's context
    CT_CUDA(once.run([] {
        return cudaFuncSetAttribute(gemm_tc_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SMEM_BYTES);
    }));
    constexpr int BK = OpTraits<OP>::BK;
    CUtensorMap ma, mb, mc;
    // op(A) = A^T, A stored K x M (K contiguous): box {BK (K), 128 (M)}.
    CT_TRY(make_map(&ma, OP == 1, g.A, g.K, g.M, g.lda, BK, BM));
    // op(B) = B, B stored K x N (K contiguous): box {BK (K), 256 (N)}.
    CT_TRY(make_map(&mb, OP == 1, g.B, g.K, g.N, g.ldb, BK, BN));
    const int epi = pick_epilogue(g, splits, split_stride);
    if (epi != EPI_THREADS) CT_TRY(make_map_c(&mc, g.C, g.M, g.N, g.ldc, splits, split_stride));
    else memset(&mc, 0, sizeof(mc));
    const int64_t work = ceil_div(g.M, BM) * ceil_div(g.N, BN) * splits;
    dim3 grid((unsigned)std::min<int64_t>(work, num_sms()));
    gemm_tc_kernel<OP><<<grid, THREADS, SMEM_BYTES, s>>>(
        ma, mb, mc, epi, g.M, g.N, g.K, kchunk, splits, (float)g.alpha, (float)g.beta,
        (float *)g.C, g.ldc, split_stride, status);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

// K-major operands only: TF32 (FP32 in memory) or BF16 copies.
ct_status gemm_tc_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                         cudaStream_t s) {
    if (g.kind != GEMM_TF32 && g.kind != GEMM_BF16) return CT_ERR_ARG;
    if (!g.ta || g.tb) {
        set_error("tensor-core GEMM takes K-major operands only");
        return CT_ERR_ARG;
    }
    const double ebytes = g.kind == GEMM_BF16 ? 2.0 : 4.0;
    ProfScope prof(g.kind == GEMM_BF16 ? PROF_TC_GEMM_BF16 : PROF_TC_GEMM, s, 2.0 * g.M * g.N * g.K,
                   ebytes * ((double)g.M * g.K + (double)g.K * g.N) +
                       4.0 * (double)g.M * g.N * splits * (g.beta != 0.0 ? 2 : 1),
                   g.M, g.N, g.K, splits);
    // Deep products with enough 256 x 256 tiles to occupy the SM pairs run on
    // the paired kernel (gemm_tc2.cu); short rank updates keep the one-SM
    // kernel and its TMA epilogues.
    if (g.K > kTmaAddMaxK && gemm_pair_tiles(g.M, g.N) * splits >= num_sms() / 2)
        return gemm_pair_launch(g, splits, kchunk, split_stride, s);
    return g.kind == GEMM_BF16 ? launch_tc<1>(g, splits, kchunk, split_stride, device_status(), s)
                               : launch_tc<0>(g, splits, kchunk, split_stride, device_status(), s);
}

// Same kernels and tile choice as gemm_tc_launch (TF32), with the status word
// given by the caller and no accounting scope; used by the allocation-free
// entry point.
ct_status gemm_tc_launch_status(const GemmArgs &g, int splits, int64_t kchunk,
                                int64_t split_stride, DevStatus *status, cudaStream_t s) {
    if (g.kind != GEMM_TF32 || !g.ta || g.tb) return CT_ERR_ARG;
    if (g.K > kTmaAddMaxK && gemm_pair_tiles(g.M, g.N) * splits >= num_sms() / 2)
        return gemm_pair_launch(g, splits, kchunk, split_stride, s, status);
    return launch_tc<0>(g, splits, kchunk, split_stride, status, s);
}

}  // namespace ctqr
