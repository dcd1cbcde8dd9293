// gemm_tc.cu -- tensor-core GEMM for the WY trailing update and the Q^T
// application (the dense contractions of the hot path), on sm_103a tcgen05.
//
// C = alpha * op(A) * op(B) + beta * C, column-major FP32 storage, TF32
// operands (the tensor core reads the FP32 bit pattern and uses its TF32
// part), FP32 accumulation in tensor memory.
//
// CTA tile 128 x 256 x 32 (UMMA M=128, N=256, K=8 per instruction, four
// instructions per 32-deep stage).  Warp roles: warp 0 issues TMA loads of
// 128B-swizzled tiles into a 4-stage shared-memory ring; warp 1 allocates
// 256 TMEM columns and one of its threads issues the MMAs; warps 2-5 read the
// accumulator back with tcgen05.ld and write C.
//
// Operand layouts: op(A) = A^T of a column-major A is "K-major" (each output
// row's K values contiguous).  TF32 operands must be K-major (the transposed,
// MN-major operand form yields zeros for 32-bit types on this hardware, as a
// layout probe showed), so the dispatcher hands this kernel K-major operands
// only ('T','N' in column-major terms), transposing the other forms first.
// A K-major tile is one TMA box of 32 x rows: 128-byte rows, 8-row swizzle
// atoms 1024 B apart.
//
// Every mbarrier wait is bounded (4 s); on expiry the kernel records
// DEV_TIMEOUT in the device status word, drains and returns.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace ctqr {

namespace {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 4;
constexpr int A_BYTES = BM * BK * 4;  // 16 KiB
constexpr int B_BYTES = BN * BK * 4;  // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int THREADS = 192;

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

// Descriptor of the kk-th K=8 slice of a K-major stage tile: the slice starts
// kk*32 bytes into each 128-byte row; 8-row swizzle atoms are 1024 B apart.
__device__ __forceinline__ uint64_t slice_desc(uint32_t tile, int kk) {
    return make_desc(tile + kk * 32, 16, 1024);
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_tf32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     int64_t M, int64_t N, int64_t K, int64_t kchunk,
                     float alpha, float beta, float *C, int64_t ldc, int64_t split_stride,
                     DevStatus *st) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accum = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = min(K, kb + kchunk);
    const int nk = (int)((ke - kb + BK - 1) / BK);
    C += (int64_t)blockIdx.z * split_stride;

    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int issued = 0;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, st, 1)) break;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            uint8_t *sa = smem + s * STAGE_BYTES;
            uint8_t *sb = sa + A_BYTES;
            const int32_t k = (int32_t)(kb + (int64_t)kt * BK);
            tma_load_2d(sa, &tmA, k, (int32_t)m0, &full[s]);
            tma_load_2d(sb, &tmB, k, (int32_t)n0, &full[s]);
            issued = kt + 1;
        }
        // Drain: every issued copy must have landed before the CTA may exit.
        for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
            mbar_wait(&full[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, st, 2);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = (1u << 4)                       // D = F32
                               | (2u << 7) | (2u << 10)        // A, B = TF32
                               /* bits 15/16 = 0: both operands K-major */
                               | ((uint32_t)(BN >> 3) << 17)   // N
                               | ((uint32_t)(BM >> 4) << 24);  // M
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % STAGES;
            const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph, st, 3)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                tc_mma<0>(tmem_d, slice_desc(sa, kk), slice_desc(sb, kk), idesc,
                          (kt > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&empty[s]);
        }
        tc_commit(accum);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const bool ok = mbar_wait(accum, 0, st, 4);
        tc_fence_after();
        const int q = warp % 4;
        const int64_t row = m0 + 32 * q + lane;
        if (ok && nk > 0) {
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_d + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * 32), r);
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t col = n0 + c * 32 + j;
                        if (col < N) {
                            float *p = C + row + col * ldc;
                            float v = alpha * __uint_as_float(r[j]);
                            if (beta != 0.0f) v += beta * *p;
                            *p = v;
                        }
                    }
                }
            }
        } else if (ok && row < M) {
            for (int64_t col = n0; col < min(N, n0 + BN); ++col) {
                float *p = C + row + col * ldc;
                *p = (beta != 0.0f) ? beta * *p : 0.0f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_d, TMEM_COLS);
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

// 2-D FP32 tensor map over a column-major rows x cols matrix (ld elements),
// box = box_rows (contiguous dim) x box_cols, 128-byte swizzle.
ct_status make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld,
                   uint32_t box_rows, uint32_t box_cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return CT_ERR_CUDA;
    }
    if (((uintptr_t)base & 15) || ((ld * 4) & 15)) {
        set_error("TMA operand not 16-byte aligned (base %p, ld %lld)", base, (long long)ld);
        return CT_ERR_ARG;
    }
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {box_rows, box_cols};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) rows=%lld cols=%lld ld=%lld", (int)r,
                  (long long)rows, (long long)cols, (long long)ld);
        return CT_ERR_CUDA;
    }
    return CT_OK;
}

}  // namespace

ct_status gemm_tc_launch(const GemmArgs &g, int splits, int64_t kchunk, int64_t split_stride,
                         cudaStream_t s) {
    if (g.kind != GEMM_TF32) {
        set_error("BF16 tensor-core GEMM not available in this build");
        return CT_ERR_UNSUPPORTED;
    }
    static bool attr_set = false;
    if (!attr_set) {
        CT_CUDA(cudaFuncSetAttribute(gemm_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_BYTES));
        attr_set = true;
    }
    if (!g.ta || g.tb) {
        set_error("tensor-core GEMM takes K-major operands only");
        return CT_ERR_ARG;
    }
    CUtensorMap ma, mb;
    // op(A) = A^T, A stored K x M (K contiguous): box {32 (K), 128 (M)}.
    CT_TRY(make_map(&ma, g.A, g.K, g.M, g.lda, BK, BM));
    // op(B) = B, B stored K x N (K contiguous): box {32 (K), 256 (N)}.
    CT_TRY(make_map(&mb, g.B, g.K, g.N, g.ldb, BK, BN));
    dim3 grid((unsigned)ceil_div(g.M, BM), (unsigned)ceil_div(g.N, BN), (unsigned)splits);
    gemm_tf32_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(
        ma, mb, g.M, g.N, g.K, kchunk, (float)g.alpha, (float)g.beta,
        (float *)g.C, g.ldc, split_stride, device_status());
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ctqr
