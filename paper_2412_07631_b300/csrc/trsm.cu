// trsm.cu -- R X = C (back-substitution, Sec. 2 Eq. 3 'X = R^-1 C';
// Sec. 2.1 'dtrsm') and R^T X = C (forward substitution, for the adjoint).
//
// Blocked as in the paper's out-of-core task list for R X = C (Sec. 2.2):
// solve the last diagonal block R_ii X_i = C_i, subtract its contribution
// C_{0:i} -= R_{0:i,i} X_i with a GEMM, move up.  The diagonal blocks are
// solved by a SIMT kernel (one thread per right-hand side, R_ii and the C
// block staged in shared memory); the updates run on the GEMM engine of the
// path's precision (tensor cores for the TF32 path).
#include <algorithm>

#include "common.cuh"
#include "handles.cuh"
#include "kernels.cuh"
#include "simt_tile.cuh"

namespace ctqr {

namespace {

constexpr int KC = 128;  // right-hand sides per CTA

template <typename T, int BS>
__global__ void __launch_bounds__(KC) diag_solve_kernel(bool trans, int ni, const T *R, int64_t ldr,
                                                        T *C, int64_t ldc, int64_t k) {
    extern __shared__ __align__(16) uint8_t dsm[];
    T *Rs = (T *)dsm;              // [BS][BS] column-major
    T *Cs = Rs + BS * BS;          // [BS][KC+1], row r at Cs[r*(KC+1)]
    const int64_t s0 = (int64_t)blockIdx.x * KC;
    const int kc = (int)((k - s0 < KC) ? (k - s0) : KC);
    for (int idx = threadIdx.x; idx < ni * ni; idx += KC) {
        int r = idx % ni, c = idx / ni;
        Rs[r + c * BS] = R[r + c * ldr];
    }
    for (int idx = threadIdx.x; idx < ni * kc; idx += KC) {
        int r = idx % ni, s = idx / ni;
        Cs[r * (KC + 1) + s] = C[r + (s0 + s) * ldc];
    }
    __syncthreads();
    const int s = threadIdx.x;
    if (s < kc) {
        if (!trans) {
            for (int l = ni - 1; l >= 0; --l) {
                T xl = Cs[l * (KC + 1) + s] / Rs[l + l * BS];
                Cs[l * (KC + 1) + s] = xl;
                for (int r = 0; r < l; ++r) Cs[r * (KC + 1) + s] -= Rs[r + l * BS] * xl;
            }
        } else {
            for (int l = 0; l < ni; ++l) {
                T acc = Cs[l * (KC + 1) + s];
                for (int r = 0; r < l; ++r) acc -= Rs[r + l * BS] * Cs[r * (KC + 1) + s];
                Cs[l * (KC + 1) + s] = acc / Rs[l + l * BS];
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ni * kc; idx += KC) {
        int r = idx % ni, s2 = idx / ni;
        C[r + (s0 + s2) * ldc] = Cs[r * (KC + 1) + s2];
    }
}

template <typename T, int BS>
ct_status diag_solve(bool trans, int ni, const T *R, int64_t ldr, T *C, int64_t ldc, int64_t k,
                     cudaStream_t s) {
    const size_t smem = sizeof(T) * ((size_t)BS * BS + (size_t)BS * (KC + 1));
    static PerContextOnce attr;
    CT_CUDA(attr.run([&] {
        return cudaFuncSetAttribute(diag_solve_kernel<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    }));
    ProfScope prof(PROF_TRSM_DIAG, s, (double)ni * ni * k, sizeof(T) * ((double)ni * ni + 2.0 * ni * k));
    diag_solve_kernel<T, BS><<<(unsigned)ceil_div(k, KC), KC, smem, s>>>(trans, ni, R, ldr, C, ldc, k);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// One CTA per diagonal block b: Rinv_b = R_bb^-1 (TB x TB, zero-padded past
// the ragged last block), by back-substitution of the identity columns, one
// thread per column; also writes the transpose.
template <typename T, int TB>
__global__ void __launch_bounds__(TB) diag_inverse_kernel(int64_t n, const T *R, int64_t ldr,
                                                          T *Rinv, T *RinvT) {
    extern __shared__ __align__(16) uint8_t dsm[];
    T *Rs = (T *)dsm;         // [TB][TB] column-major
    T *Xs = Rs + TB * TB;     // [TB][TB+1], row r at Xs[r*(TB+1)]
    const int64_t i0 = (int64_t)blockIdx.x * TB;
    const int ni = (int)((n - i0 < TB) ? (n - i0) : TB);
    const T *Rb = R + i0 + i0 * ldr;
    for (int idx = threadIdx.x; idx < TB * TB; idx += TB) {
        int r = idx % TB, c = idx / TB;
        Rs[r + c * TB] = (r < ni && c < ni) ? Rb[r + c * ldr] : T(0);
        Xs[r * (TB + 1) + c] = (r == c && r < ni) ? T(1) : T(0);
    }
    __syncthreads();
    const int s = threadIdx.x;
    if (s < ni) {
        for (int l = ni - 1; l >= 0; --l) {
            T xl = Xs[l * (TB + 1) + s] / Rs[l + l * TB];
            Xs[l * (TB + 1) + s] = xl;
            for (int r = 0; r < l; ++r) Xs[r * (TB + 1) + s] -= Rs[r + l * TB] * xl;
        }
    }
    __syncthreads();
    T *Ib = Rinv + (size_t)blockIdx.x * TB * TB;
    T *It = RinvT + (size_t)blockIdx.x * TB * TB;
    for (int idx = threadIdx.x; idx < TB * TB; idx += TB) {
        int r = idx % TB, c = idx / TB;
        Ib[r + c * TB] = Xs[r * (TB + 1) + c];
        It[c + r * TB] = Xs[r * (TB + 1) + c];
    }
}

template <typename T, int TB>
ct_status diag_inverse_launch(int64_t n, const T *R, int64_t ldr, T *Rinv, T *RinvT, cudaStream_t s) {
    const size_t smem = sizeof(T) * ((size_t)TB * TB + (size_t)TB * (TB + 1));
    static PerContextOnce attr;
    CT_CUDA(attr.run([&] {
        return cudaFuncSetAttribute(diag_inverse_kernel<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    }));
    diag_inverse_kernel<T, TB><<<(unsigned)ceil_div(n, TB), TB, smem, s>>>(n, R, ldr, Rinv, RinvT);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

// Copy the TB x TB inverse blocks onto the diagonals of the SB x SB superblock
// inverses (zero elsewhere): block b at superblock (b*TB)/SB, local offset.
template <typename T>
__global__ void scatter_diag_kernel(int64_t nblk, int TB, int SB, const T *Rinv, T *RinvB) {
    const int64_t b = blockIdx.x;
    const int64_t g0 = b * TB;
    const int64_t sb = g0 / SB, loc = g0 - sb * SB;
    const T *src = Rinv + (size_t)b * TB * TB;
    T *dst = RinvB + (size_t)sb * SB * SB + loc + loc * SB;
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int r = idx % TB, c = idx / TB;
        if (loc + r < SB && loc + c < SB) dst[r + (int64_t)c * SB] = src[r + c * TB];
    }
}

// One doubling level of the superblock inverses, for every superblock and
// every pair of b x b diagonal blocks at once (blockIdx.z = superblock t x
// pairs_per_sb + pair i).  The pair starting at local row p of superblock t
// holds inv(A) and inv(C) on the diagonal of RinvB_t already; with the
// coupling block R12 = R[p:p+b, p+b:p+b+bb] of R,
//   stage 1:  Y = R12 inv(C)                        (b x bb, scratch of the pair)
//   stage 2:  inv block (p, p+b) of RinvB_t = -inv(A) Y.
// inv(C) and inv(A) are upper triangular, so the k range of a tile stops at
// the tile's last column (stage 1) or starts at its first row (stage 2): the
// terms left out are exact zeros.
template <int STAGE>
__global__ void __launch_bounds__(256) inv_double_kernel(int64_t n, int64_t SB, int64_t b,
                                                         int64_t pairs_per_sb, const float *R,
                                                         int64_t ldr, float *RinvB, float *Y) {
    constexpr int BT = 128;
    const int64_t z = blockIdx.z;
    const int64_t t = z / pairs_per_sb, i = z - t * pairs_per_sb;
    const int64_t s0 = t * SB, s1 = min(n, s0 + SB);
    const int64_t pl = 2 * b * i, p = s0 + pl;
    if (p + b >= s1) return;
    const int64_t bb = min(b, s1 - p - b);
    const int64_t m0 = (int64_t)blockIdx.x * BT, n0 = (int64_t)blockIdx.y * BT;
    if (m0 >= b || n0 >= bb) return;
    float *inv = RinvB + t * SB * SB;
    float *Yz = Y + z * b * b;  // ld b
    if (STAGE == 1)
        simt_tile<float, BT, BT, 8, 8, 8>(false, false, b, bb, 0, min(bb, n0 + BT), 1.0f,
                                           R + p + (p + b) * ldr, ldr, inv + (pl + b) + (pl + b) * SB, SB,
                                           0.0f, Yz, b, m0, n0);
    else
        simt_tile<float, BT, BT, 8, 8, 8>(false, false, b, bb, m0, b, -1.0f, inv + pl + pl * SB, SB, Yz, b,
                                           0.0f, inv + pl + (pl + b) * SB, SB, m0, n0);
}

}  // namespace

// Tensor-core path: inverses of the SB x SB diagonal superblocks of R, by
// doubling from the TB x TB inverses,
//   inv([A B; 0 C]) = [inv(A), -inv(A) B inv(C); 0, inv(C)]
// (exact transposes of each other are kept for R^-1 and R^-T, so the two
// applications stay adjoint).  The narrow levels (blocks below kInvTensorB)
// run on the FP32 CUDA cores, two launches per level covering every
// superblock and every block pair of it (inv_double_kernel), so the grid
// fills the machine where one product is a single tile; the wide levels,
// which hold most of the flops, run on the tensor-core GEMM engine in split
// TF32 (TF32x3), two products per block pair.
constexpr int64_t kInvTensorB = 512;

static ct_status build_superblock_inverses(ct_factor f, cudaStream_t s) {
    const int TB = f->trsm_tb;
    const int64_t n = f->n;
    const int SB = (int)std::min<int64_t>(f->solve_sb_req > 0 ? f->solve_sb_req : 2048, round_up(n, TB));
    const int64_t nsb = ceil_div(n, SB), nblk = ceil_div(n, TB);
    const size_t es = f->es(), blk = (size_t)SB * SB;
    CT_CUDA(cudaMalloc(&f->RinvB, es * nsb * blk));
    CT_CUDA(cudaMalloc(&f->RinvTB, es * nsb * blk));
    CT_CUDA(cudaMemsetAsync(f->RinvB, 0, es * nsb * blk, s));
    scatter_diag_kernel<float><<<(unsigned)nblk, 256, 0, s>>>(nblk, TB, SB, (const float *)f->Rinv,
                                                              (float *)f->RinvB);
    count_launch();
    CT_CUDA(cudaGetLastError());
    // scratch Y: one b x b block per pair of a level (pairs of a superblock:
    // ceil(SB / 2b), the last one possibly ragged or empty)
    int64_t ymax = 1;
    for (int64_t b = TB; b < SB; b *= 2)
        ymax = std::max(ymax, b >= kInvTensorB ? b * b : nsb * ceil_div(SB, 2 * b) * b * b);
    Scratch ys;
    CT_TRY(ys.ensure(sizeof(float) * (size_t)ymax));
    for (int64_t b = TB; b < SB; b *= 2) {
        const int64_t pairs = ceil_div(SB, 2 * b);
        if (b >= kInvTensorB) {
            // the wide levels (most of the flops) as two products per pair on
            // the tensor-core engine, split TF32 (TF32x3: near-FP32 accuracy);
            // the zero halves of the triangular factors are multiplied too
            for (int64_t t = 0; t < nsb; ++t) {
                const int64_t s0 = t * SB, len = std::min<int64_t>(n - s0, SB);
                char *inv = (char *)f->RinvB + es * t * blk;
                for (int64_t i = 0; i < pairs; ++i) {
                    const int64_t pl = 2 * b * i;
                    if (pl + b >= len) continue;
                    const int64_t bb = std::min<int64_t>(b, len - pl - b);
                    GemmArgs g1{GEMM_TF32X3, false, false, b, bb, bb, 1.0,
                                (const char *)f->Rm + es * ((s0 + pl) + (s0 + pl + b) * f->ldr), f->ldr,
                                inv + es * ((pl + b) + (pl + b) * SB), SB, 0.0, ys.ptr, b};
                    CT_TRY(gemm(g1, f->trsm_ws, s));
                    GemmArgs g2{GEMM_TF32X3, false, false, b, bb, b, -1.0, inv + es * (pl + pl * SB), SB, ys.ptr, b,
                                0.0, inv + es * (pl + (pl + b) * SB), SB};
                    CT_TRY(gemm(g2, f->trsm_ws, s));
                }
            }
            continue;
        }
        const int64_t tiles = ceil_div(b, 128);
        dim3 grid((unsigned)tiles, (unsigned)tiles, (unsigned)(nsb * pairs));
        const double fl = 2.0 * (double)nsb * pairs * b * b * b;  // both stages, triangular halves
        ProfScope prof(PROF_SIMT_GEMM, s, fl, 4.0 * 4.0 * (double)nsb * pairs * b * b, b, b, b, nsb * pairs);
        inv_double_kernel<1><<<grid, 256, 0, s>>>(n, SB, b, pairs, (const float *)f->Rm, f->ldr,
                                                   (float *)f->RinvB, (float *)ys.ptr);
        count_launch();
        inv_double_kernel<2><<<grid, 256, 0, s>>>(n, SB, b, pairs, (const float *)f->Rm, f->ldr,
                                                   (float *)f->RinvB, (float *)ys.ptr);
        count_launch();
        CT_CUDA(cudaGetLastError());
    }
    for (int64_t t = 0; t < nsb; ++t)
        CT_TRY(transpose_any(0, (char *)f->RinvB + es * t * blk, SB, 0, (char *)f->RinvTB + es * t * blk, SB,
                             SB, SB, s));
    // the scratch goes away with this call: its last readers must be done
    CT_CUDA(cudaStreamSynchronize(s));
    f->trsm_sb = SB;
    return CT_OK;
}

// Inverse diagonal blocks of R (and, for the tensor-core path, R^T and the
// superblock inverses), built once per factor on first use.
ct_status trsm_prepare(ct_factor f, cudaStream_t s) {
    if (f->Rinv) {
        // superblock inverses dropped by a change of the solve plan: rebuilt
        if (tensor_kind(f->kind) && f->trsm_sb == 0) CT_TRY(build_superblock_inverses(f, s));
        return CT_OK;
    }
    const size_t es = f->es();
    const int TB = f->fp64 ? 64 : 128;
    const int64_t nbt = ceil_div(f->n, TB);
    CT_CUDA(cudaMalloc(&f->Rinv, es * (size_t)nbt * TB * TB));
    CT_CUDA(cudaMalloc(&f->RinvT, es * (size_t)nbt * TB * TB));
    f->trsm_tb = TB;
    if (f->fp64)
        CT_TRY((diag_inverse_launch<double, 64>(f->n, (const double *)f->Rm, f->ldr,
                                                (double *)f->Rinv, (double *)f->RinvT, s)));
    else
        CT_TRY((diag_inverse_launch<float, 128>(f->n, (const float *)f->Rm, f->ldr,
                                                (float *)f->Rinv, (float *)f->RinvT, s)));
    if (tensor_kind(f->kind)) {
        f->ldrt = round_up(f->n, 32);
        CT_CUDA(cudaMalloc(&f->Rt, es * (size_t)f->ldrt * f->n));
        CT_TRY(transpose_any(0, f->Rm, f->ldr, 0, f->Rt, f->ldrt, f->n, f->n, s));
        CT_TRY(build_superblock_inverses(f, s));
    }
    return CT_OK;
}

// R X = C (trans = false) or R^T X = C (trans = true) in place, C: n x k (ldc).
// Superblocks of SB = 4 TB rows, taken from the last (back-substitution) or
// the first (forward substitution).  Inside a superblock, block by block:
//   X_i = R_ii^-1 C_i  (GEMM with the stored inverse block),
//   the rest of the superblock -= its coupling block times X_i;
// then once per superblock the off-diagonal update of everything beyond it,
//   C_{0:s0} -= R_{0:s0, s0:s1} X_s   or   C_{s1:n} -= R_{s0:s1, s1:n}^T X_s,
// a GEMM with K = SB.  Every product is an op(A) = A^T GEMM on the
// tensor-core path (R^T supplies the non-transposed couplings).
ct_status trsm_factor(ct_factor f, bool trans, void *C, int64_t ldc, int64_t k, cudaStream_t s) {
    const int64_t n = f->n;
    if (n == 0 || k == 0) return CT_OK;
    CT_TRY(trsm_prepare(f, s));
    const size_t es = f->es();
    const int TB = f->trsm_tb;
    const int64_t SB = 4 * (int64_t)TB;
    const int64_t nblk = ceil_div(n, TB);
    const int64_t nsb = ceil_div(n, SB);
    CT_TRY(f->misc2.ensure(es * (size_t)TB * k));
    void *tmp = f->misc2.ptr;
    const bool tc = tensor_kind(f->kind);
    auto Cp = [&](int64_t i) { return (char *)C + es * i; };
    // C[r0:r0+rows] -= R[r0:r0+rows, c0:c0+cols] X   with X = C[c0:c0+cols]   (back)
    // C[r0:r0+rows] -= R[c0:c0+cols, r0:r0+rows]^T X with X = C[c0:c0+cols]   (forward)
    auto couple = [&](int64_t r0, int64_t rows, int64_t c0, int64_t cols) -> ct_status {
        if (rows <= 0 || cols <= 0) return CT_OK;
        GemmArgs g{};
        g.kind = f->kind;
        g.min_chunk = f->solve_chunk;
        g.alpha = -1.0;
        g.beta = 1.0;
        g.M = rows;
        g.N = k;
        g.K = cols;
        g.B = Cp(c0);
        g.ldb = ldc;
        g.C = Cp(r0);
        g.ldc = ldc;
        if (!trans) {
            if (tc) {  // R[r0:, c0:] = (Rt[c0:c0+cols, r0:r0+rows])^T
                g.ta = true;
                g.A = (char *)f->Rt + es * (size_t)(c0 + r0 * f->ldrt);
                g.lda = f->ldrt;
            } else {
                g.ta = false;
                g.A = (char *)f->Rm + es * (size_t)(r0 + c0 * f->ldr);
                g.lda = f->ldr;
            }
        } else {
            g.ta = true;
            g.A = (char *)f->Rm + es * (size_t)(c0 + r0 * f->ldr);
            g.lda = f->ldr;
        }
        return gemm(g, f->trsm_ws, s);
    };
    if (f->trsm_sb > 0) {
        // one GEMM per superblock with its stored inverse, then the coupling
        const int64_t BS = f->trsm_sb, nbs = ceil_div(n, BS);
        CT_TRY(f->misc2.ensure(es * (size_t)BS * k));
        void *tmpB = f->misc2.ptr;
        for (int64_t t = 0; t < nbs; ++t) {
            const int64_t sbi = trans ? t : nbs - 1 - t;
            const int64_t s0 = sbi * BS, s1 = std::min<int64_t>(n, s0 + BS), ns = s1 - s0;
            CT_CUDA(cudaMemcpy2DAsync(tmpB, es * BS, Cp(s0), es * ldc, es * ns, k,
                                      cudaMemcpyDeviceToDevice, s));
            GemmArgs d{};
            d.kind = f->kind;
            d.min_chunk = f->solve_chunk;
            d.M = ns;
            d.N = k;
            d.K = ns;
            d.alpha = 1.0;
            d.beta = 0.0;
            d.B = tmpB;
            d.ldb = BS;
            d.C = Cp(s0);
            d.ldc = ldc;
            d.lda = BS;
            d.tb = false;
            // op(A) = inv(R_ss) = (RinvTB_s)^T, or inv(R_ss)^T = (RinvB_s)^T
            d.ta = true;
            d.A = (char *)(trans ? f->RinvB : f->RinvTB) + es * (size_t)sbi * BS * BS;
            CT_TRY(gemm(d, f->trsm_ws, s));
            if (!trans) CT_TRY(couple(0, s0, s0, ns));
            else CT_TRY(couple(s1, n - s1, s0, ns));
        }
        return CT_OK;
    }
    for (int64_t t = 0; t < nsb; ++t) {
        const int64_t sbi = trans ? t : nsb - 1 - t;
        const int64_t s0 = sbi * SB, s1 = std::min<int64_t>(n, s0 + SB);
        const int64_t b_lo = s0 / TB, b_hi = ceil_div(s1, TB);  // base blocks [b_lo, b_hi)
        for (int64_t u = 0; u < b_hi - b_lo; ++u) {
            const int64_t ib = trans ? b_lo + u : b_hi - 1 - u;
            const int64_t i0 = ib * TB;
            const int ni = (int)std::min<int64_t>(TB, n - i0);
            CT_CUDA(cudaMemcpy2DAsync(tmp, es * TB, Cp(i0), es * ldc, es * ni, k,
                                      cudaMemcpyDeviceToDevice, s));
            GemmArgs d{};
            d.kind = f->kind;
            d.M = ni;
            d.N = k;
            d.K = ni;
            d.alpha = 1.0;
            d.beta = 0.0;
            d.B = tmp;
            d.ldb = TB;
            d.C = Cp(i0);
            d.ldc = ldc;
            d.lda = TB;
            d.tb = false;
            // op(A) = R_ii^-1 = (RinvT_i)^T, or R_ii^-T = (Rinv_i)^T
            d.ta = true;
            d.A = (char *)(trans ? f->Rinv : f->RinvT) + es * (size_t)ib * TB * TB;
            CT_TRY(gemm(d, f->trsm_ws, s));
            if (!trans) CT_TRY(couple(s0, i0 - s0, i0, ni));                 // rows above, in the superblock
            else CT_TRY(couple(i0 + ni, s1 - (i0 + ni), i0, ni));          // rows below, in the superblock
        }
        if (!trans) CT_TRY(couple(0, s0, s0, s1 - s0));
        else CT_TRY(couple(s1, n - s1, s0, s1 - s0));
    }
    return CT_OK;
}

ct_status trsm_upper(GemmKind kind, bool trans, int64_t n, int64_t k, const void *R, int64_t ldr,
                     void *C, int64_t ldc, Scratch &ws, cudaStream_t s) {
    if (n == 0 || k == 0) return CT_OK;
    const bool fp64 = kind == GEMM_F64;
    const int BS = fp64 ? 64 : 128;
    const size_t es = fp64 ? 8 : 4;
    const int64_t nblk = ceil_div(n, BS);
    auto Rp = [&](int64_t i, int64_t j) { return (const char *)R + es * (i + j * ldr); };
    auto Cp = [&](int64_t i) { return (char *)C + es * i; };
    for (int64_t t = 0; t < nblk; ++t) {
        const int64_t ib = trans ? t : nblk - 1 - t;
        const int64_t i0 = ib * BS;
        const int ni = (int)std::min<int64_t>(BS, n - i0);
        if (fp64)
            CT_TRY((diag_solve<double, 64>(trans, ni, (const double *)Rp(i0, i0), ldr,
                                           (double *)Cp(i0), ldc, k, s)));
        else
            CT_TRY((diag_solve<float, 128>(trans, ni, (const float *)Rp(i0, i0), ldr,
                                           (float *)Cp(i0), ldc, k, s)));
        GemmArgs g{};
        g.kind = kind;
        g.alpha = -1.0;
        g.beta = 1.0;
        g.N = k;
        g.K = ni;
        g.ldb = ldc;
        g.ldc = ldc;
        g.lda = ldr;
        g.B = Cp(i0);
        if (!trans) {
            if (i0 == 0) continue;
            g.ta = false;
            g.tb = false;
            g.M = i0;
            g.A = Rp(0, i0);
            g.C = Cp(0);
        } else {
            if (i0 + ni >= n) continue;
            g.ta = true;
            g.tb = false;
            g.M = n - i0 - ni;
            g.A = Rp(i0, i0 + ni);
            g.C = Cp(i0 + ni);
        }
        CT_TRY(gemm(g, ws, s));
    }
    return CT_OK;
}

}  // namespace ctqr
