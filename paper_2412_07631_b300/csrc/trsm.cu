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
#include "kernels.cuh"

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
    static bool attr = false;
    if (!attr) {
        CT_CUDA(cudaFuncSetAttribute(diag_solve_kernel<T, BS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    diag_solve_kernel<T, BS><<<(unsigned)ceil_div(k, KC), KC, smem, s>>>(trans, ni, R, ldr, C, ldc, k);
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

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
