// qr.cu -- blocked Householder QR driver (Sec. 2 Eq. 2; 'dgeqrf' of Sec. 2.1)
// and the block-reflector application used by the solve (Eq. 3, 'dormqr').
//
// Two-level right-looking blocking.  Outer blocks of NB columns; inside a
// block, panels of nb columns are factored by the cooperative panel kernel
// and applied to the rest of the block with their own compact-WY factors.
// When a block is finished its T_J (larft from the Gram matrix V_J^T V_J) and
// the unit-lower top of V_J are kept, and the trailing matrix is updated
//      C <- (I - V_J T_J V_J^T)^T C = C - V_J (T_J^T (V_J^T C))
// with three GEMMs (two of them large, on the precision's GEMM engine).
// V_J lives in place below the diagonal of A; only its NB x NB top triangle
// (ones on the diagonal, R above it in A) is copied out, so the GEMMs split
// V_J into that small top block and the in-place rows below it.  With the
// regularisation rows sqrt(lambda) I below A, the reflectors of block J have
// no support below row m + j + w (row_end), so the panels, the Gram matrices
// and both trailing-update GEMMs stop there: the skipped terms are exact
// zeros, and on average a fifth of the rows drop out at 256x256.
#include <algorithm>

#include "diskstore.cuh"
#include "handles.cuh"

namespace ctqr {

namespace {

inline char *at(void *base, int64_t i, int64_t j, int64_t ld, size_t es) {
    return (char *)base + es * (size_t)(i + j * ld);
}

GemmArgs mk(ct_factor f, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
            const void *A, int64_t lda, const void *B, int64_t ldb, double beta, void *C,
            int64_t ldc) {
    GemmArgs g;
    g.kind = f->kind;
    g.ta = ta;
    g.tb = tb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.alpha = alpha;
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.beta = beta;
    g.C = C;
    g.ldc = ldc;
    g.min_chunk = f->solve_chunk;  // 0 during the factorisation
    return g;
}

// G = V^T V of the block reflector at column j (w columns).  Its users (the
// T recurrences and assemblies) read G on and above the diagonal only, so
// the deep product below the top block may leave tiles strictly below the
// diagonal undefined.
ct_status gram(ct_factor f, int64_t j, int w, const void *Vt, void *G, cudaStream_t s) {
    const int64_t NB = f->NB;
    CT_TRY(gemm(mk(f, true, false, w, w, w, 1.0, Vt, NB, Vt, NB, 0.0, G, NB), f->gemm_ws, s));
    const int64_t kb = f->row_end(j + w) - j - w;
    if (kb > 0) {
        const void *Vb = at(f->VR, j + w, j, f->lda, f->es());
        GemmArgs g = mk(f, true, false, w, w, kb, 1.0, Vb, f->lda, Vb, f->lda, 1.0, G, NB);
        g.upper_only = true;
        CT_TRY(gemm(g, f->gemm_ws, s));
    }
    return CT_OK;
}

// The top-block part of a narrow (w <= 32 columns) block reflector applied
// to ncols columns, one warp per column, lane i holding row i:
//   w  = W[:, c] + Vt^T C_top[:, c]     (W = Vb^T C_b from the rows below, or 0)
//   w2 = op(T) w,   C_top[:, c] -= Vt w2,   W2[:, c] = w2
// Vt (unit lower, explicit) and T (upper) are staged in shared memory; every
// sum runs over r in ascending order.  Replaces three tiny GEMM launches per
// panel update by one.  With splits > 0, W is the sum of the engine's
// unreduced split-K partials P (each w x ncols, ld w), added in split order
// here instead of by a reduction launch; with W2b, the BF16 rounding of W2 is
// stored as well (K-major for the BF16 product C -= V W2: element (k, c) at
// W2b[k + c * ldb16]).
template <typename T>
__global__ void __launch_bounds__(256) top_block_kernel(int w, int64_t ncols, const T *Vt, const T *Tm,
                                                        int64_t ldt, bool trans_t, const T *W, T *W2,
                                                        int64_t ldw, T *C, int64_t ldc, const T *P, int splits,
                                                        __nv_bfloat16 *W2b, int64_t ldb16) {
    __shared__ T sV[32][33], sT[32][33];
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int r = idx % 32, c = idx / 32;
        const bool in = r < w && c < w;
        sV[r][c] = in ? Vt[r + (int64_t)c * ldt] : T(0);
        // sT[r][c] = op(T)(r, c)
        sT[r][c] = in ? (trans_t ? Tm[c + (int64_t)r * ldt] : Tm[r + (int64_t)c * ldt]) : T(0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t col = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (col >= ncols) return;
    const T cv = lane < w ? C[lane + col * ldc] : T(0);
    T acc = T(0);
    if (splits > 0) {
        if (lane < w) {  // in split order, the loads eight at a time
            const int64_t wn = (int64_t)w * ncols;
            const T *p = P + lane + col * w;
            int z = 0;
            for (; z + 8 <= splits; z += 8) {
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = p[(int64_t)(z + u) * wn];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += v[u];
            }
            for (; z < splits; ++z) acc += p[(int64_t)z * wn];
        }
    } else if (lane < w) {
        acc = W[lane + col * ldw];
    }
    for (int r = 0; r < w; ++r) acc += sV[r][lane] * __shfl_sync(0xffffffffu, cv, r);  // (Vt^T C)_lane
    T w2 = T(0);
    for (int r = 0; r < w; ++r) w2 += sT[lane][r] * __shfl_sync(0xffffffffu, acc, r);   // (op(T) w)_lane
    T upd = T(0);
    for (int r = 0; r < w; ++r) upd += sV[lane][r] * __shfl_sync(0xffffffffu, w2, r);   // (Vt w2)_lane
    if (lane < w) {
        C[lane + col * ldc] = cv - upd;
        W2[lane + col * ldw] = w2;
        if (W2b != nullptr) W2b[lane + col * ldb16] = __float2bfloat16_rn((float)w2);
    }
}

template <typename T>
ct_status top_block(int w, int64_t ncols, const void *Vt, const void *Tm, int64_t ldt, bool trans_t,
                    const void *W, void *W2, int64_t ldw, void *C, int64_t ldc, cudaStream_t s,
                    const void *P = nullptr, int splits = 0, void *W2b = nullptr, int64_t ldb16 = 0) {
    const unsigned grid = (unsigned)ceil_div(ncols, 8);
    top_block_kernel<T><<<grid, 256, 0, s>>>(w, ncols, (const T *)Vt, (const T *)Tm, ldt, trans_t,
                                             (const T *)W, (T *)W2, ldw, (T *)C, ldc, (const T *)P, splits,
                                             (__nv_bfloat16 *)W2b, ldb16);
    count_launch();
    CT_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace

// C[j:M, 0:ncols] <- (I - V op(T) V^T) C, op(T) = T^T for Q^T, T for Q.
// C points at row j of the target; V is the block at column j of width w.
// `big` is the engine of the two products over the rows below the top block
// (V_b^T C_b and C_b -= V_b W2), the bulk of the flops.  V_b (rows j+w ..
// row_end(j+w) of the block) is read in place in VR, or from `vb` (ld ldvb)
// when given (a block streamed from host memory).
ct_status apply_block(ct_factor f, int64_t j, int w, const void *Vt, const void *T, bool qt,
                      void *C, int64_t ldc, int64_t ncols, cudaStream_t s, GemmKind big,
                      const void *vb, int64_t ldvb, const void *v16r_made) {
    if (ncols <= 0) return CT_OK;
    const int64_t NB = f->NB;
    const size_t es = f->es();
    CT_TRY(f->W.ensure(es * (size_t)NB * ncols));
    CT_TRY(f->W2.ensure(es * (size_t)NB * ncols));
    void *W = f->W.ptr, *W2 = f->W2.ptr;
    const int64_t kb = f->row_end(j + w) - j - w;  // rows beyond: V is zero there
    const void *Vb = vb ? vb : at(f->VR, j + w, j, f->lda, es);
    const int64_t ldV = vb ? ldvb : f->lda;
    void *Cb = (char *)C + es * (size_t)w;
    // BF16 products.  W = V^T C of a panel's or mid block's reflector (w <=
    // 256) is short and deep: it is bound by reading C, so it takes the FP32
    // C directly on the TF32 path rather than paying a BF16 copy of C first.
    // V below its top block is rounded to BF16 once, into each K-major
    // layout a BF16 product reads (V^T C takes it as stored, C -= V W2
    // transposed), instead of one conversion per product.
    GemmKind tn_kind = big;
    const void *v16c = nullptr, *v16r = nullptr;
    int64_t ld16c = 0, ld16r = 0;
    if (big == GEMM_BF16 && kb > 0 && w <= 32 && v16r_made != nullptr) {
        // the panel kernel rounded V already (row-major, the layout C -= V W2 reads)
        tn_kind = GEMM_TF32;
        ld16r = round_up(w, 64);
        v16r = v16r_made;
    } else if (big == GEMM_BF16 && kb > 0) {
        if (w <= 256) tn_kind = GEMM_TF32;
        ld16c = round_up(kb, 64);
        ld16r = round_up(w, 64);
        const size_t cb = tn_kind == GEMM_BF16 ? (size_t)round_up(2 * ld16c * w, 256) : 0;
        const size_t rb = (size_t)round_up(2 * ld16r * kb, 256);
        CT_TRY(f->V16.ensure(cb + rb));
        v16c = cb ? f->V16.ptr : nullptr;
        v16r = (char *)f->V16.ptr + cb;
        CT_TRY(convert_bf16_dual((const float *)Vb, ldV, kb, w, const_cast<void *>(v16c), ld16c,
                                 const_cast<void *>(v16r), ld16r, s));
    }
    if (w <= 32) {
        // narrow reflector (a panel's): the bulk products over the rows below
        // on the engine, the w x w top-block work fused into one small kernel
        // W = V_b^T C_b: a split-K product leaves its partials to the
        // top-block kernel, which adds them in split order
        void *P = nullptr;
        int splits = 0;
        if (kb > 0) {
            GemmArgs g = mk(f, true, false, w, ncols, kb, 1.0, Vb, ldV, Cb, ldc, 0.0, W, NB);
            g.kind = tn_kind;
            g.A16 = v16c;
            g.lda16 = ld16c;
            g.partials_out = &P;
            g.splits_out = &splits;
            CT_TRY(gemm(g, f->gemm_ws, s));
        } else {
            CT_TRY(fill_zero_2d(f->fp64, W, NB, w, ncols, s));
        }
        // BF16 product below: the top-block kernel also rounds W2 for it
        void *w2b = nullptr;
        const int64_t ldw2b = round_up(w, 64);
        if (kb > 0 && big == GEMM_BF16) {
            CT_TRY(f->W2h.ensure(2 * (size_t)ldw2b * ncols));
            w2b = f->W2h.ptr;
        }
        CT_TRY(f->fp64 ? top_block<double>(w, ncols, Vt, T, NB, qt, W, W2, NB, C, ldc, s, P, splits)
                       : top_block<float>(w, ncols, Vt, T, NB, qt, W, W2, NB, C, ldc, s, P, splits, w2b,
                                          ldw2b));
        if (kb > 0) {
            GemmArgs g = mk(f, false, false, kb, ncols, w, -1.0, Vb, ldV, W2, NB, 1.0, Cb, ldc);
            g.kind = big;
            g.A16 = v16r;
            g.lda16 = ld16r;
            if (w2b != nullptr) {
                g.B16 = w2b;
                g.ldb16 = ldw2b;
            }
            CT_TRY(gemm(g, f->gemm_ws, s));
        }
        return CT_OK;
    }
    // W = V^T C
    CT_TRY(gemm(mk(f, true, false, w, ncols, w, 1.0, Vt, NB, C, ldc, 0.0, W, NB), f->gemm_ws, s));
    if (kb > 0) {
        GemmArgs g = mk(f, true, false, w, ncols, kb, 1.0, Vb, ldV, Cb, ldc, 1.0, W, NB);
        g.kind = tn_kind;
        g.A16 = v16c;
        g.lda16 = ld16c;
        CT_TRY(gemm(g, f->gemm_ws, s));
    }
    // W2 = op(T) W
    CT_TRY(gemm(mk(f, qt, false, w, ncols, w, 1.0, T, NB, W, NB, 0.0, W2, NB), f->gemm_ws, s));
    // C -= V W2
    CT_TRY(gemm(mk(f, false, false, w, ncols, w, -1.0, Vt, NB, W2, NB, 1.0, C, ldc), f->gemm_ws, s));
    if (kb > 0) {
        GemmArgs g = mk(f, false, false, kb, ncols, w, -1.0, Vb, ldV, W2, NB, 1.0, Cb, ldc);
        g.kind = big;
        g.A16 = v16r;
        g.lda16 = ld16r;
        CT_TRY(gemm(g, f->gemm_ws, s));
    }
    return CT_OK;
}

// Factor outer blocks [J0, J1) of VR; trailing updates reach column col_end.
// (In core: all blocks, col_end = n.  Out of core: the blocks of one
// superpanel, whose columns [c0, col_end) are resident; VR is then offset so
// that global column indices address the superpanel buffer.)
// T of a block reflector of width wblk from its panels' T_p (already on the
// diagonal of T, ld NB) and its Gram matrix G = V^T V (ld NB): for the panel
// at offset o,  T[0:o, o:o+wp] = -T[0:o, 0:o] * G[0:o, o:o+wp] * T_p,  the
// off-diagonal block of the product of two block reflectors.
// `step` is the width of the diagonal blocks already in place (the panels'
// T_p, or the mid blocks' T when an outer block is assembled from them).
static ct_status assemble_t(ct_factor f, int64_t wblk, const void *G, void *T, void *Y, cudaStream_t s,
                            int64_t step) {
    const size_t es = f->es();
    const int64_t NB = f->NB;
    // The refining precisions assemble T from split-TF32 products on the
    // tensor cores (TF32x3: near FP32, three passes); FP32 and FP64 factors
    // keep their own arithmetic.
    const GemmKind small_kind = f->fp64 ? GEMM_F64 : (is_refine_prec(f->prec) ? GEMM_TF32X3 : GEMM_F32);
    for (int64_t o = step; o < wblk; o += step) {
        const int64_t wp = std::min<int64_t>(step, wblk - o);
        if (!f->fp64 && wp <= 32 && (size_t)o * 33 * sizeof(float) <= 200 * 1024) {
            CT_TRY(t_assemble(o, (int)wp, (const float *)G, NB, (float *)T, NB, s));
            continue;
        }
        const void *Tp = at(T, o, o, NB, es);
        GemmArgs g1{small_kind, false, false, o, wp, wp, 1.0, at(const_cast<void *>(G), 0, o, NB, es), NB,
                    Tp, NB, 0.0, Y, NB};
        CT_TRY(gemm(g1, f->gemm_ws, s));
        GemmArgs g2{small_kind, false, false, o, wp, o, -1.0, T, NB, Y, NB, 0.0, at(T, 0, o, NB, es), NB};
        CT_TRY(gemm(g2, f->gemm_ws, s));
    }
    return CT_OK;
}

// Factor outer blocks [J0, J1) of VR; trailing updates reach column col_end.
// (In core: all blocks, col_end = n.  Out of core: the blocks of one
// superpanel, whose columns [c0, col_end) are resident; VR is then offset so
// that global column indices address the superpanel buffer.)
//
// Three levels for the tensor-core paths: panels of nb = 32 update only the
// rest of their mid block of MB = 256 columns; a finished mid block updates
// the rest of its outer block with one rank-256 product (its T from its own
// Gram matrix); a finished outer block updates the trailing matrix.  The
// rank-32 updates then sweep at most 224 columns instead of the whole block.
ct_status qr_factor_range(ct_factor f, int64_t J0, int64_t J1, int64_t col_end, cudaStream_t s) {
    const size_t es = f->es();
    const int64_t NB = f->NB, nb = f->nb, n = col_end, lda = f->lda;
    const int64_t MB = (!f->fp64 && NB >= 512) ? 256 : NB;
    CT_TRY(f->G.ensure(es * (size_t)NB * NB));
    // misc (each NB x NB, ld NB): Vt_p of a panel | Y for the T assembly | Vt_q, G_q of a mid block
    CT_TRY(f->misc.ensure(4 * es * (size_t)NB * NB));
    void *Vtp = f->misc.ptr;
    void *Y = (char *)f->misc.ptr + es * (size_t)NB * NB;
    void *Vtq = (char *)f->misc.ptr + 2 * es * (size_t)NB * NB;
    void *Gq = (char *)f->misc.ptr + 3 * es * (size_t)NB * NB;
    for (int64_t J = J0; J < J1; ++J) {
        const int64_t j = J * NB;
        const int w = (int)std::min<int64_t>(NB, f->n - j);
        void *VtJ = (char *)f->Vtop + es * (size_t)J * NB * NB;
        void *TJ = (char *)f->Tall + es * (size_t)J * NB * NB;
        CT_CUDA(cudaMemsetAsync(TJ, 0, es * (size_t)NB * NB, s));
        for (int64_t q = j; q < j + w; q += MB) {
            const int wq = (int)std::min<int64_t>(MB, j + w - q);
            for (int64_t p = q; p < q + wq; p += nb) {
                const int wp = (int)std::min<int64_t>(nb, q + wq - p);
                // T_p of this panel goes straight into its diagonal block of T_J;
                // the Gram panel kernels write it with the top of V
                void *Tp = at(TJ, p - j, p - j, NB, es);
                bool made = false, made16 = false;
                const int64_t ncols_in = q + wq - (p + wp);
                // BF16 updates: the panel kernel also rounds V below its top
                // block for the update of the rest of the mid block
                void *v16 = nullptr;
                const int64_t kbp = f->row_end(p + wp) - p - wp;
                if (!f->fp64 && f->upd_kind == GEMM_BF16 && wp == 32 && ncols_in > 0 && kbp > 0) {
                    CT_TRY(f->V16.ensure(2 * (size_t)round_up(wp, 64) * (size_t)kbp));
                    v16 = f->V16.ptr;
                }
                CT_TRY(panel_qr(f->fp64, f->VR, lda, f->row_end(p + wp), p, wp, f->tau, f->panel_ws, s,
                                f->gram_panel, Tp, Vtp, NB, &made, v16, round_up(wp, 64), &made16));
                if (!made) {
                    CT_TRY(extract_vtop(f->fp64, f->VR, lda, p, wp, Vtp, NB, s));
                    CT_TRY(gram(f, p, wp, Vtp, f->G.ptr, s));
                    CT_TRY(larft_from_gram(f->fp64, wp, f->G.ptr, NB, (char *)f->tau + es * p, Tp, NB, s));
                }
                if (ncols_in > 0)
                    CT_TRY(apply_block(f, p, wp, Vtp, Tp, true, at(f->VR, p, p + wp, lda, es), lda,
                                       ncols_in, s, f->upd_kind, nullptr, 0, made16 ? v16 : nullptr));
            }
            const int64_t ncols_mid = j + w - (q + wq);
            if (wq < w && ncols_mid > 0) {
                // the mid block's reflector on the rest of the outer block
                void *Tq = at(TJ, q - j, q - j, NB, es);
                CT_TRY(extract_vtop(f->fp64, f->VR, lda, q, wq, Vtq, NB, s));
                CT_TRY(gram(f, q, wq, Vtq, Gq, s));
                CT_TRY(assemble_t(f, wq, Gq, Tq, Y, s, nb));
                CT_TRY(apply_block(f, q, wq, Vtq, Tq, true, at(f->VR, q, q + wq, lda, es), lda, ncols_mid,
                                   s, f->upd_kind, nullptr, 0));
            }
        }
        CT_TRY(extract_vtop(f->fp64, f->VR, lda, j, w, VtJ, NB, s));
        if (w > nb) {
            CT_TRY(gram(f, j, w, VtJ, f->G.ptr, s));
            if (MB < NB && w > MB) {
                // from the mid blocks' T on the diagonal; the last mid block's
                // own T (not needed inside the loop) first, from its part of G
                const int64_t ql = (w - 1) / MB * MB, wl = w - ql;
                if (wl > nb)
                    CT_TRY(assemble_t(f, wl, at(f->G.ptr, ql, ql, NB, es), at(TJ, ql, ql, NB, es), Y, s, nb));
                CT_TRY(assemble_t(f, w, f->G.ptr, TJ, Y, s, MB));
            } else {
                CT_TRY(assemble_t(f, w, f->G.ptr, TJ, Y, s, nb));
            }
        }
        if (j + w < n)
            CT_TRY(apply_block(f, j, w, VtJ, TJ, true, at(f->VR, j, j + w, lda, es), lda, n - j - w, s,
                               f->upd_kind, nullptr, 0));
    }
    return CT_OK;
}

ct_status qr_factor_run(ct_factor f, cudaStream_t s) { return qr_factor_range(f, 0, f->nblocks, f->n, s); }

// Rows j+w .. row_end(j+w) of V_J (the part below its top block) from the
// host copy into the staging buffer (ld = rows rounded up to 32).
ct_status stage_v_block(ct_factor f, int64_t J, void *dst, int64_t *ldd, cudaStream_t s) {
    const size_t es = f->es();
    const int64_t j = J * f->NB;
    const int w = (int)std::min<int64_t>(f->NB, f->n - j);
    const int64_t kb = f->row_end(j + w) - j - w;
    *ldd = round_up(std::max<int64_t>(kb, 1), 32);
    if (kb <= 0) return CT_OK;
    ProfScope prof(PROF_H2D_V, s, 0.0, (double)es * kb * w);
    if (f->store) {  // disk tier: block J from the cache (read on demand if missing)
        DiskStore *d = f->store;
        int slot = -1;
        CT_TRY(d->acquire(J, s, &slot));
        const int64_t rb = d->block_rows(J);  // = row_end(j + w)
        const cudaError_t e = cudaMemcpy2DAsync(dst, es * (size_t)*ldd, (const char *)d->slot_ptr(slot) + es * (size_t)(j + w),
                                                es * (size_t)rb, es * (size_t)kb, w, cudaMemcpyHostToDevice, s);
        CT_TRY(d->release(slot, s));
        CT_CUDA(e);
        return CT_OK;
    }
    CT_CUDA(cudaMemcpy2DAsync(dst, es * (size_t)*ldd, (const char *)f->VR_host + es * (size_t)(j + w + j * f->lda),
                              es * (size_t)f->lda, es * (size_t)kb, w, cudaMemcpyHostToDevice, s));
    return CT_OK;
}

ct_status apply_q_blocks(ct_factor f, bool transpose, void *C, int64_t ldc, int64_t k,
                         cudaStream_t s) {
    const size_t es = f->es();
    const int64_t NB = f->NB;
    for (int64_t t = 0; t < f->nblocks; ++t) {
        const int64_t J = transpose ? t : f->nblocks - 1 - t;
        const int64_t j = J * NB;
        const int w = (int)std::min<int64_t>(NB, f->n - j);
        const void *VtJ = (char *)f->Vtop + es * (size_t)J * NB * NB;
        const void *TJ = (char *)f->Tall + es * (size_t)J * NB * NB;
        if (f->ooc) {  // stream the block's V from host memory or the file
            if (f->store) {  // read the next blocks ahead while this one is applied
                const int ahead = std::max(1, f->store->nslots() / 2 - 1);
                for (int64_t q = 1; q <= ahead && t + q < f->nblocks; ++q)
                    f->store->prefetch(transpose ? t + q : f->nblocks - 1 - t - q);
            }
            int64_t ldv = 0;
            CT_TRY(stage_v_block(f, J, f->stage, &ldv, s));
            CT_TRY(apply_block(f, j, w, VtJ, TJ, transpose, (char *)C + es * (size_t)j, ldc, k, s, f->kind,
                               f->stage, ldv));
            continue;
        }
        CT_TRY(apply_block(f, j, w, VtJ, TJ, transpose, (char *)C + es * (size_t)j, ldc, k, s, f->kind,
                           nullptr, 0));
    }
    return CT_OK;
}

}  // namespace ctqr
