"""CPU oracle for the CT-QR hot path (arxiv 2412.07631).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.  It shares no code
with the CUDA path.

Two routes compute the least-squares image x* = argmin ||A~ x - b~||:
  * ``qr_solve``: the plain C loops of ctqr_oracle.c (unblocked Householder QR,
    reflector-by-reflector Q^T application, back-substitution; Sec. 2 Eqs. 2-3).
    Level-2 work, used up to a few thousand unknowns.
  * ``lapack_qr_solve``: the paper's in-core route, Sec. 2.1: three LAPACK
    calls, dgeqrf (A = QR), dormqr (C = Q^T B), dtrtrs/dtrsm (R X = C), through
    scipy.  Used for the 128x128 geometry, where the plain loops are too slow.
    It is pinned against ``qr_solve`` and the long-double normal equations on
    the small cases.

Functions and the passage they follow:
  view_table, siddon_csr, dense_system ... Sec. 2 Eq. 1 (a_ij), Siddon lengths
  householder_qr .......................... Sec. 2 Eq. 2, Sec. 2.1 (dgeqrf)
  apply_qt / apply_q ...................... Sec. 2 Eq. 3 (C = Q^T B), Q implicit
  backsolve ............................... Sec. 2 Eq. 3 (R X = C), Sec. 2.1 (dtrsm)
  lapack_qr_gradient ...................... the transpose of Eq. 3's steps (loss gradient)
  normal_eq_ld ............................ brute force, (A~^T A~) x = A~^T b~
  residual_ld / certificate ............... ||x - x*|| <= ||A~^T(b~ - A~ x)|| / lambda
  quality ................................. Sec. 3.1.3, Eqs. for SNR, MSE, PSNR
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """The compiled oracle.  CTQR_ORACLE_LIB names another build of
    ctqr_oracle.c instead (the mutation tests load deliberately broken copies
    this way to show that the pins reject them)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("CTQR_ORACLE_LIB") or _build.build())
        dp = C.POINTER(C.c_double)
        i32p = C.POINTER(C.c_int32)
        i64p = C.POINTER(C.c_int64)
        I64 = C.c_int64
        _lib.oracle_view_table.argtypes = [C.c_int, C.c_double, dp]
        _lib.oracle_siddon_ray.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                           i32p, dp, dp]
        _lib.oracle_siddon_ray.restype = C.c_int
        _lib.oracle_siddon_count.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                             C.c_double, i32p]
        _lib.oracle_siddon_count.restype = I64
        _lib.oracle_siddon_fill.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                            C.c_double, i64p, i32p, dp]
        _lib.oracle_joseph_ray.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, i32p, dp]
        _lib.oracle_joseph_count_rays.argtypes = [C.c_int, C.c_double, I64, dp, i32p]
        _lib.oracle_joseph_count_rays.restype = I64
        _lib.oracle_joseph_fill_rays.argtypes = [C.c_int, C.c_double, I64, dp, i64p, i32p, dp]
        _lib.oracle_fan_rays.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp]
        _lib.oracle_siddon_count_rays.argtypes = [C.c_int, C.c_double, I64, dp, i32p]
        _lib.oracle_siddon_count_rays.restype = I64
        _lib.oracle_siddon_fill_rays.argtypes = [C.c_int, C.c_double, I64, dp, i64p, i32p, dp]
        _lib.oracle_dense_from_csr.argtypes = [I64, I64, i64p, i32p, dp, C.c_double, dp, I64]
        _lib.oracle_forward.argtypes = [I64, I64, i64p, i32p, dp, I64, dp, I64, dp, I64]
        _lib.oracle_householder_qr.argtypes = [I64, I64, dp, I64, dp]
        for name in ("oracle_apply_qt", "oracle_apply_q"):
            getattr(_lib, name).argtypes = [I64, I64, dp, I64, dp, I64, dp, I64]
        for name in ("oracle_backsolve", "oracle_forwardsolve_rt"):
            getattr(_lib, name).argtypes = [I64, dp, I64, I64, dp, I64]
        _lib.oracle_normal_eq_ld.argtypes = [I64, I64, i64p, i32p, dp, C.c_double, I64, dp, I64,
                                             dp, I64]
        _lib.oracle_normal_eq_ld.restype = C.c_int
        _lib.oracle_residual_ld.argtypes = [I64, I64, i64p, i32p, dp, C.c_double, I64, dp, I64,
                                            dp, I64, dp, I64, dp, I64]
    return _lib


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Parallel-beam geometry: n_side^2 pixels of width pixel_width centred on
    the origin, n_views angles over arc_deg (endpoint excluded), n_bins
    detector bins of width bin_width centred on the axis; optional
    sqrt(lambda)*I rows below the ray rows.  kind="fan": the scanner of the
    paper's Tables (Sec. 3.1, 3.2): a point source at distance source_dist
    from the axis, n_views source positions over arc_deg, n_bins detectors
    of an equiangular arc spanning fan_deg (bin_width unused)."""
    n_side: int
    n_views: int
    n_bins: int
    pixel_width: float = 1.0
    bin_width: float = 1.0
    arc_deg: float = 180.0
    sqrt_lambda: float = 0.0
    kind: str = "parallel"
    source_dist: float = 0.0
    fan_deg: float = 0.0
    projector: str = "siddon"  # or "joseph"

    @property
    def n(self) -> int:
        return self.n_side * self.n_side

    @property
    def m(self) -> int:
        return self.n_views * self.n_bins

    @property
    def rows(self) -> int:
        return self.m + (self.n if self.sqrt_lambda > 0 else 0)


def view_table(g: Geometry) -> np.ndarray:
    cs = np.empty(2 * g.n_views, np.float64)
    lib().oracle_view_table(g.n_views, g.arc_deg, _p(cs))
    return cs.reshape(g.n_views, 2)


def siddon_ray(g: Geometry, c: float, s: float, t: float):
    """Segments (pixel index, length) of one ray, in walk order."""
    cap = 2 * g.n_side + 4
    pix = np.empty(cap, np.int32)
    ln = np.empty(cap, np.float64)
    work = np.empty(cap, np.float64)
    k = lib().oracle_siddon_ray(g.n_side, g.pixel_width, c, s, t, _p(pix, C.c_int32), _p(ln),
                                _p(work))
    return pix[:k].copy(), ln[:k].copy()


@dataclasses.dataclass
class CSR:
    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col_idx: np.ndarray  # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    def args(self):
        return (_p(self.row_ptr, C.c_int64), _p(self.col_idx, C.c_int32), _p(self.val))

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def fan_rays(g: Geometry) -> np.ndarray:
    """(m, 3) table of (c, s, t) per fan-beam ray, i = v n_bins + d."""
    out = np.empty(3 * g.m, np.float64)
    lib().oracle_fan_rays(g.n_views, g.n_bins, g.arc_deg, g.fan_deg, g.source_dist, _p(out))
    return out.reshape(g.m, 3)


def ray_table(g: Geometry) -> np.ndarray:
    """(m, 3) table of (c, s, t) per ray of either geometry."""
    if g.kind == "fan":
        return fan_rays(g)
    cs = view_table(g)
    d = np.arange(g.n_bins, dtype=np.float64)
    t = (d - 0.5 * (g.n_bins - 1)) * g.bin_width  # the same two roundings as the kernels
    out = np.empty((g.n_views, g.n_bins, 3))
    out[:, :, 0] = cs[:, None, 0]
    out[:, :, 1] = cs[:, None, 1]
    out[:, :, 2] = t[None, :]
    return out.reshape(g.m, 3)


def joseph_ray(g: Geometry, c: float, s: float, t: float):
    """Entries (pixel index, weight) of one ray under Joseph's projector."""
    cap = 2 * g.n_side + 2
    pix = np.empty(cap, np.int32)
    val = np.empty(cap, np.float64)
    k = lib().oracle_joseph_ray(g.n_side, g.pixel_width, c, s, t, _p(pix, C.c_int32), _p(val))
    return pix[:k].copy(), val[:k].copy()


def siddon_csr(g: Geometry) -> CSR:
    """The system matrix A (ray rows only) as CSR, entries in walk order:
    Siddon's exact lengths, or Joseph's interpolation weights when
    g.projector == "joseph"."""
    L = lib()
    if g.projector == "joseph":
        rays = np.ascontiguousarray(ray_table(g))
        cnt = np.empty(g.m, np.int32)
        nnz = L.oracle_joseph_count_rays(g.n_side, g.pixel_width, g.m, _p(rays), _p(cnt, C.c_int32))
        row_ptr = np.zeros(g.m + 1, np.int64)
        np.cumsum(cnt, out=row_ptr[1:])
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        L.oracle_joseph_fill_rays(g.n_side, g.pixel_width, g.m, _p(rays), _p(row_ptr, C.c_int64),
                                  _p(col, C.c_int32), _p(val))
        return CSR(g.m, g.n, row_ptr, col, val)
    if g.kind == "fan":
        rays = np.ascontiguousarray(fan_rays(g))
        cnt = np.empty(g.m, np.int32)
        nnz = L.oracle_siddon_count_rays(g.n_side, g.pixel_width, g.m, _p(rays), _p(cnt, C.c_int32))
        row_ptr = np.zeros(g.m + 1, np.int64)
        np.cumsum(cnt, out=row_ptr[1:])
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        L.oracle_siddon_fill_rays(g.n_side, g.pixel_width, g.m, _p(rays), _p(row_ptr, C.c_int64),
                                  _p(col, C.c_int32), _p(val))
        return CSR(g.m, g.n, row_ptr, col, val)
    cnt = np.empty(g.m, np.int32)
    nnz = L.oracle_siddon_count(g.n_side, g.n_views, g.n_bins, g.pixel_width, g.bin_width,
                                g.arc_deg, _p(cnt, C.c_int32))
    row_ptr = np.zeros(g.m + 1, np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    assert row_ptr[-1] == nnz
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    L.oracle_siddon_fill(g.n_side, g.n_views, g.n_bins, g.pixel_width, g.bin_width, g.arc_deg,
                         _p(row_ptr, C.c_int64), _p(col, C.c_int32), _p(val))
    return CSR(g.m, g.n, row_ptr, col, val)


def dense_system(g: Geometry, csr: CSR | None = None) -> np.ndarray:
    """Dense column-major A~ = [A; sqrt(lambda) I] (Fortran-ordered array)."""
    csr = csr if csr is not None else siddon_csr(g)
    A = np.zeros((g.rows, g.n), np.float64, order="F")
    lib().oracle_dense_from_csr(g.m, g.n, *csr.args(), g.sqrt_lambda, _p(A), g.rows)
    return A


def forward(csr: CSR, X: np.ndarray) -> np.ndarray:
    """P = A X for images X (n x k, any order) -> (m x k) Fortran-ordered."""
    X = np.asfortranarray(X.reshape(csr.n, -1), dtype=np.float64)
    k = X.shape[1]
    P = np.empty((csr.m, k), np.float64, order="F")
    lib().oracle_forward(csr.m, csr.n, *csr.args(), k, _p(X), csr.n, _p(P), csr.m)
    return P


def householder_qr(A: np.ndarray):
    """Unblocked Householder QR of a copy of A; returns (VR, tau) in LAPACK layout."""
    VR = np.array(A, dtype=np.float64, order="F", copy=True)
    M, n = VR.shape
    tau = np.zeros(n, np.float64)
    lib().oracle_householder_qr(M, n, _p(VR), M, _p(tau))
    return VR, tau


def apply_qt(VR, tau, B):
    B = np.array(B, dtype=np.float64, order="F", copy=True).reshape(VR.shape[0], -1, order="F")
    lib().oracle_apply_qt(VR.shape[0], VR.shape[1], _p(VR), VR.shape[0], _p(tau), B.shape[1],
                          _p(B), B.shape[0])
    return B


def apply_q(VR, tau, B):
    B = np.array(B, dtype=np.float64, order="F", copy=True).reshape(VR.shape[0], -1, order="F")
    lib().oracle_apply_q(VR.shape[0], VR.shape[1], _p(VR), VR.shape[0], _p(tau), B.shape[1],
                         _p(B), B.shape[0])
    return B


def backsolve(VR, C_):
    """X = R^{-1} C[0:n] with R the upper triangle of VR[0:n, 0:n]."""
    n = VR.shape[1]
    X = np.array(C_[:n], dtype=np.float64, order="F", copy=True).reshape(n, -1, order="F")
    lib().oracle_backsolve(n, _p(VR), VR.shape[0], X.shape[1], _p(X), n)
    return X


def forwardsolve_rt(VR, G):
    """Y = R^{-T} G."""
    n = VR.shape[1]
    Y = np.array(G, dtype=np.float64, order="F", copy=True).reshape(n, -1, order="F")
    lib().oracle_forwardsolve_rt(n, _p(VR), VR.shape[0], Y.shape[1], _p(Y), n)
    return Y


def extend_rhs(g: Geometry, B: np.ndarray) -> np.ndarray:
    """b~ = [b; 0] (zeros in the sqrt(lambda) rows)."""
    B = B.reshape(g.m, -1, order="F")
    Bt = np.zeros((g.rows, B.shape[1]), np.float64, order="F")
    Bt[: g.m] = B
    return Bt


def qr_solve(g: Geometry, A: np.ndarray, B: np.ndarray):
    """x = R^{-1} (Q^T b~) with the plain C Householder route.  Returns (X, VR, tau)."""
    VR, tau = householder_qr(A)
    Ct = apply_qt(VR, tau, extend_rhs(g, B))
    return backsolve(VR, Ct), VR, tau


def lapack_qr_solve(g: Geometry, A: np.ndarray, B: np.ndarray, overwrite: bool = False):
    """The paper's in-core route (Sec. 2.1): dgeqrf, dormqr, dtrtrs.

    Returns (X, R) where R is the n x n upper-triangular factor."""
    from scipy.linalg import lapack
    A = np.asfortranarray(A, dtype=np.float64)
    qr, tau, work, info = lapack.dgeqrf(A, overwrite_a=overwrite)
    assert info == 0, info
    Bt = extend_rhs(g, B)
    lwork = max(1, int(lapack.dormqr("L", "T", qr, tau, Bt, -1)[1][0].real))
    c, work, info = lapack.dormqr("L", "T", qr, tau, Bt, lwork, overwrite_c=True)
    assert info == 0, info
    n = g.n
    R = np.triu(qr[:n, :n])
    X, info = lapack.dtrtrs(R, np.asfortranarray(c[:n]), lower=0, trans=0)
    assert info == 0, info
    return X, R


def lapack_qr_gradient(g: Geometry, A: np.ndarray, B: np.ndarray, X_true: np.ndarray, k_total: int,
                       overwrite: bool = False):
    """Gradient of the loss L = ||X - X_true||_F^2 / (n k_total) with respect
    to the sinograms, through x = R^-1 Q1^T b~ (Sec. 2 Eq. 3) on the LAPACK
    route of Sec. 2.1.  With g = dL/dx = 2 (x - x_true) / (n k_total) the
    gradient is [Q [R^-T g; 0]]_{0:m}: the transposes of Eq. 3's two steps
    in reverse order (dtrtrs transposed, then dormqr 'N').  B and X_true hold
    the sampled slices as columns; k_total is the batch size the loss
    averages over.  Returns (grad_b (m x s), x (n x s))."""
    from scipy.linalg import lapack
    A = np.asfortranarray(A, dtype=np.float64)
    qr, tau, work, info = lapack.dgeqrf(A, overwrite_a=overwrite)
    assert info == 0, info
    n, m = g.n, g.m

    def ormqr(trans, C_):
        lwork = max(1, int(lapack.dormqr("L", trans, qr, tau, C_, -1)[1][0].real))
        out, _, inf = lapack.dormqr("L", trans, qr, tau, C_, lwork, overwrite_c=True)
        assert inf == 0, inf
        return out

    R = np.triu(qr[:n, :n])
    c = ormqr("T", extend_rhs(g, B))
    X, info = lapack.dtrtrs(R, np.asfortranarray(c[:n]), lower=0, trans=0)
    assert info == 0, info
    gx = 2.0 * (X - np.asarray(X_true, np.float64).reshape(n, -1, order="F")) / (n * k_total)
    z, info = lapack.dtrtrs(R, np.asfortranarray(gx), lower=0, trans=1)
    assert info == 0, info
    full = np.zeros((g.rows, z.shape[1]), np.float64, order="F")
    full[:n] = z
    return np.asfortranarray(ormqr("N", full)[:m]), X


def normal_eq_ld(g: Geometry, csr: CSR, B: np.ndarray) -> np.ndarray:
    """Brute force: (A^T A + lambda I) x = A^T b by long-double Cholesky."""
    B = np.asfortranarray(B.reshape(g.m, -1, order="F"), dtype=np.float64)
    k = B.shape[1]
    X = np.empty((g.n, k), np.float64, order="F")
    rc = lib().oracle_normal_eq_ld(g.m, g.n, *csr.args(), g.sqrt_lambda, k, _p(B), g.m, _p(X), g.n)
    if rc != 0:
        raise np.linalg.LinAlgError(f"normal equations not positive definite at pivot {rc - 1}")
    return X


def residual_ld(g: Geometry, csr: CSR, B: np.ndarray, X: np.ndarray):
    """(r, g) with r = b~ - A~ x and g = A~^T r, accumulated in long double."""
    B = np.asfortranarray(B.reshape(g.m, -1, order="F"), dtype=np.float64)
    X = np.asfortranarray(X.reshape(g.n, -1, order="F"), dtype=np.float64)
    k = B.shape[1]
    r = np.empty((g.rows if g.sqrt_lambda > 0 else g.m, k), np.float64, order="F")
    gg = np.empty((g.n, k), np.float64, order="F")
    lib().oracle_residual_ld(g.m, g.n, *csr.args(), g.sqrt_lambda, k, _p(B), g.m, _p(X), g.n,
                             _p(r), r.shape[0], _p(gg), g.n)
    return r, gg


def certificate(g: Geometry, csr: CSR, B: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Per-slice bound on ||x - x*|| / ||x||: ||A~^T(b~ - A~ x)|| / (lambda ||x||).

    Every singular value of A~ = [A; sqrt(lambda) I] is >= sqrt(lambda), so
    ||A~^T A~ e|| >= lambda ||e|| for the error e = x - x*, and A~^T A~ e = -g."""
    assert g.sqrt_lambda > 0
    _, gg = residual_ld(g, csr, B, X)
    lam = g.sqrt_lambda ** 2
    xn = np.linalg.norm(X.reshape(g.n, -1, order="F"), axis=0)
    return np.linalg.norm(gg, axis=0) / lam / np.maximum(xn, 1e-300)


def quality(x_ref: np.ndarray, x: np.ndarray, max_val: float = 1.0) -> dict:
    """SNR, MSE, RMSE and PSNR of one image against its reference (Sec. 3.1.3;
    MAX = the largest value a pixel can take, 1 for the phantoms used here)."""
    x_ref = np.asarray(x_ref, np.float64).ravel()
    x = np.asarray(x, np.float64).ravel()
    err = float(np.sum((x_ref - x) ** 2))
    sig = float(np.sum(x_ref ** 2))
    mse = err / x_ref.size
    return {
        "snr": 10.0 * math.log10(sig / err) if err > 0 else math.inf,
        "mse": mse,
        "rmse": math.sqrt(mse),
        "psnr": 10.0 * math.log10(max_val ** 2 / mse) if mse > 0 else math.inf,
    }
