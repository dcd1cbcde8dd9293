"""Python binding of libctqr (include/ctqr.h): direct algebraic CT
reconstruction by dense Householder QR on a B300 (arxiv 2412.07631).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libctqr.so; torch supplies device memory and the current stream.
If the compiled library is missing and cannot be built, importing the
binding's entry points raises -- there is no CPU fallback.

Layout convention: a batch of k sinograms is a torch tensor of shape (k, m)
(row s = sinogram s), which is exactly the column-major m x k matrix B of the
C ABI with ldb = m; likewise images X are (k, n).
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "tf32x3": 4, "bf16x3": 5}
GEMM_KINDS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "tf32x3": 4, "bf16x3": 5}


class Geometry(C.Structure):
    _fields_ = [("n_side", C.c_int32), ("n_views", C.c_int32), ("n_bins", C.c_int32),
                ("pixel_width", C.c_double), ("bin_width", C.c_double),
                ("arc_deg", C.c_double), ("sqrt_lambda", C.c_double), ("kind", C.c_int32),
                ("source_dist", C.c_double), ("fan_deg", C.c_double), ("projector", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("refine_max_iter", C.c_int32),
                ("refine_tol", C.c_double), ("nb_outer", C.c_int32), ("nb_inner", C.c_int32),
                ("flags", C.c_int32), ("stop_after", C.c_int32), ("solve_block", C.c_int32),
                ("solve_split", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("stop_measure", C.c_double),
                ("rjj_min_abs", C.c_double), ("rjj_max_abs", C.c_double),
                ("inner_iterations", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class CTQRError(RuntimeError):
    def __init__(self, status: int, name: str, detail: str):
        super().__init__(f"{name}: {detail}")
        self.status = status
        self.name = name


_LIB = None
SYMBOLS = ["ct_status_str", "ct_last_error", "ct_build_system", "ct_system_info",
           "ct_system_device_ptrs", "ct_system_export", "ct_forward_project", "ct_qr_factor",
           "ct_factor_device_ptrs", "ct_factor_export", "ct_solve", "ct_solve_host",
           "ct_solve_adjoint", "ct_system_free", "ct_factor_free", "ct_gemm", "ct_stats_reset",
           "ct_stats_read", "ct_stats_dump", "ct_gemm_noalloc", "ct_factor_save",
           "ct_factor_load", "ct_build_system_host", "ct_qr_factor_ooc", "ct_host_cache_release",
           "ct_build_system_disk", "ct_system_open_disk", "ct_disk_progress", "ct_disk_stats",
           "ct_selftest_wait_timeout", "ct_debug_canaries", "ct_debug_check_canaries"]


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libctqr.so (building it in-tree with nvcc if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build()
    L = C.CDLL(path)
    vp, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
    L.ct_status_str.restype = C.c_char_p
    L.ct_status_str.argtypes = [C.c_int]
    L.ct_last_error.restype = C.c_char_p
    L.ct_build_system.argtypes = [C.POINTER(Geometry), C.c_int, vp, C.POINTER(vp)]
    L.ct_system_info.argtypes = [vp] + [C.POINTER(I64)] * 5
    L.ct_system_device_ptrs.argtypes = [vp] + [C.POINTER(vp)] * 4
    L.ct_system_export.argtypes = [vp, vp, vp, vp, vp, I64]
    L.ct_forward_project.argtypes = [vp, vp, I64, I32, vp, I64, vp]
    L.ct_qr_factor.argtypes = [vp, C.POINTER(Opts), vp, C.POINTER(vp)]
    L.ct_factor_device_ptrs.argtypes = [vp, C.POINTER(vp), C.POINTER(I64), C.POINTER(vp)]
    L.ct_factor_export.argtypes = [vp, vp, I64, vp]
    for name in ("ct_solve", "ct_solve_host", "ct_solve_adjoint"):
        getattr(L, name).argtypes = [vp, vp, I64, I32, vp, I64, C.POINTER(Opts), vp,
                                     C.POINTER(SolveInfo)]
    L.ct_system_free.argtypes = [vp]
    L.ct_system_free.restype = None
    L.ct_factor_free.argtypes = [vp]
    L.ct_factor_free.restype = None
    L.ct_gemm.argtypes = [I32, C.c_char, C.c_char, I64, I64, I64, C.c_double, vp, I64, vp, I64,
                          C.c_double, vp, I64, vp]
    L.ct_gemm_noalloc.argtypes = list(L.ct_gemm.argtypes)
    L.ct_factor_save.argtypes = [vp, C.c_char_p]
    L.ct_build_system_host.argtypes = [C.POINTER(Geometry), I32, C.c_size_t, vp, C.POINTER(vp)]
    L.ct_qr_factor_ooc.argtypes = [vp, C.POINTER(Opts), C.c_size_t, vp, C.POINTER(vp)]
    L.ct_host_cache_release.argtypes = []
    L.ct_host_cache_release.restype = None
    L.ct_factor_load.argtypes = [vp, C.c_char_p, vp, C.POINTER(vp)]
    L.ct_stats_reset.argtypes = [I32]
    L.ct_stats_read.argtypes = [C.POINTER(I64), vp, vp, vp, vp]
    L.ct_stats_dump.argtypes = [C.c_char_p]
    L.ct_build_system_disk.argtypes = [C.POINTER(Geometry), C.c_int, C.c_char_p, I32, C.c_size_t, vp,
                                       C.POINTER(vp)]
    L.ct_system_open_disk.argtypes = [C.c_char_p, C.c_size_t, vp, C.POINTER(vp)]
    L.ct_disk_progress.argtypes = [vp, C.POINTER(I32), C.POINTER(I64)]
    L.ct_disk_stats.argtypes = [I32] + [C.POINTER(I64)] * 5 + [C.POINTER(C.c_double)] * 2
    L.ct_selftest_wait_timeout.argtypes = [vp]
    L.ct_debug_canaries.argtypes = [I32]
    L.ct_debug_check_canaries.argtypes = [I32, C.POINTER(I64), C.POINTER(I64)]
    for name in SYMBOLS:
        if name not in ("ct_status_str", "ct_last_error", "ct_system_free", "ct_factor_free"):
            getattr(L, name).restype = C.c_int
    _LIB = L
    return L


def _check(st: int, allow=()):
    if st == 0 or st in allow:
        return st
    L = lib()
    raise CTQRError(st, L.ct_status_str(st).decode(), (L.ct_last_error() or b"").decode())


def _check_factor(st: int, h, system, precision: str):
    """_check for the factorisations.  A rank-deficient system (CT_ERR_RANK)
    still returns its factor; it travels with the exception as `.factor`
    (freed with it) so the caller can inspect |R_jj|."""
    if st == RANK and h.value:
        try:
            _check(st)
        except CTQRError as e:
            e.factor = Factor(h, system, precision)
            raise
    _check(st)


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


GEOMETRY_KINDS = {"parallel": 0, "fan": 1}
PROJECTORS = {"siddon": 0, "joseph": 1}


def make_geometry(n_side, n_views, n_bins, sqrt_lambda=0.0, pixel_width=1.0, bin_width=1.0,
                  arc_deg=None, kind="parallel", source_dist=0.0, fan_deg=0.0,
                  projector="siddon") -> Geometry:
    """Parallel beam (arc 180 by default) or kind="fan": a point source at
    source_dist from the axis and an equiangular arc of n_bins detectors
    spanning fan_deg (arc 360 by default).  projector: "siddon" (exact
    lengths) or "joseph" (interpolated samples)."""
    if arc_deg is None:
        arc_deg = 360.0 if kind == "fan" else 180.0
    return Geometry(n_side, n_views, n_bins, pixel_width, bin_width, arc_deg, sqrt_lambda,
                    GEOMETRY_KINDS[kind], source_dist, fan_deg, PROJECTORS[projector])


INTERRUPTED = 12  # ct_status CT_ERR_INTERRUPTED
RANK = 4  # ct_status CT_ERR_RANK


class System:
    """Device-resident system matrix A~ = [A; sqrt(lambda) I] (dense, column
    major) plus the FP64 CSR/CSC of A, built by the Siddon kernels."""

    def __init__(self, geom: Geometry, storage: str = "fp32", stream=None, host_budget: int = 0,
                 disk_path: str | None = None, host_cache: int = 1 << 30, block_cols: int = 0,
                 _handle=None):
        """host_budget > 0: keep the dense matrix in pinned host memory (built in
        column slabs of at most host_budget device bytes) for factor_ooc.
        disk_path: keep it in that file instead (column blocks of block_cols
        columns, host_cache bytes of pinned block cache) for factor_ooc."""
        self.geom = geom
        self.storage = storage
        h = C.c_void_p()
        if _handle is not None:
            h = _handle
        elif disk_path is not None:
            _check(lib().ct_build_system_disk(C.byref(geom), PRECISIONS[storage], disk_path.encode(),
                                              int(block_cols), C.c_size_t(int(host_cache)),
                                              _stream(stream), C.byref(h)))
        elif host_budget > 0:
            _check(lib().ct_build_system_host(C.byref(geom), PRECISIONS[storage], int(host_budget),
                                              _stream(stream), C.byref(h)))
        else:
            _check(lib().ct_build_system(C.byref(geom), PRECISIONS[storage], _stream(stream), C.byref(h)))
        self.h = h
        vals = [C.c_int64() for _ in range(5)]
        try:
            _check(lib().ct_system_info(h, *[C.byref(v) for v in vals]))
        except CTQRError:
            self.free()
            raise
        self.m, self.n, self.rows, self.lda, self.nnz = (v.value for v in vals)

    @classmethod
    def open_disk(cls, path: str, host_cache: int = 1 << 30, stream=None) -> "System":
        """Reopen a disk-backed system's file (assembled, partly or fully factored)."""
        import struct
        h = C.c_void_p()
        _check(lib().ct_system_open_disk(path.encode(), C.c_size_t(int(host_cache)), _stream(stream),
                                         C.byref(h)))
        # file header: magic[8], version u32, element size u32, then the geometry
        with open(path, "rb") as fh:
            head = fh.read(16 + C.sizeof(Geometry))
        es = struct.unpack_from("<I", head, 12)[0]
        geom = Geometry.from_buffer_copy(head, 16)
        return cls(geom, "fp64" if es == 8 else "fp32", _handle=h)

    def disk_progress(self) -> tuple[int, int]:
        """(state, done_cols) of a disk-backed system's file: state 0 assembled,
        1 factorisation in progress, 2 factored."""
        st, done = C.c_int32(), C.c_int64()
        _check(lib().ct_disk_progress(self.h, C.byref(st), C.byref(done)))
        return st.value, done.value

    def export_csr(self):
        import numpy as np
        rp = np.empty(self.m + 1, np.int64)
        ci = np.empty(max(self.nnz, 1), np.int32)
        va = np.empty(max(self.nnz, 1), np.float64)
        _check(lib().ct_system_export(self.h, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, None, 0))
        return rp, ci[: self.nnz], va[: self.nnz]

    def export_dense(self):
        import numpy as np
        dt = np.float64 if self.storage == "fp64" else np.float32
        A = np.empty((self.rows, self.n), dt, order="F")
        _check(lib().ct_system_export(self.h, None, None, None, A.ctypes.data, self.rows))
        return A

    def forward(self, X, stream=None):
        """P = A X for images X: torch float64 CUDA tensor (k, n) -> (k, m)."""
        import torch
        assert X.dtype == torch.float64 and X.is_cuda and X.is_contiguous()
        k = X.shape[0]
        P = torch.empty((k, self.m), dtype=torch.float64, device=X.device)
        _check(lib().ct_forward_project(self.h, _ptr(X), self.n, k, _ptr(P), self.m, _stream(stream)))
        return P

    def factor(self, precision: str | None = None, nb_outer: int | str = 0, nb_inner: int = 0,
               stream=None, column_panel: bool = False) -> "Factor":
        """nb_outer: outer block width (0: library default; "auto": the
        autotuner's cached choice for this geometry, measured on first use).
        column_panel: factor every panel column by column (CT_OPT_COLUMN_PANEL)
        instead of from its Gram matrices."""
        if precision is None:
            precision = "fp64" if self.storage == "fp64" else "tf32"
        if nb_outer == "auto":
            from . import autotune
            nb_outer = autotune.outer_block(self.geom, precision)
        o = Opts(PRECISIONS[precision], 0, 0.0, nb_outer, nb_inner, 2 if column_panel else 0)
        h = C.c_void_p()
        st = lib().ct_qr_factor(self.h, C.byref(o), _stream(stream), C.byref(h))
        _check_factor(st, h, self, precision)
        return Factor(h, self, precision)

    def factor_ooc(self, precision: str | None = None, device_budget: int = 16 << 30,
                   nb_outer: int = 0, nb_inner: int = 0, stream=None,
                   stop_after: int = 0, column_panel: bool = False) -> "Factor | None":
        """Out-of-core QR of a host- or disk-resident system (see
        ct_qr_factor_ooc).  stop_after > 0 (disk): stop after that many
        superpanels and return None; calling again resumes."""
        if precision is None:
            precision = "fp64" if self.storage == "fp64" else "tf32"
        o = Opts(PRECISIONS[precision], 0, 0.0, nb_outer, nb_inner, 2 if column_panel else 0,
                 int(stop_after))
        h = C.c_void_p()
        st = lib().ct_qr_factor_ooc(self.h, C.byref(o), C.c_size_t(int(device_budget)), _stream(stream),
                                    C.byref(h))
        if st == INTERRUPTED:
            return None
        _check_factor(st, h, self, precision)
        return Factor(h, self, precision)

    def free(self):
        if getattr(self, "h", None):
            lib().ct_system_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Factor:
    """Householder factors (V, T blocks, R) of a System, on the device."""

    def __init__(self, h, system: System, precision: str):
        self.h = h
        self.system = system  # kept alive: refinement reads its sparse rows
        self.precision = precision
        self.m, self.n, self.rows = system.m, system.n, system.rows
        self.last_info = None

    @property
    def io_dtype(self):
        import torch
        return torch.float32 if self.precision == "fp32" else torch.float64

    graphs = True  # capture repeated solve work in CUDA graphs (library default)
    # solve plan (ct_opts.solve_block, ct_opts.solve_split): superblock rows of
    # the triangular solve and least split-K depth of the solve's GEMMs (0, 0:
    # library defaults); autotune.solve_plan measures the best for a geometry
    solve_plan = (0, 0)

    def _opts(self, max_iter=0, tol=0.0):
        sb, split = self.solve_plan
        return Opts(PRECISIONS[self.precision], max_iter, tol, 0, 0, 0 if self.graphs else 1, 0,
                    int(sb), int(split))

    def solve(self, B, out=None, max_iter: int = 0, tol: float = 0.0, stream=None,
              allow_noconv: bool = False):
        """X = R^-1 (Q^T b~) (+ FP64 refinement for refining precisions).
        B: CUDA tensor (k, m) of io_dtype; returns X (k, n)."""
        import torch
        assert B.is_cuda and B.dtype == self.io_dtype and B.is_contiguous() and B.shape[1] == self.m
        k = B.shape[0]
        X = out if out is not None else torch.empty((k, self.n), dtype=B.dtype, device=B.device)
        info = SolveInfo()
        o = self._opts(max_iter, tol)
        st = lib().ct_solve(self.h, _ptr(B), self.m, k, _ptr(X), self.n, C.byref(o),
                            _stream(stream), C.byref(info))
        _check(st, allow=(5,) if allow_noconv else ())
        self.last_info = info.as_dict()
        return X

    def solve_host(self, B, out=None, max_iter: int = 0, tol: float = 0.0, stream=None):
        """As solve() with HOST tensors (k, m) -> (k, n); the copies are inside the call."""
        import torch
        assert not B.is_cuda and B.dtype == self.io_dtype and B.is_contiguous()
        k = B.shape[0]
        X = out if out is not None else torch.empty((k, self.n), dtype=B.dtype)
        info = SolveInfo()
        o = self._opts(max_iter, tol)
        _check(lib().ct_solve_host(self.h, _ptr(B), self.m, k, _ptr(X), self.n, C.byref(o),
                                   _stream(stream), C.byref(info)))
        self.last_info = info.as_dict()
        return X

    def adjoint(self, gX, out=None, max_iter: int = 0, tol: float = 0.0, stream=None,
                allow_noconv: bool = False):
        """gB = [Q [R^-T gX; 0]]_{0:m} for gX (k, n) -> (k, m); with refining
        factors, the same map refined in FP64 (gB = [A~ u]_{0:m},
        A~^T A~ u = gX)."""
        import torch
        assert gX.is_cuda and gX.dtype == self.io_dtype and gX.is_contiguous()
        k = gX.shape[0]
        gB = out if out is not None else torch.empty((k, self.m), dtype=gX.dtype, device=gX.device)
        info = SolveInfo()
        o = self._opts(max_iter, tol)
        st = lib().ct_solve_adjoint(self.h, _ptr(gX), self.n, k, _ptr(gB), self.m, C.byref(o),
                                    _stream(stream), C.byref(info))
        _check(st, allow=(5,) if allow_noconv else ())
        self.last_info = info.as_dict()
        return gB

    def export(self):
        import numpy as np
        dt = np.float64 if self.precision == "fp64" else np.float32
        VR = np.empty((self.rows, self.n), dt, order="F")
        tau = np.empty(self.n, dt)
        _check(lib().ct_factor_export(self.h, VR.ctypes.data, self.rows, tau.ctypes.data))
        return VR, tau

    def save(self, path: str):
        """Write this factorisation to a checkpoint file."""
        _check(lib().ct_factor_save(self.h, path.encode()))

    @classmethod
    def load(cls, system: "System", path: str, stream=None) -> "Factor":
        """Read a checkpoint written by save() for a system of the same geometry."""
        h = C.c_void_p()
        _check(lib().ct_factor_load(system.h, path.encode(), _stream(stream), C.byref(h)))
        prec = {v: k for k, v in PRECISIONS.items()}
        import struct
        with open(path, "rb") as fh:
            code = struct.unpack_from("<i", fh.read(16), 12)[0]
        return cls(h, system, prec[code])

    def free(self):
        if getattr(self, "h", None):
            lib().ct_factor_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gemm(kind: str, transa: str, transb: str, M: int, N: int, K: int, alpha: float, A, lda: int,
         B, ldb: int, beta: float, Cm, ldc: int, stream=None):
    """C = alpha op(A) op(B) + beta C on column-major device buffers (torch
    tensors used as raw storage)."""
    _check(lib().ct_gemm(GEMM_KINDS[kind], transa.encode(), transb.encode(), M, N, K, alpha,
                         _ptr(A), lda, _ptr(B), ldb, beta, _ptr(Cm), ldc, _stream(stream)))


class CTSolve:
    """Differentiable reconstruction layer: X = solve(B) with the backward
    pass grad_B = adjoint(grad_X) (Q R^-T grad_X on the ray rows, refined in
    FP64 for refining factors).  Use CTSolve.apply(B, factor[, max_iter,
    tol]); B is a CUDA tensor (k, m) of the factor's I/O dtype."""

    _fn = None

    @classmethod
    def apply(cls, B, factor, max_iter: int = 0, tol: float = 0.0):
        if cls._fn is None:
            import torch

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, B_, f_, it_, tol_):
                    ctx.f, ctx.it, ctx.tol = f_, it_, tol_
                    return f_.solve(B_.contiguous(), max_iter=it_, tol=tol_)

                @staticmethod
                def backward(ctx, gX):
                    gB = ctx.f.adjoint(gX.contiguous(), max_iter=ctx.it, tol=ctx.tol)
                    return gB, None, None, None

            cls._fn = _Fn
        return cls._fn.apply(B, factor, max_iter, tol)


STAT_CLASSES = ["tc_gemm", "simt_gemm", "panel", "trsm_diag", "spmm_fp64", "siddon", "other",
                "spmm_fp32", "tc_gemm_bf16", "h2d_v", "h2d_cols", "d2h_cols", "copy_wait", "convert"]


def selftest_wait_timeout(stream=None) -> str:
    """Run one device wait that cannot complete (a grid meet of a one-CTA grid
    that expects two) and return the status name the library reports for it:
    "CT_ERR_TIMEOUT" once the bounded wait has given up (about 4 s)."""
    st = lib().ct_selftest_wait_timeout(_stream(stream))
    return lib().ct_status_str(st).decode()


def debug_canaries(enable: bool = True):
    """ct_debug_canaries: guard bands past the capacity of scratch buffers
    allocated from now on (a sanitizer substitute)."""
    _check(lib().ct_debug_canaries(1 if enable else 0))


def debug_check_canaries(corrupt_first: bool = False) -> tuple[int, int]:
    """ct_debug_check_canaries: (buffers checked, buffers whose guard band was
    overwritten).  corrupt_first overwrites one guard byte first (a test of
    the check itself)."""
    checked, corrupted = C.c_int64(), C.c_int64()
    _check(lib().ct_debug_check_canaries(1 if corrupt_first else 0, C.byref(checked), C.byref(corrupted)))
    return checked.value, corrupted.value


def disk_stats(reset: bool = False) -> dict:
    """Disk-tier I/O counters (bytes, cache hits/prefetched/misses, I/O seconds)."""
    v = [C.c_int64() for _ in range(5)]
    t = [C.c_double() for _ in range(2)]
    _check(lib().ct_disk_stats(1 if reset else 0, *[C.byref(x) for x in v], *[C.byref(x) for x in t]))
    keys = ["bytes_read", "bytes_written", "hits", "prefetched", "misses"]
    out = {k: x.value for k, x in zip(keys, v)}
    out["read_s"], out["write_s"] = t[0].value, t[1].value
    return out


def stats_reset(timing: bool = False):
    """Zero the library's launch counter (and per-class event timing if asked)."""
    _check(lib().ct_stats_reset(1 if timing else 0))


def stats_dump(path: str):
    """CSV of every timed launch since stats_reset(True)."""
    _check(lib().ct_stats_dump(path.encode()))


def stats_read() -> dict:
    """Launches since the last reset and per-class time/flops/bytes/count."""
    import numpy as np
    n = C.c_int64()
    nc = len(STAT_CLASSES)
    ms, fl, by = (np.zeros(nc) for _ in range(3))
    cnt = np.zeros(nc, np.int64)
    _check(lib().ct_stats_read(C.byref(n), ms.ctypes.data, fl.ctypes.data, by.ctypes.data,
                               cnt.ctypes.data))
    out = {"launches": int(n.value)}
    for i, name in enumerate(STAT_CLASSES):
        out[name] = {"ms": float(ms[i]), "flops": float(fl[i]), "bytes": float(by[i]),
                     "count": int(cnt[i])}
    return out


__all__ = ["CTSolve", "disk_stats", "stats_reset", "stats_read", "stats_dump", "STAT_CLASSES", "Geometry", "Opts", "SolveInfo", "CTQRError", "System", "Factor", "gemm", "lib",
           "lib_path", "make_geometry", "PRECISIONS", "SYMBOLS"]


# ---- The C entry points under their own names (the ct_ prefix dropped) -----
# Thin marshalling over the classes above; every one maps to one call of
# include/ctqr.h.

def status_str(st: int) -> str:
    """ct_status_str."""
    return lib().ct_status_str(st).decode()


def last_error() -> str:
    """ct_last_error (the calling thread's last error detail)."""
    return (lib().ct_last_error() or b"").decode()


def build_system(geom: Geometry, storage: str = "fp32", stream=None) -> System:
    """ct_build_system: A~ on the device (Sec. 2 Eq. 1)."""
    return System(geom, storage, stream)


def build_system_host(geom: Geometry, storage: str, device_budget: int, stream=None) -> System:
    """ct_build_system_host: A~ in pinned host memory, built in device slabs."""
    return System(geom, storage, stream, host_budget=device_budget)


def build_system_disk(geom: Geometry, storage: str, path: str, block_cols: int = 0,
                      host_cache: int = 1 << 30, stream=None) -> System:
    """ct_build_system_disk: A~ in a file of column blocks."""
    return System(geom, storage, stream, disk_path=path, host_cache=host_cache, block_cols=block_cols)


def system_open_disk(path: str, host_cache: int = 1 << 30, stream=None) -> System:
    """ct_system_open_disk."""
    return System.open_disk(path, host_cache, stream)


def system_info(system: System) -> dict:
    """ct_system_info: m rays, n pixels, M' rows, dense leading dimension, nnz."""
    return {"m": system.m, "n": system.n, "rows": system.rows, "lda": system.lda, "nnz": system.nnz}


def system_device_ptrs(system: System) -> dict:
    """ct_system_device_ptrs: device addresses (ints) of the dense A~ (0 once
    factored) and the CSR arrays."""
    p = [C.c_void_p() for _ in range(4)]
    _check(lib().ct_system_device_ptrs(system.h, *[C.byref(x) for x in p]))
    return dict(zip(("dense", "row_ptr", "col_idx", "val"), (x.value or 0 for x in p)))


def system_export(system: System, dense: bool = False):
    """ct_system_export: the CSR of A (row_ptr, col_idx, val) as numpy
    arrays, or with dense=True the column-major A~."""
    return system.export_dense() if dense else system.export_csr()


def forward_project(system: System, X, stream=None):
    """ct_forward_project: P = A X (X: float64 CUDA tensor (k, n) -> (k, m))."""
    return system.forward(X, stream)


def qr_factor(system: System, precision: str | None = None, **kw) -> "Factor":
    """ct_qr_factor (Sec. 2 Eq. 2); keywords as System.factor."""
    return system.factor(precision, **kw)


def qr_factor_ooc(system: System, precision: str | None = None, device_budget: int = 16 << 30,
                  **kw) -> "Factor | None":
    """ct_qr_factor_ooc (Sec. 2.2); keywords as System.factor_ooc."""
    return system.factor_ooc(precision, device_budget, **kw)


def factor_device_ptrs(factor: "Factor") -> dict:
    """ct_factor_device_ptrs: device addresses (ints) of VR and tau, and lda."""
    vr, tau, lda = C.c_void_p(), C.c_void_p(), C.c_int64()
    _check(lib().ct_factor_device_ptrs(factor.h, C.byref(vr), C.byref(lda), C.byref(tau)))
    return {"VR": vr.value or 0, "lda": lda.value, "tau": tau.value or 0}


def factor_export(factor: "Factor"):
    """ct_factor_export: (VR, tau) as numpy arrays."""
    return factor.export()


def solve(factor: "Factor", B, **kw):
    """ct_solve (Sec. 2 Eq. 3); keywords as Factor.solve."""
    return factor.solve(B, **kw)


def solve_host(factor: "Factor", B, **kw):
    """ct_solve_host; keywords as Factor.solve_host."""
    return factor.solve_host(B, **kw)


def solve_adjoint(factor: "Factor", gX, **kw):
    """ct_solve_adjoint; keywords as Factor.adjoint."""
    return factor.adjoint(gX, **kw)


def factor_save(factor: "Factor", path: str):
    """ct_factor_save."""
    factor.save(path)


def factor_load(system: System, path: str, stream=None) -> "Factor":
    """ct_factor_load."""
    return Factor.load(system, path, stream)


def disk_progress(system: System) -> tuple[int, int]:
    """ct_disk_progress: (state, done_cols)."""
    return system.disk_progress()


def host_cache_release():
    """ct_host_cache_release."""
    lib().ct_host_cache_release()


def system_free(system: System):
    """ct_system_free."""
    system.free()


def factor_free(factor: "Factor"):
    """ct_factor_free."""
    factor.free()


def gemm_noalloc(kind: str, transa: str, transb: str, M: int, N: int, K: int, alpha: float, A,
                 lda: int, B, ldb: int, beta: float, Cm, ldc: int, stream=None):
    """ct_gemm_noalloc: as gemm() for callers that cannot allocate device
    memory (the library's scratch is a fixed 16 MiB static device array);
    kinds fp64, fp32 and tf32."""
    _check(lib().ct_gemm_noalloc(GEMM_KINDS[kind], transa.encode(), transb.encode(), M, N, K, alpha,
                                 _ptr(A), lda, _ptr(B), ldb, beta, _ptr(Cm), ldc, _stream(stream)))
