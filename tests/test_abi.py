"""The C ABI library loads without a GPU and exports every entry point that
include/ctqr.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ctqr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ct_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for want in ("ct_build_system", "ct_qr_factor", "ct_solve", "ct_solve_adjoint",
                 "ct_solve_host", "ct_gemm"):
        assert want in syms


def test_library_exports_every_declared_symbol():
    import paper_2412_07631_b300 as ct
    L = ctypes.CDLL(ct.lib_path() if os.path.exists(ct.lib_path()) else ct.build.build())
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing
    assert set(declared_symbols()) == set(ct.SYMBOLS)


def test_status_strings_without_gpu():
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    assert L.ct_status_str(0) == b"CT_OK"
    assert L.ct_status_str(4) == b"CT_ERR_RANK"


def test_bad_arguments_are_rejected_without_touching_the_device():
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    h = ctypes.c_void_p()
    g = ct.make_geometry(0, 10, 10)
    assert L.ct_build_system(ctypes.byref(g), 0, None, ctypes.byref(h)) == 1
    g = ct.make_geometry(64, 2, 8)  # fewer rays than pixels, no regularisation rows
    assert L.ct_build_system(ctypes.byref(g), 0, None, ctypes.byref(h)) == 1
    assert L.ct_solve(None, None, 0, 1, None, 0, None, None, None) == 1
    assert L.ct_gemm(7, b"N", b"N", 1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1, None) == 1
