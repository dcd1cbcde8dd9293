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
    assert L.ct_debug_check_canaries(0, None, None) == 1
    assert L.ct_debug_canaries(0) == 0


def test_disk_tier_refuses_bad_files_and_blocks_without_a_gpu(tmp_path):
    """The disk tier checks its file header and block width before any
    device work: a missing file, a foreign file, a header whose checksum does
    not match and a block width that is not a multiple of 32 are refused."""
    import paper_2412_07631_b300 as ct
    L = ct.lib()
    h = ctypes.c_void_p()
    assert L.ct_system_open_disk(str(tmp_path / "none").encode(), 0, None, ctypes.byref(h)) == 1
    foreign = tmp_path / "foreign.bin"
    foreign.write_bytes(bytes(range(256)) * 32)
    assert L.ct_system_open_disk(str(foreign).encode(), 0, None, ctypes.byref(h)) == 1
    # right magic and version, wrong checksum
    bad = tmp_path / "bad.ctqrd"
    bad.write_bytes(b"CTQRDSK1" + (1).to_bytes(4, "little") + (4).to_bytes(4, "little") + bytes(4080))
    assert L.ct_system_open_disk(str(bad).encode(), 0, None, ctypes.byref(h)) == 1
    assert b"checksum" in L.ct_last_error()
    assert not h.value
    g = ct.make_geometry(16, 30, 24, 0.05)
    assert L.ct_build_system_disk(ctypes.byref(g), 1, str(tmp_path / "x").encode(), 33, 0, None,
                                  ctypes.byref(h)) == 1
    assert L.ct_build_system_disk(ctypes.byref(g), 1, None, 64, 0, None, ctypes.byref(h)) == 1
    assert L.ct_status_str(11) == b"CT_ERR_IO"
    assert L.ct_status_str(12) == b"CT_ERR_INTERRUPTED"


def test_every_entry_point_cites_its_passage():
    """Each declaration's comment names the passage of the paper that defines
    the operation (a section or an equation), or says that the paper has no
    counterpart, and states its errors or that it cannot fail."""
    text = open(os.path.join(ROOT, "include", "ctqr.h")).read()
    uncited = []
    for m in re.finditer(r"CT_API[^;(]*?\b(ct_[a-z_0-9]+)\s*\(", text):
        end = text.rfind("*/", 0, m.start())
        comment = text[text.rfind("/*", 0, end):end]
        comment = re.sub(r"\s*\n\s*\*\s?", " ", comment)
        if not re.search(r"Sec\. \d|Eq\. \d|no counterpart", comment):
            uncited.append(m.group(1))
        if not re.search(r"Errors|CT_ERR_|CT_OK|Cannot fail", comment):
            uncited.append(m.group(1) + " (errors)")
    assert not uncited, uncited


def test_binding_names_every_entry_point():
    """The Python binding carries each C entry point under its own name (the
    ct_ prefix dropped)."""
    import paper_2412_07631_b300 as ct
    missing = [s for s in declared_symbols() if not callable(getattr(ct, s[3:], None))]
    assert not missing, missing
    assert ct.status_str(4) == "CT_ERR_RANK"
    assert isinstance(ct.last_error(), str)


def _struct_fields(text, name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    m = re.search(r"typedef struct \{([^{}]*)\} " + name + ";", text, re.S)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    return [re.split(r"\s+", d.strip())[-1] for d in body.split(";") if d.strip()]


def test_binding_structs_match_the_header():
    """The ctypes structures mirror the header's structs field by field (names,
    order and sizes), so the library reads what the binding writes."""
    import ctypes
    import paper_2412_07631_b300 as ct
    text = open(os.path.join(ROOT, "include", "ctqr.h")).read()
    for cls, name in ((ct.Opts, "ct_opts"), (ct.SolveInfo, "ct_solve_info"), (ct.Geometry, "ct_geometry")):
        assert [f for f, _ in cls._fields_] == _struct_fields(text, name), name
    # the ABI sizes the library was built with (x86-64 System V alignment)
    assert ctypes.sizeof(ct.Opts) == 40 and ctypes.sizeof(ct.Geometry) == 80
