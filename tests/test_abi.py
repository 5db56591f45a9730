"""CPU checks of the C ABI boundary: the library builds, loads and exports every
entry point declared in include/*.h.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(asdsm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    return asdsm.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("asdsm_setup", "asdsm_solve", "asdsm_residual", "asdsm_destroy", "asdsm_initial_guess",
                     "asdsm_submesh_solve", "asdsm_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_structs_match_the_header_layout(lib):
    from paper_2303_01163_gb300 import asdsm
    assert ctypes.sizeof(asdsm.Desc) == 4 * 4 + 6 * 8
    assert ctypes.sizeof(asdsm.Opts) == 8 + 4 * 4 + 8 + 8 + 8 + 4 + 4 + 8
    assert ctypes.sizeof(asdsm.Stats) == 4 * 4 + 4 * 8 + 8 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(asdsm.KProf) == 24 + 2 * 8 + 3 * 8


def test_strerror_and_defaults_need_no_gpu(lib):
    from paper_2303_01163_gb300 import asdsm
    assert lib.asdsm_strerror(0) == b"ok"
    assert b"invalid" in lib.asdsm_strerror(-1)
    o = asdsm.default_opts()
    assert o.tol == 1e-10 and o.accel_m == 8 and o.precision == asdsm.MIXED


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    from paper_2303_01163_gb300 import asdsm
    h = ctypes.c_void_p()
    assert lib.asdsm_setup(None, None, None, ctypes.byref(h)) == asdsm.ERR_INVALID
    d = asdsm.Desc()
    d.d, d.n, d.mc = 2, 66, 8              # N-1 = 65 is not a power of two
    d.alpha[0] = d.alpha[1] = 1.0
    assert lib.asdsm_setup(ctypes.byref(d), None, None, ctypes.byref(h)) == asdsm.ERR_INVALID
    d.n, d.mc = 65, 3                      # mc not a power of two
    assert lib.asdsm_setup(ctypes.byref(d), None, None, ctypes.byref(h)) == asdsm.ERR_INVALID
    d.n, d.mc = 65537, 4096                # N above 32769 (grid offsets beyond 32 bits)
    assert lib.asdsm_setup(ctypes.byref(d), None, None, ctypes.byref(h)) == asdsm.ERR_INVALID
    d.n, d.mc = 65, 8
    d.alpha[0] = 0.0                       # alpha must be positive
    assert lib.asdsm_setup(ctypes.byref(d), None, None, ctypes.byref(h)) == asdsm.ERR_INVALID
    assert lib.asdsm_solve(None, None, None, None) == asdsm.ERR_INVALID
    lib.asdsm_destroy(None)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2303_01163_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, flags=re.M), path


def _tune_check(lib, entries):
    arr = (ctypes.c_int32 * len(entries))(*entries)
    return lib.asdsm_tune_check(arr, len(entries))


def test_saved_tuning_passes_the_check_and_bad_entries_fail(lib):
    import json
    saved = json.load(open(os.path.join(ROOT, "profiles", "tune_state_4097_mixed.json")))
    assert len(saved) == 130
    assert _tune_check(lib, saved) == 0
    assert _tune_check(lib, [0] * 130) == 0
    assert _tune_check(lib, saved[:129]) == -1                      # wrong count
    good = list(saved)
    good[65], good[66] = (128 << 8) | 2, (128 << 8) | 4               # tcgen05 kernel split 2 and 4 ways
    assert _tune_check(lib, good) == 0
    for index, value in [(0, (48 << 8) | 1),       # rows per CTA not in {16, 64}
                         (1, (16 << 8) | 3),       # split factor not a power of two up to 8
                         (2, (128 << 8) | 1),      # tcgen05 kernel in the FP64 half
                         (3, (32 << 8) | 1),       # mma.sync kernel in the FP64 half
                         (65, (128 << 8) | 8),     # tcgen05 kernel split 8 ways (1, 2 or 4 only)
                         (66, (32 << 8) | 2),      # mma.sync kernel split
                         (64, 16),                 # tensor-core Filler in the FP64 half
                         (129, 9),                 # Filler warps above 8
                         (70, -1)]:
        bad = list(saved)
        bad[index] = value
        assert _tune_check(lib, bad) == -1, (index, value)
