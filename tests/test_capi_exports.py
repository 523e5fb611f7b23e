"""The C ABI library builds for sm_103a, loads, and exports every declared entry point.

No compute calls: this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(cse_[a-z0-9_]+)\s*\(",
                                 txt, flags=re.M):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2212_10042_gb300 import build
    return build.build()


def test_declared_symbols_exported(libpath):
    names = _declared()
    assert {"cse_create", "cse_destroy", "cse_simulate_tiles", "cse_validate", "cse_calibrate",
            "cse_step", "cse_score_backward", "cse_status_str", "cse_validate_lower",
            "cse_validate_band", "cse_validate_rand", "cse_calibrate_rand"} <= names
    lib = ctypes.CDLL(libpath)
    for n in sorted(names):
        assert hasattr(lib, n), "missing export " + n


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.cse_status_str.restype = ctypes.c_char_p
    assert lib.cse_status_str(0) == b"ok"
    assert lib.cse_status_str(-1) == b"invalid argument"
    assert lib.cse_status_str(12345) == b"unknown status"


def test_invalid_arguments_rejected_on_host(libpath):
    # argument checks happen on the host before any CUDA call
    from paper_2212_10042_gb300 import binding as B
    lib = B.lib()
    h = ctypes.c_void_p()
    assert lib.cse_create(None, None, 0, 16, None) == -1
    D = B.cse_design()
    D.stat, D.d, D.n_looks = 1, 2, 1
    D.look_n[0] = 100
    assert lib.cse_create(ctypes.byref(h), ctypes.byref(D), 0, 0, None) == -1          # K_max < 1
    D.look_n[0] = 500
    assert lib.cse_create(ctypes.byref(h), ctypes.byref(D), 0, 16, None) == -2         # n_max > 128
    D.look_n[0] = 100
    D.d = 3
    assert lib.cse_create(ctypes.byref(h), ctypes.byref(D), 0, 16, None) == -2         # d mismatch
    # basket design: one analysis, n_max <= 63, finite null logits
    D.stat, D.d, D.n_looks = 3, 4, 1
    D.look_n[0] = 70
    assert lib.cse_create(ctypes.byref(h), ctypes.byref(D), 0, 16, None) == -2         # table too large
    D.look_n[0], D.look_n[1], D.n_looks = 10, 35, 2
    assert lib.cse_create(ctypes.byref(h), ctypes.byref(D), 0, 16, None) == -2         # two analyses
    D.look_n[0], D.n_looks = 35, 1
    D.arm_null[2] = float("nan")
    assert lib.cse_create(ctypes.byref(h), ctypes.byref(D), 0, 16, None) == -2         # null logit NaN
    assert lib.cse_score_backward(-1, 2, None, None, None, None, None) == -1
    assert lib.cse_sync(None, None) == -1
    assert lib.cse_profile_only(None, b"sim_ztest") == -1
    assert lib.cse_type1_error(None, 4, None, None, None, 16, -1.96, None, None, None, None, None) == -1
    # the pipe probes check their arguments before any CUDA call
    assert lib.cse_probe_peak(99, 1, 1, 1, None, None, None) == -1                     # unknown pipe
    assert lib.cse_probe_peak(0, 0, 1, 1, None, None, None) == -1                      # no blocks
    assert lib.cse_probe_peak(0, 1, 1 << 21, 1, None, None, None) == -1                # iters too large


def test_oracle_is_not_linked_into_the_product(libpath):
    # the CUDA library and the oracle share no code: no oracle symbol in the product
    out = os.popen("nm -D --defined-only %s" % libpath).read()
    assert "orc_" not in out
    src = os.path.join(ROOT, "paper_2212_10042_gb300")
    for dirpath, _, files in os.walk(src):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
