"""The C ABI library builds, loads and exports every symbol include/sj.h declares.

CPU only: no compute call needs a GPU here.
"""
import ctypes
import os
import re

import pytest

from paper_2112_07552_gb300 import _build, sj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sj.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sj_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return sj.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("sj_create", "sj_topk", "sj_threshold", "sj_batch", "sj_backward",
                 "sj_destroy", "sj_contrastive_fwd", "sj_status_string", "sj_version"):
        assert want in names
    assert sorted(sj.EXPORTS) == names


def test_library_exports_every_declared_symbol(L):
    raw = ctypes.CDLL(_build.LIB)
    for name in declared_symbols():
        assert hasattr(raw, name), name


def test_status_strings_and_version(L):
    for code in range(10):
        s = L.sj_status_string(code).decode()
        assert s and s != "unknown status"
    assert L.sj_status_string(99).decode() == "unknown status"
    assert L.sj_version() >= 100


def test_invalid_arguments_are_rejected_without_device(L):
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    assert L.sj_create(None, None) == sj.SJ_ERR_INVALID_ARG
    cfg = sj.SjConfig(0, None, sj.SJ_BF16, 0, 0, 0)  # d = 0
    assert L.sj_create(ctypes.byref(h), ctypes.byref(cfg)) == sj.SJ_ERR_INVALID_ARG
    assert L.sj_topk(None, None, 0, None, 0, 1, None, None, None) == sj.SJ_ERR_INVALID_ARG
    n = sj.I64(0)
    assert L.sj_threshold(None, None, 0, None, 0, 0.5, None, 0, ctypes.byref(n), None) == \
        sj.SJ_ERR_INVALID_ARG
    assert L.sj_batch(None, None, 0, None) == sj.SJ_ERR_INVALID_ARG
    assert L.sj_destroy(None) == sj.SJ_OK


def test_struct_layouts_match_header():
    assert ctypes.sizeof(sj.SjPair) == 24
    assert ctypes.sizeof(sj.SjConfig) == 48
    assert ctypes.sizeof(sj.SjStats) == 4 * 8 + 5 * 8 + 2 * 8 + 3 * 8 + 8 + 2 * 8
    assert ctypes.sizeof(sj.SjGroup) == 32 and sj.SjGroup.sum_hi.offset == 16
    assert ctypes.sizeof(sj.SjPlanInfo) == 8 + 5 * 4 * 8 + 8


def test_relational_calls_reject_bad_arguments_without_device(L):
    n = sj.I64(0)
    assert L.sj_block(None, None, 0, None, 0, 1, 1, None, 0, ctypes.byref(n), None) == \
        sj.SJ_ERR_INVALID_ARG
    assert L.sj_join_groupby_sum(None, None, None, 0, None, None, 0, None, 0,
                                 ctypes.byref(n)) == sj.SJ_ERR_INVALID_ARG
    assert L.sj_join_sum_product(None, None, None, 0, None, None, 0, None) == \
        sj.SJ_ERR_INVALID_ARG


def test_header_is_plain_c():
    """include/sj.h compiles as pedantic C99 (the ABI serves C callers)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    out = subprocess.run([gcc, "-fsyntax-only", "-std=c99", "-Wall", "-Wextra", "-pedantic",
                          "-Werror", "-x", "c", os.path.join(ROOT, "include", "sj.h")],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
