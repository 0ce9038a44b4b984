"""The C-ABI library builds, loads and exports every entry point that
include/ctp.h declares; host-side argument checks reject bad calls before any
device work (these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1305_2353_gb300 import build as B
from paper_1305_2353_gb300 import ctp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ctp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctp.load()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "ctp_factor_supernode" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(ctp.EXPORTS)


def test_max_p(lib):
    assert lib.ctp_max_p() == 256


def test_host_argument_checks(lib):
    opt = ctp.options()
    sz = ctypes.c_size_t()
    # null context
    assert lib.ctp_workspace_size(None, 100, 10, ctypes.byref(opt), ctypes.byref(sz)) == ctp.CTP_EINVAL
    assert lib.ctp_factor_supernode(None, 100, 10, None, 100, ctypes.byref(opt), None, None, None,
                                    None, None, 0, None, 0, None) == ctp.CTP_EINVAL
    assert lib.ctp_compress_strict(None, 10, 4, None, 10, None, None, None, 0, None) == ctp.CTP_EINVAL
    assert lib.ctp_read_info(None, None, None, None) == ctp.CTP_EINVAL


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.ctp_create(ctypes.byref(h), 0) == ctp.CTP_ECUDA
    assert not h.value


def test_system_entry_points_check_arguments(lib):
    sz = ctypes.c_size_t()
    assert lib.ctp_solve_workspace_size(-1, 1, ctypes.byref(sz)) == ctp.CTP_EINVAL
    assert lib.ctp_solve_workspace_size(100, 0, ctypes.byref(sz)) == ctp.CTP_EINVAL
    assert lib.ctp_solve_workspace_size(100, 2, ctypes.byref(sz)) == ctp.CTP_OK and sz.value > 0
    assert lib.ctp_refine_workspace_size(0, 10, 1, ctypes.byref(sz)) == ctp.CTP_EINVAL
    assert lib.ctp_solve(None, 0, None, 10, 1, None, 10, None, 0, None) == ctp.CTP_EINVAL
    assert lib.ctp_backward_error(None, 10, None, 10, 1, None, 10, None, 10, None, None, 0,
                                  None) == ctp.CTP_EINVAL
    steps = ctypes.c_int32()
    assert lib.ctp_refine(None, 0, None, 10, None, 10, 1, None, 10, None, 10, 10, 1e-14, None,
                          ctypes.byref(steps), None, 0, None) == ctp.CTP_EINVAL
    opt = ctp.options()
    h = ctypes.c_void_p()
    assert lib.ctp_factor_dense(None, 10, None, 10, 4, ctypes.byref(opt), 4, ctypes.byref(opt),
                                ctypes.byref(h), None) == ctp.CTP_EINVAL
    nf = ctypes.c_int32()
    arr = ctypes.c_void_p()
    assert lib.ctp_chain_fronts(None, ctypes.byref(nf), ctypes.byref(arr)) == ctp.CTP_EINVAL
    assert lib.ctp_chain_destroy(None) == ctp.CTP_OK


def test_sfront_mirror_matches_header():
    """The Python mirror of ctp_sfront has the header's field order and size."""
    assert ctypes.sizeof(ctp.SFront) == 8 + 4 + 4 + 8 + 8 + 5 * 8
    assert [f for f, _ in ctp.SFront._fields_] == ["n", "p", "reserved", "L", "ldl", "perm", "piv",
                                                  "D", "nelim", "rows"]


def test_tuning_knobs_check_arguments(lib):
    v = ctypes.c_int32()
    assert lib.ctp_tune_set(None, 0, 0) == ctp.CTP_EINVAL
    assert lib.ctp_tune_get(None, 0, ctypes.byref(v)) == ctp.CTP_EINVAL
    assert lib.ctp_autotune_batch(None, 1, None, None, None, None, None, 1, None, 1, None, None,
                                  None, None) == ctp.CTP_EINVAL
    assert lib.ctp_autotune_supernode(None, 10, 2, None, 10, None, None, None, None, None, None, 0,
                                      None, 0, 1, None, 1, None, None, None, None) == ctp.CTP_EINVAL


def test_row_split_entry_points_check_arguments(lib):
    sz = ctypes.c_size_t()
    assert lib.ctp_relaxed_candidates_size(0, 4, ctypes.byref(sz)) == ctp.CTP_EINVAL
    assert lib.ctp_relaxed_candidates_size(9, 4, ctypes.byref(sz)) == ctp.CTP_EUNSUPPORTED
    assert lib.ctp_relaxed_candidates_size(2, 257, ctypes.byref(sz)) == ctp.CTP_EUNSUPPORTED
    assert lib.ctp_relaxed_candidates_size(8, 256, ctypes.byref(sz)) == ctp.CTP_OK
    # 256-byte info word, then (16-byte candidate) x p x P x p lists and P x p lengths
    assert sz.value == 256 + 16 * 256 * 8 * 256 + 4 * 256 * 8
    assert lib.ctp_compress_strict_merge(None, 2, 4, None, 16, None, None) == ctp.CTP_EINVAL
    assert lib.ctp_compress_relaxed_candidates(None, 10, 4, None, 10, 0, 2, 0, None, 0,
                                               None) == ctp.CTP_EINVAL
    assert lib.ctp_compress_relaxed_select(None, 2, 4, None, 0, None, None) == ctp.CTP_EINVAL
    assert lib.ctp_gather_rows(None, 4, None, 10, None, None, None) == ctp.CTP_EINVAL
