"""The C-ABI library loads and exports every entry point include/mis2.h
declares (no GPU needed: only calls that touch no device)."""
import ctypes
import os
import re

import pytest

from paper_2204_02934_gb300 import _build, mis2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mis2_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return mis2._lib()


def test_header_declares_the_binding_exports():
    assert _declared() == set(mis2.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_host_only_calls(lib):
    cfg = mis2.mis2_config_default()
    assert cfg.hash_variant == 0 and cfg.agg_mode == 0 and cfg.block_size == 256
    assert cfg.warp_degree <= cfg.block_degree and cfg.spin_limit > 0
    assert mis2.mis2_status_string(0) == "MIS2_OK"
    assert mis2.mis2_status_string(-5) == "MIS2_ERR_TIMEOUT"
    assert mis2.mis2_version().count(".") == 2


def test_struct_sizes_match_header():
    # int64 n, nnz; int32 x2; two pointers
    assert ctypes.sizeof(mis2.mis2_csr) == 40
    assert ctypes.sizeof(mis2.mis2_config) == 56
    assert ctypes.sizeof(mis2.mis2_stats) == 4 + 4 + 8 * 4 + 2 * 64 * 4 * 8 + 8 * 8 + 8 * 8 + 8 + 2 * (4 + 4 * 64) * 8


def test_null_context_is_rejected(lib):
    nr = ctypes.c_int64(0)
    assert lib.mis2_run(None, None, 0, None, None, ctypes.byref(nr), None, None) == -1


def test_debug_bits_match_the_header():
    hdr = open(os.path.join(ROOT, "include", "mis2.h")).read()
    for name in ("MIS2_DEBUG_VALIDATE", "MIS2_DEBUG_FORCE_TIMEOUT"):
        m = re.search(r"#define\s+" + name + r"\s+(0x[0-9a-fA-F]+|\d+)", hdr)
        assert m, name
        assert int(m.group(1), 0) == getattr(mis2, name)


def test_every_status_code_has_a_name():
    hdr = open(os.path.join(ROOT, "include", "mis2.h")).read()
    codes = dict((name, int(val)) for name, val in re.findall(r"(MIS2_(?:OK|ERR_[A-Z_]+))\s*=\s*(-?\d+)", hdr))
    assert "MIS2_ERR_CANCELLED" in codes and len(codes) >= 8
    for name, val in codes.items():
        assert mis2.mis2_status_string(val) == name
        assert mis2.STATUS[val] == name  # the binding's error text names it too
    assert mis2.mis2_status_string(-99) == "MIS2_ERR_UNKNOWN"


def test_ablation_bits_match_the_header():
    hdr = open(os.path.join(ROOT, "include", "mis2.h")).read()
    for name in ("MIS2_ABLATE_NO_WORKLISTS", "MIS2_ABLATE_TUPLE_ENGINE", "MIS2_ABLATE_UNPACKED_TUPLES"):
        m = re.search(r"#define\s+" + name + r"\s+(0x[0-9a-fA-F]+|\d+)", hdr)
        assert m, name
        assert int(m.group(1), 0) == getattr(mis2, name)
