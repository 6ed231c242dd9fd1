"""The C-ABI library builds for sm_103a here (no GPU needed), loads, and
exports every entry point include/sacra2d.h declares."""
import ctypes
import os
import re

import pytest

from paper_2502_03223_gb300 import build as B
from paper_2502_03223_gb300 import sacra2d as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def _declared():
    txt = open(os.path.join(ROOT, "include", "sacra2d.h")).read()
    return sorted(set(re.findall(r"\b(sacra_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_binding_exports():
    assert sorted(S.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_arena_size_and_argument_checks(lib_path):
    L = S.load(lib_path)
    from paper_2502_03223_gb300 import workloads as W
    cfg, _ = W.config_tov_stable()
    p = S.make_params(cfg)
    n = ctypes.c_size_t(0)
    assert L.sacra_arena_bytes(ctypes.byref(p), ctypes.byref(n)) == 0
    assert n.value > 3 * 30 * 4 * 272 * 272 * 8
    p.n_levels = 0
    assert L.sacra_arena_bytes(ctypes.byref(p), ctypes.byref(n)) == -1
    p.n_levels = 3
    p.nx = 255      # odd N with FMR is rejected
    assert L.sacra_arena_bytes(ctypes.byref(p), ctypes.byref(n)) == -1
