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


def test_parameter_checks_of_the_eos_variants_and_boundaries(lib_path):
    L = S.load(lib_path)
    from paper_2502_03223_gb300 import workloads as W
    cfg, _ = W.config_tov_stable()
    n = ctypes.c_size_t(0)

    def ok(**kw):
        import dataclasses
        p = S.make_params(dataclasses.replace(cfg, **kw))
        return L.sacra_arena_bytes(ctypes.byref(p), ctypes.byref(n)) == 0

    assert ok(pwp=((1e-4, 2.5), (8e-4, 3.0)))
    assert not ok(pwp=((8e-4, 2.5), (1e-4, 3.0)))          # transitions must increase
    assert not ok(pwp=((1e-4, 1.0),))                      # Gamma_i > 1
    p = S.make_params(cfg)
    p.n_pieces = 9                                         # at most 8 pieces
    assert L.sacra_arena_bytes(ctypes.byref(p), ctypes.byref(n)) == -1
    assert ok(eos_adiabatic=1) and not ok(eos_adiabatic=1, K=0.0) and not ok(eos_adiabatic=2)
    assert not ok(r_hold=-1.0) and not ok(hydro_outer=2) and not ok(subcycle_from=-1)
    assert ok(bssn=1) and not ok(bssn=2) and not ok(bssn=-1)
    # the allocation-free entry point has no device memory for a piece table
    p = S.make_params(dataclasses_replace(cfg, n_levels=1, pwp=((1e-4, 2.5),)))
    null = ctypes.c_void_p(1)
    assert L.sacra_hydro_rhs_noalloc(ctypes.byref(p), 0, null, null, null, None) == -1


def dataclasses_replace(cfg, **kw):
    import dataclasses
    return dataclasses.replace(cfg, **kw)
