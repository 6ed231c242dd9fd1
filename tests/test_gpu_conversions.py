"""The integer-only FP64 -> FP32 views the mixed-precision kernels take of the
FP64 state (split into hi + lo, rounding to FP32, exact widening), checked
against the hardware conversions and against exact arithmetic on the host."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probe():
    from paper_2502_03223_gb300 import build as B
    B.build()
    lib = C.CDLL(B.PROBE)
    fp, dp = C.POINTER(C.c_float), C.POINTER(C.c_double)
    lib.sacra_probe_split.argtypes = [dp, C.c_int, fp, fp, fp, fp, dp]
    lib.sacra_probe_split.restype = C.c_int

    def run(u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        n = u.size
        hi, lo, f, hw = (np.empty(n, np.float32) for _ in range(4))
        back = np.empty(n, np.float64)
        args = [a.ctypes.data_as(fp) for a in (hi, lo, f, hw)]
        assert lib.sacra_probe_split(u.ctypes.data_as(dp), n, *args, back.ctypes.data_as(dp)) == 0
        return hi, lo, f, hw, back
    return run


def _values(rng, n=20000):
    mag = 10.0 ** rng.uniform(-30, 30, n)
    u = mag * rng.choice([-1.0, 1.0], n)
    # values that sit on FP32 rounding boundaries and powers of two
    ties = np.float32(rng.uniform(1, 2, 200)).astype(np.float64) * (1 + 2.0 ** -24)
    return np.concatenate([u, ties, 2.0 ** np.arange(-100, 100), [0.0, -0.0, 1.0, -1.0]])


def test_split_is_exact_to_46_bits(probe):
    u = _values(np.random.default_rng(1))
    hi, lo, f, hw, back = probe(u)
    h = hi.astype(np.float64)
    # hi: truncation to 24 significant bits (never larger in magnitude, within one FP32 ulp)
    assert np.all(np.abs(h) <= np.abs(u))
    assert np.all(np.abs(u - h) <= np.spacing(np.abs(hi)).astype(np.float64))
    assert np.all(np.sign(h[h != 0]) == np.sign(u[h != 0]))
    ok = np.abs(u) > 2.0 ** -100
    r = u - (h + lo.astype(np.float64))
    assert np.all(np.abs(r[ok]) <= 2.0 ** -46 * np.abs(u[ok]))


def test_rounding_matches_hardware(probe):
    u = _values(np.random.default_rng(2))
    hi, lo, f, hw, back = probe(u)
    normal = np.abs(u) >= 2.0 ** -126
    # round to nearest of the 47-bit hi + lo: equal to the hardware rounding of u,
    # except where u is within 2^-46 of a tie (the exactly-constructed ties above)
    same = f[normal] == hw[normal]
    assert same.mean() > 0.99
    diff_ulp = np.abs(f[normal].astype(np.float64) - hw[normal]) / np.spacing(np.abs(hw[normal])).astype(np.float64)
    assert np.all(diff_ulp <= 1.0)
    assert np.all(f[~normal] == 0.0)
    # widening back to FP64 is exact
    assert np.all(back == 0.0)


def test_difference_of_nearby_values_is_one_rounding(probe):
    rng = np.random.default_rng(3)
    base = 10.0 ** rng.uniform(-8, 8, 5000) * rng.choice([-1.0, 1.0], 5000)
    v = base * (1.0 + rng.uniform(1e-5, 1e-3, 5000) * rng.choice([-1.0, 1.0], 5000))
    hb, lb, _, _, _ = probe(base)
    hv, lv, _, _, _ = probe(v)
    # the FP32 difference the kernels form: (hi_a - hi_b) + (lo_a - lo_b)
    d32 = (hv - hb) + (lv - lb)
    exact = v - base
    rel = np.abs(d32.astype(np.float64) - exact) / np.abs(exact)
    assert np.max(rel) < 1.2e-7          # one FP32 rounding (2^-24) plus 2^-46 |u| / |difference|
