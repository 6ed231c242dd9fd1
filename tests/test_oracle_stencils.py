"""Pins of the oracle's derived stencils (Sec. II.B.1, II.B.2, II.C.2, II.D):
each weight set must be exact on the polynomials its order promises and fail
on the first degree beyond, so a dropped or transposed weight is caught."""
import numpy as np
import pytest

import oracle as O


def _apply(w, nodes, f):
    return sum(wi * f(s) for wi, s in zip(w, nodes))


@pytest.fixture(scope="module")
def st():
    return O.stencils()


def test_central_first_derivative_sixth_order(st):
    nodes = np.arange(-3, 4)
    for m in range(0, 7):
        exact = 1.0 if m == 1 else 0.0
        assert abs(_apply(st["c1"], nodes, lambda s: s ** m) - exact) < 1e-12
    # degree 7 is not differentiated exactly -> 6th order, not higher
    assert abs(_apply(st["c1"], nodes, lambda s: s ** 7)) > 1.0
    assert np.allclose(st["c1"], -st["c1"][::-1])


def test_central_second_derivative_sixth_order(st):
    nodes = np.arange(-3, 4)
    for m in range(0, 8):
        exact = 2.0 if m == 2 else 0.0
        assert abs(_apply(st["c2"], nodes, lambda s: s ** m) - exact) < 1e-11
    assert abs(_apply(st["c2"], nodes, lambda s: s ** 8)) > 1.0


def test_lopsided_upwind_stencil(st):
    nodes = np.arange(-2, 5)
    for m in range(0, 7):
        exact = 1.0 if m == 1 else 0.0
        assert abs(_apply(st["lop"], nodes, lambda s: s ** m) - exact) < 1e-11
    # the 60ths of the published 6th-order lopsided operator
    assert np.allclose(st["lop"] * 60.0, [2, -24, -35, 80, -30, 8, -1], atol=1e-10)


def test_ko_eighth_difference(st):
    nodes = np.arange(-4, 5)
    for m in range(0, 8):
        assert abs(_apply(st["ko"], nodes, lambda s: s ** m)) < 1e-8
    # Nyquist mode (-1)^j: the 8th difference is +256 at j = 0, so the
    # dissipation term -(eps/256) D^8 Q damps it at rate eps/dx
    assert abs(_apply(st["ko"], nodes, lambda s: (-1.0) ** s) - 256.0) < 1e-9


def test_face_interpolation_sixth_order(st):
    nodes = np.arange(-2, 4)
    for m in range(0, 6):
        assert abs(_apply(st["face6"], nodes, lambda s: s ** m) - 0.5 ** m) < 1e-13
    assert np.allclose(st["face6"] * 256.0, [3, -25, 150, 150, -25, 3])


def test_prolongation_restriction_eighth_order(st):
    nodes = np.arange(-3, 5)
    for m in range(0, 8):
        assert abs(_apply(st["prol8"], nodes, lambda s: s ** m) - 0.25 ** m) < 1e-12
        assert abs(_apply(st["rest8"], nodes, lambda s: s ** m) - 0.5 ** m) < 1e-12
    assert abs(_apply(st["rest8"], nodes, lambda s: s ** 8) - 0.5 ** 8) > 1e-3


def test_generic_lagrange_and_fd():
    rng = np.random.default_rng(1)
    nodes = np.sort(rng.uniform(-3, 3, 5))
    x = 0.37
    w = O.lagrange(nodes, x)
    c = rng.normal(size=5)
    poly = np.polynomial.Polynomial(c)
    assert abs(np.dot(w, poly(nodes)) - poly(x)) < 1e-10
    wd = O.fd_weights(nodes, x, 2)
    assert abs(np.dot(wd, poly(nodes)) - poly.deriv(2)(x)) < 1e-8
