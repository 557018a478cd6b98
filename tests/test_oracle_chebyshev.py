"""Pins for the scalar Chebyshev definitions and the exp-semicircle filter (Fig. 1)."""

import math

import numpy as np

from oracle import chebyshev as C
from tests.conftest import read_golden


def test_closed_form_equals_recurrence():
    x = np.linspace(-1.6, 1.6, 161)
    for k in range(0, 41):
        a = C.cheb_closed(k, x)
        b = C.cheb_recurrence(k, x)
        assert np.allclose(a, b, rtol=1e-9, atol=1e-9), k


def test_low_orders():
    x = np.linspace(-2, 2, 9)
    assert np.allclose(C.cheb_recurrence(2, x), 2 * x * x - 1)
    assert np.allclose(C.cheb_recurrence(3, x), 4 * x ** 3 - 3 * x)
    assert np.allclose(C.cheb_closed(5, x), 16 * x ** 5 - 20 * x ** 3 + 5 * x)


def test_product_identity_scalar():
    x = np.linspace(-1, 1, 33)
    for i, j in [(3, 7), (10, 2), (5, 5), (0, 9)]:
        lhs = C.cheb_closed(i, x) * C.cheb_closed(j, x)
        rhs = 0.5 * (C.cheb_closed(i + j, x) + C.cheb_closed(abs(i - j), x))
        assert np.allclose(lhs, rhs, atol=1e-12)


def test_fig1_filter_peak_and_shape():
    """Fig. 1: E_max = 1, k a = 24. At x = 0, F(0) = -(1+a^2)/(1-a^2) = -cosh(2 atanh a),
    so T_K(F(0)) = (-1)^K cosh(2 K atanh a); the dashed approximation gives exp(2 K a)."""
    for a_s, ka_s in read_golden("fig1_filter.txt"):
        a, K = float(a_s), int(round(float(ka_s) / float(a_s)))
        peak = C.filter_exact(np.array([0.0]), 1.0, a, K)[0]
        closed = (-1) ** K * math.cosh(2 * K * math.atanh(a))
        assert abs(peak - closed) < 1e-9 * abs(closed)
        # Eq. filter: log|T_K(F(x))| ~ 2K sqrt(a^2 - x^2) inside the window
        xs = np.linspace(0, 0.5 * a, 6)
        ex = np.log(np.abs(C.filter_exact(xs, 1.0, a, K)))
        ap = np.log(C.filter_approx(xs, 1.0, a, K))
        assert np.all(np.abs(ex - ap) < 0.03 * ap)
        # outside the window the filter is bounded by 1
        xo = np.linspace(a * 1.0001, 1.0, 200)
        assert np.all(np.abs(C.filter_exact(xo, 1.0, a, K)) <= 1.0 + 1e-9)


def test_basis_orders():
    a_r = 0.0123
    x = C.basis_orders(a_r, 7)
    assert len(x) == 15 and x[0] == 0
    for m in range(1, 8):
        km = math.floor(m * math.pi / a_r)
        assert x[2 * m] == km and x[2 * m - 1] == km - 1
    assert np.all(np.diff(x) > 0)
