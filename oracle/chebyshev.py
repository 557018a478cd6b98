"""Chebyshev polynomials of the first kind and the exp-semicircle filter (oracle).

Definitions follow Appendix A (Eqs. cheb, cheb2, rec) and Sec. II A
(Eqs. F, filter): the piecewise closed form, the three-term recurrence and the
map F(x) = (x^2 - E_c)/E_0 with E_c = (E_max^2 + a^2)/2, E_0 = (E_max^2 - a^2)/2.
"""

from __future__ import annotations

import numpy as np


def cheb_closed(k: int, x):
    """T_k(x) from the piecewise definition of Appendix A (Eq. cheb)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(k * np.arccos(x[inside]))
    hi = x > 1.0
    out[hi] = np.cosh(k * np.arccosh(x[hi]))
    lo = x < -1.0
    out[lo] = (-1.0) ** k * np.cosh(k * np.arccosh(-x[lo]))
    return out


def cheb_recurrence(k: int, x):
    """T_k(x) from T_0 = 1, T_1 = x and T_{k+1} = 2x T_k - T_{k-1} (Eq. rec)."""
    x = np.asarray(x, dtype=np.float64)
    t0 = np.ones_like(x)
    if k == 0:
        return t0
    t1 = x.copy()
    for _ in range(1, k):
        t0, t1 = t1, 2.0 * x * t1 - t0
    return t1


def filter_map(x, emax: float, a: float):
    """F(x) = (x^2 - E_c)/E_0 (Eq. F)."""
    ec = (emax * emax + a * a) / 2.0
    e0 = (emax * emax - a * a) / 2.0
    return (np.asarray(x, dtype=np.float64) ** 2 - ec) / e0


def filter_exact(x, emax: float, a: float, K: int):
    """T_K(F(x)), the exact filter response (solid lines of Fig. 1)."""
    return cheb_closed(K, filter_map(x, emax, a))


def filter_approx(x, emax: float, a: float, K: int):
    """exp((2K/E_max) sqrt(a^2 - x^2)) for |x| <= a (Eq. filter, dashed lines of Fig. 1)."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(2.0 * K / emax * np.sqrt(np.maximum(a * a - x * x, 0.0)))


def basis_orders(a_r: float, n: int) -> np.ndarray:
    """Chebyshev orders of the basis (Eq. set2): [0, k_1-1, k_1, ..., k_n-1, k_n].

    k_m = floor(m*pi/a_r), m = 1..n (Sec. II B and Appendix C). Since a_r < 1,
    consecutive k_m differ by at least 3, so the list never repeats an order.
    """
    ks = [int(np.floor(m * np.pi / a_r)) for m in range(1, n + 1)]
    x = [0]
    for k in ks:
        x += [k - 1, k]
    return np.array(x, dtype=np.int64)
