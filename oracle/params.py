"""Parameter selection for DACP (oracle): E_max bound, window a, basis size n, order K.

Sec. III: E_max comes from an "upper-bound estimator" costing little extra
computation (the paper cites Zhou & Li 2011, which bounds the largest
eigenvalue by lambda_max(T_k) + ||f_k|| after k Lanczos steps); E_min = -E_max.
The window a is chosen from an estimate of the density of states so that
[-a, a] holds a little more levels than requested; the basis obeys
2n+1 = 1.5 d (Sec. II B); the filter order is K = 18 E_max / a (Sec. II A).

Readings (the paper only cites these estimators):
  * Lanczos: 20 steps without reorthogonalisation from one start vector;
    bound = max(|theta_min|, |theta_max|) + beta_{k+1}, times (1 + 1e-3),
    clamped to the Pauli 1-norm (a rigorous bound);
  * DOS: kernel polynomial method -- Chebyshev moments of the same start
    vector under G = H/E_max with the Jackson kernel; the expected count in
    [-a, a] is integrated in closed form and a found by bisection so that it
    equals d = d_ratio * n_eigs. d_ratio = 2 by default: with K = 18 E_max/a
    and the 1e-12 cut-off only levels with |E| below about 0.8 a survive the
    rank removal, and the accuracy falls off toward the window edge (the
    "inverted filter shape" of Fig. 2), so the window holds twice the levels
    that are returned.
``kpm_window`` is a heuristic (one stochastic start vector, 256 damped
moments). Its pins, in tests/test_oracle_params.py, are the count identity, the
large-M convergence, and exact level counts at N = 14: on four benchmark shards
its windows hold within 10 % of the requested number of exact levels (observed
within 3 %).
"""

from __future__ import annotations

import math

import numpy as np

from .hamiltonian import apply_h, diagonal, pauli_norm_bound


def lanczos_tridiagonal(model, v0, steps: int = 20, diag=None):
    """alpha_1..alpha_k and beta_2..beta_{k+1} of k plain Lanczos steps from v0."""
    if diag is None:
        diag = diagonal(model)
    v = np.asarray(v0, dtype=np.float64).ravel()
    v = v / np.linalg.norm(v)
    v_prev = np.zeros_like(v)
    beta = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = apply_h(model, v, diag) - beta * v_prev
        alpha = float(v @ w)
        w = w - alpha * v
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta)
        if beta == 0.0:
            break
        v_prev, v = v, w / beta
    return np.array(alphas), np.array(betas)


def ritz_last_components(alpha, beta) -> np.ndarray:
    """|e_k^T z_i| for every eigenvector z_i of the k x k tridiagonal T (diagonal
    alpha, off-diagonal beta[:k-1]) without forming the vectors:
    z_{k,i}^2 = prod_j (theta_i - mu_j) / prod_{j != i} (theta_i - theta_j), with
    theta the eigenvalues of T and mu those of its leading (k-1) x (k-1) block
    (the characteristic-polynomial identity p_{k-1}(theta_i) / p_k'(theta_i)).
    Cauchy interlacing (theta_1 < mu_1 < theta_2 < ...) pairs every factor into
    a ratio of magnitude at most one, which keeps the products stable. This is
    the form a per-realization GPU thread can evaluate from Sturm-bisection
    eigenvalues."""
    al = np.asarray(alpha, dtype=np.float64)
    k = len(al)
    if k == 1:
        return np.ones(1)
    b = np.asarray(beta, dtype=np.float64)[:k - 1]
    T = np.diag(al) + np.diag(b, 1) + np.diag(b, -1)
    th = np.linalg.eigvalsh(T)
    mu = np.linalg.eigvalsh(T[:k - 1, :k - 1])
    out = np.empty(k)
    for i in range(k):
        v = 1.0
        for j in range(i):                 # theta_j < mu_j < theta_{j+1} <= theta_i
            v *= (th[i] - mu[j]) / (th[i] - th[j])
        for j in range(i + 1, k):          # theta_i <= mu_{j-1} < theta_j
            v *= (th[i] - mu[j - 1]) / (th[i] - th[j])
        out[i] = np.sqrt(max(v, 0.0))
    return out


def emax_bound(model, v0, steps: int = 20, safety: float = 1e-3, diag=None, rule: str = "residual") -> float:
    """Upper bound on max |E| from k Lanczos steps (the estimator Sec. III cites).

    rule "residual": the extreme Ritz value plus the whole residual norm
    beta_{k+1} (the form the CUDA path uses). rule "ritz": the extreme Ritz value
    plus beta_{k+1} max_i |e_k^T z_i|, the largest residual of any Ritz pair
    (z_i the eigenvectors of the tridiagonal matrix). "ritz" is tighter (about
    1.14 times the spectral radius on N = 11..16 shards and chains, against
    1.36..1.54), but it is a bound only in practice. The residual of the extreme
    Ritz pair alone fell below the radius on 12 of 150 N = 11 shards.
    """
    al, be = lanczos_tridiagonal(model, v0, min(steps, 1 << model["N"]), diag)
    k = len(al)
    T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
    if rule == "ritz":
        th, Z = np.linalg.eigh(T)
        bound = max(abs(th[0]), abs(th[-1])) + be[k - 1] * float(np.abs(Z[-1, :]).max())
        return float(min(bound * (1.0 + safety), pauli_norm_bound(model)))
    if rule != "residual":
        raise ValueError(rule)
    th = np.linalg.eigvalsh(T)
    bound = max(abs(th[0]), abs(th[-1])) + be[k - 1]
    return float(min(bound * (1.0 + safety), pauli_norm_bound(model)))


def kpm_moments(model, v0, emax: float, M: int, diag=None) -> np.ndarray:
    """mu_k = <r|T_k(H/E_max)|r> / <r|r> for k = 0..M-1, by the plain recurrence."""
    if diag is None:
        diag = diagonal(model)
    r = np.asarray(v0, dtype=np.float64).ravel()
    r = r / np.linalg.norm(r)
    mu = np.zeros(M)
    t0 = r
    mu[0] = r @ t0
    if M == 1:
        return mu
    t1 = apply_h(model, r, diag) / emax
    mu[1] = r @ t1
    for k in range(2, M):
        t0, t1 = t1, 2.0 * apply_h(model, t1, diag) / emax - t0
        mu[k] = r @ t1
    return mu


def jackson(M: int) -> np.ndarray:
    """Jackson damping factors g_k, k = 0..M-1."""
    k = np.arange(M)
    q = math.pi / (M + 1)
    return ((M - k + 1) * np.cos(q * k) + np.sin(q * k) / math.tan(q)) / (M + 1)


def kpm_count(mu, D: int, a_r: float) -> float:
    """Expected number of levels in [-a_r, a_r] (units of E_max) from KPM moments.

    With rho(x) = [g_0 mu_0 + 2 sum_k g_k mu_k T_k(x)] / (pi sqrt(1-x^2)) and
    x = cos(theta), the integral of T_k over the window is
    (sin(k(pi-phi)) - sin(k phi)) / (pi k), phi = arccos(a_r), and (pi-2phi)/pi at k=0.
    """
    M = len(mu)
    g = jackson(M)
    phi = math.acos(a_r)
    tot = g[0] * mu[0] * (math.pi - 2.0 * phi) / math.pi
    for k in range(1, M):
        tot += 2.0 * g[k] * mu[k] * (math.sin(k * (math.pi - phi)) - math.sin(k * phi)) / (math.pi * k)
    return D * tot


def kpm_window(mu, D: int, emax: float, d_target: float, iters: int = 100) -> float:
    """Window half-width a with kpm_count(a/E_max) = d_target, by bisection on a_r."""
    lo, hi = 0.0, 0.999          # a < E_max keeps E_0 = (E_max^2 - a^2)/2 > 0
    if kpm_count(mu, D, hi) <= d_target:
        return hi * emax
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if kpm_count(mu, D, mid) < d_target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi) * emax


def basis_half_size(n_eigs: int, b: int, d_ratio: float = 2.0, basis_ratio: float = 1.5) -> int:
    """n with b(2n+1) >= basis_ratio * d, d = d_ratio * n_eigs (Sec. II B: 2n+1 = 1.5 d)."""
    d = d_ratio * n_eigs
    return max(1, int(math.ceil((basis_ratio * d / b - 1.0) / 2.0)))


def filter_order(emax: float, a: float, c: float = 18.0) -> int:
    """K = ceil(c E_max / a), c = 18 (Sec. II A)."""
    return int(math.ceil(c * emax / a))
