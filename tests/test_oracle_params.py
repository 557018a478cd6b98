"""Pins for the oracle's parameter selection (E_max bound, KPM window)."""

import math

import numpy as np

import workloads as W
from oracle import chebyshev as C
from oracle import hamiltonian as Hm
from oracle import params as P


def test_lanczos_complete_krylov_is_exact():
    m = W.random_model(3, seed=2)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    v0 = np.random.default_rng(0).standard_normal(8)
    al, be = P.lanczos_tridiagonal(m, v0, steps=8)
    k = len(al)
    T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
    th = np.linalg.eigvalsh(T)
    assert abs(th[0] - E[0]) < 1e-9 and abs(th[-1] - E[-1]) < 1e-9


def test_emax_is_an_upper_bound():
    for seed in range(8):
        m = W.random_model(8, seed=100 + seed)
        E = np.linalg.eigvalsh(Hm.dense_h(m))
        v0 = W.start_vectors(8, 1, seed=seed)[:, 0]
        bnd = P.emax_bound(m, v0)
        assert np.abs(E).max() <= bnd <= Hm.pauli_norm_bound(m) + 1e-12


def test_kpm_moments_from_spectrum():
    m = W.random_model(8, seed=7)
    E, V = np.linalg.eigh(Hm.dense_h(m))
    emax = Hm.pauli_norm_bound(m)
    r = W.start_vectors(8, 1, seed=9)[:, 0]
    mu = P.kpm_moments(m, r, emax, 64)
    w = (V.T @ (r / np.linalg.norm(r))) ** 2
    for k in (0, 1, 5, 63):
        assert abs(mu[k] - w @ C.cheb_closed(k, E / emax)) < 1e-12


def test_jackson_and_count_identities():
    g = P.jackson(64)
    assert abs(g[0] - 1.0) < 1e-12 and np.all(np.diff(g) < 0)
    # A flat moment sequence (mu_0 = 1, others 0) is the Chebyshev weight
    # 1/(pi sqrt(1-x^2)); its mass in [-a, a] is (pi - 2 acos a)/pi.
    mu = np.zeros(32)
    mu[0] = 1.0
    for ar in (0.1, 0.5, 0.9):
        assert abs(P.kpm_count(mu, 1, ar) - (math.pi - 2 * math.acos(ar)) / math.pi) < 1e-12


def test_kpm_count_converges_to_weighted_count():
    m = W.chain(10)
    E, V = np.linalg.eigh(Hm.dense_h(m))
    emax = P.emax_bound(m, W.start_vectors(10, 1, 0)[:, 0])
    r = W.start_vectors(10, 1, seed=3)[:, 0]
    w = (V.T @ (r / np.linalg.norm(r))) ** 2
    mu = P.kpm_moments(m, r, emax, 2048)
    a = 2.0
    exact = 1024 * w[np.abs(E) <= a].sum()
    assert abs(P.kpm_count(mu, 1024, a / emax) - exact) < 0.05 * exact
    a_found = P.kpm_window(mu, 1024, emax, exact)
    assert abs(a_found - a) < 0.1 * a


def test_filter_order_and_basis():
    assert P.filter_order(10.0, 1.0) == 180
    assert P.basis_half_size(100, 4, d_ratio=2.0) == 37     # 4(2n+1) = 300


def test_kpm_window_counts_against_exact_levels_at_benchmark_size():
    """At N = 14 (four shards of the benchmark batch), the window that the KPM
    estimate from one start vector and 256 Jackson-damped moments puts around
    d levels holds d levels of the exact spectrum (dense eigh,
    tests/golden/shard14_dense_central_levels.txt) to within 10 %."""
    from tests.conftest import read_golden
    lv = {}
    for row in read_golden("shard14_dense_central_levels.txt"):
        if len(row) == 2:
            lv.setdefault(int(row[0]), []).append(float(row[1]))
    for seed, v in lv.items():
        m = W.spin_glass_shard(14, seed=seed)
        psi = W.start_vectors(14, 1, seed=0, r=seed)[:, 0]
        diag = Hm.diagonal(m)
        emax = P.emax_bound(m, psi, diag=diag)
        mu = P.kpm_moments(m, psi, emax, 256, diag=diag)
        v = np.asarray(v)
        for target in (200, 400, 600):
            a = P.kpm_window(mu, 1 << 14, emax, target)
            assert a < v[-1] and -a > v[0]                  # inside the stored levels
            count = int(np.sum(np.abs(v) <= a))
            assert abs(count - target) <= 0.1 * target, (seed, target, count)


def test_emax_bound_holds_against_exact_extremes_at_benchmark_sizes():
    """The Lanczos E_max bound must exceed every |E| (Sec. II A: a level beyond it
    grows exponentially in both recurrences). Checked against the exact extreme
    levels (dense eigh, tests/golden) of four N = 14 shards and of the N = 16
    mixed-field chain. The bound is loose: 1.36 to 1.50 times the spectral
    radius on these five, which the filter order and the evolution length pay
    for in proportion (both scale with E_max / a)."""
    from tests.conftest import read_golden
    cases = []
    for row in read_golden("shard14_dense_central_levels.txt"):
        if len(row) == 3:
            cases.append((W.spin_glass_shard(14, seed=int(row[0])), float(row[1]), float(row[2]), int(row[0])))
    row = read_golden("chain16_dense_central_levels.txt")[0]
    cases.append((W.chain(16), float(row[0]), float(row[1]), 0))
    for m, emin, emax_exact, r in cases:
        psi = W.start_vectors(m["N"], 1, seed=0, r=r)[:, 0]
        radius = max(-emin, emax_exact)
        bound = P.emax_bound(m, psi)
        assert radius <= bound <= min(1.6 * radius, Hm.pauli_norm_bound(m)), (m["N"], r, radius, bound)


def test_ritz_rule_is_tighter_and_still_above_the_radius():
    """The Ritz-residual rule against exact spectral radii: 16 N = 10 shards
    (dense eigh) and the five benchmark-size cases (tests/golden). It stays
    above the radius on every one and below 1.25 times it, where the residual
    rule sits near 1.46."""
    from tests.conftest import read_golden
    cases = []
    for seed in range(16):
        m = W.spin_glass_shard(10, seed=500 + seed)
        E = np.linalg.eigvalsh(Hm.dense_h(m))
        cases.append((m, max(-E[0], E[-1]), seed))
    for row in read_golden("shard14_dense_central_levels.txt"):
        if len(row) == 3:
            cases.append((W.spin_glass_shard(14, seed=int(row[0])), max(-float(row[1]), float(row[2])), int(row[0])))
    row = read_golden("chain16_dense_central_levels.txt")[0]
    cases.append((W.chain(16), max(-float(row[0]), float(row[1])), 0))
    for m, radius, r in cases:
        psi = W.start_vectors(m["N"], 1, seed=0, r=r)[:, 0]
        diag = Hm.diagonal(m)
        tight = P.emax_bound(m, psi, diag=diag, rule="ritz")
        loose = P.emax_bound(m, psi, diag=diag)
        assert radius <= tight <= 1.25 * radius < loose, (m["N"], r, radius, tight, loose)


def test_ritz_last_components_from_the_interlacing_identity():
    """The eigenvector-free last components equal those of eigh's eigenvectors
    on random tridiagonals and on a Lanczos tridiagonal of a shard."""
    rng = np.random.default_rng(7)
    cases = [(rng.standard_normal(k), np.abs(rng.standard_normal(k)) + 0.1) for k in (1, 2, 5, 20)]
    m = W.spin_glass_shard(10, seed=3)
    cases.append(P.lanczos_tridiagonal(m, W.start_vectors(10, 1, seed=1)[:, 0], 20)[:2])
    for al, be in cases:
        k = len(al)
        T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
        _, Z = np.linalg.eigh(T)
        got, ref = P.ritz_last_components(al, be), np.abs(Z[-1, :])
        # components far below one (nearly converged Ritz pairs) are where both forms lose digits
        assert np.abs(got - ref).max() < 1e-7
        assert abs(got.max() - ref.max()) < 1e-10          # the one the Ritz-residual rule uses
