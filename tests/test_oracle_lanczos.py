"""Pins of the Appendix D comparison method (oracle.lanczos): Krylov space of the filtered operator.

Each pin rests on something other than the oracle's own arithmetic:
  * the basis is orthonormal, and it spans the space of the explicit powers
    v, A v, A^2 v, A^3 v with A = T_K(F(H)) built from the dense
    eigendecomposition and the closed form T_K(x) = cos(K acos x) / cosh(K acosh x);
  * a start vector inside an invariant subspace of three eigenvectors gives a
    three-dimensional space (then a breakdown) whose Ritz values are those
    three eigenvalues;
  * +-E blindness: for a start vector c+ phi(E) + c- phi(-E) of a chain with a
    symmetric spectrum, A acts as one number, the space is one-dimensional,
    its Ritz value is theta = E (c+^2 - c-^2) / (c+^2 + c-^2), not +-E, with
    residual sqrt(c+^2 (E - theta)^2 + c-^2 (E + theta)^2) / |c|, so the
    residual test rejects it and no level is returned;
  * without +-E partners among the central levels, 3R steps give the R
    central levels of dense eigh; with such a pair, what comes back is still
    only levels (the residual test drops the mixed Ritz values).
"""

import numpy as np

import workloads as W
from oracle import hamiltonian as Hm
from oracle import lanczos as LZ
from oracle import metrics as MT


def _dense_filter(E, Q, emax, a, K):
    ec, e0 = (emax * emax + a * a) / 2.0, (emax * emax - a * a) / 2.0
    x = (E * E - ec) / e0
    t = np.where(np.abs(x) <= 1.0, np.cos(K * np.arccos(np.clip(x, -1, 1))),
                 np.sign(x) ** K * np.cosh(K * np.arccosh(np.maximum(np.abs(x), 1.0))))
    return (Q * t) @ Q.T


def test_basis_is_orthonormal_and_spans_the_explicit_krylov_space():
    m = W.random_model(6, seed=3)
    E, Q = np.linalg.eigh(Hm.dense_h(m))
    emax = 1.05 * np.abs(E).max()
    a, K = 0.5 * emax, 2
    psi = W.start_vectors(6, 1, seed=1)[:, 0]
    V = LZ.krylov_filtered(m, psi, emax, a, K, 4)
    assert V.shape == (64, 4)
    assert np.abs(V.T @ V - np.eye(4)).max() < 1e-12
    A = _dense_filter(E, Q, emax, a, K)
    cols = [psi / np.linalg.norm(psi)]
    for _ in range(3):
        w = A @ cols[-1]
        cols.append(w / np.linalg.norm(w))
    Qk, _ = np.linalg.qr(np.stack(cols, axis=1))
    assert np.abs(V @ V.T - Qk @ Qk.T).max() < 1e-8


def test_invariant_subspace_gives_its_eigenvalues_and_breaks_down():
    m = W.random_model(7, seed=5)
    E, Q = np.linalg.eigh(Hm.dense_h(m))
    emax = 1.05 * np.abs(E).max()
    idx = np.argsort(np.abs(E))[:3]                       # three central levels: distinct filter values
    psi = Q[:, idx] @ np.array([0.6, -0.5, 0.8])
    a = 2.0 * np.abs(E[idx]).max()
    lam, dim = LZ.lanczos_filtered(m, psi, emax, a, 30, 8, 10)
    assert dim == 3
    assert np.abs(np.sort(lam) - np.sort(E[idx])).max() < 1e-10


def test_plus_minus_e_pairs_are_not_resolved():
    """The integrable chain's spectrum is symmetric; the filter is even in E."""
    m = W.chain(4, J=1.0, hx=1.0, hz=0.0)
    E, Q = np.linalg.eigh(Hm.dense_h(m))
    gaps = np.diff(E)
    k = [i for i in range(len(E)) if E[i] > 1e-6 and np.min(np.abs(E + E[i])) < 1e-10
         and (i == 0 or gaps[i - 1] > 1e-6) and (i == len(E) - 1 or gaps[i] > 1e-6)][0]
    j = int(np.argmin(np.abs(E + E[k])))
    cp, cm = 0.8, 0.3
    psi = cp * Q[:, k] + cm * Q[:, j]
    emax = 1.05 * np.abs(E).max()
    V = LZ.krylov_filtered(m, psi, emax, 2.0 * E[k], 12, 5)
    assert V.shape[1] == 1
    th, res = LZ.ritz_pairs(m, V)
    theta = E[k] * (cp ** 2 - cm ** 2) / (cp ** 2 + cm ** 2)
    assert abs(th[0] - theta) < 1e-10
    assert abs(res[0] - np.sqrt(cp ** 2 * (E[k] - theta) ** 2 + cm ** 2 * (E[k] + theta) ** 2) /
               np.hypot(cp, cm)) < 1e-10
    lam, dim = LZ.lanczos_filtered(m, psi, emax, 2.0 * E[k], 12, 5, 5)
    assert dim == 1 and len(lam) == 0


def test_central_levels_converge_without_plus_minus_partners():
    """3R steps give the R central levels of dense eigh where no two of the 3R central levels
    nearly cancel (|E_i + E_j| above a quarter of the mean spacing: their filter values then
    differ); the same method on a model with such a pair returns a value between the partners,
    which is no level (the even filter of test_plus_minus_e_pairs_are_not_resolved)."""
    R = 4
    m = W.random_model(8, seed=15)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    c = E[np.argsort(np.abs(E))[:3 * R]]
    s = np.abs(c[:, None] + c[None, :])
    np.fill_diagonal(s, np.inf)
    assert s.min() > 0.25 * np.mean(np.diff(np.sort(c)))          # the precondition holds
    emax = 1.05 * np.abs(E).max()
    a = np.sort(np.abs(E))[2 * R]                                # the window holds about 2R levels
    K = int(np.ceil(18 * emax / a))
    psi = W.start_vectors(8, 1, seed=2)[:, 0]
    lam, dim = LZ.lanczos_filtered(m, psi, emax, a, K, 3 * R, R)
    assert dim == 3 * R and len(lam) == R
    assert np.abs(lam - MT.central_exact(E, R)).max() < 1e-8 * (E[-1] - E[0])
    # a model whose central levels include a near pair (0.1604 and -0.1571 ..): only levels come back
    m2 = W.random_model(8, seed=11)
    E2 = np.linalg.eigvalsh(Hm.dense_h(m2))
    emax2 = 1.05 * np.abs(E2).max()
    a2 = np.sort(np.abs(E2))[12]
    lam2, _ = LZ.lanczos_filtered(m2, psi, emax2, a2, int(np.ceil(18 * emax2 / a2)), 18, 6)
    assert len(lam2) > 0
    assert max(np.min(np.abs(E2 - x)) for x in lam2) < 1e-8 * (E2[-1] - E2[0])
