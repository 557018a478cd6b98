"""Pins for the oracle's DACP steps against the exact eigendecomposition.

For N <= 10 the dense spectral decomposition H = sum_i E_i |phi_i><phi_i| gives
closed forms for every step: the filtered coefficients, every moment, the
product identity, the Gram matrices and, with a complete basis, the whole
spectrum. The end-to-end case is the N=10 mixed-field chain against dense eigh.
"""

import numpy as np
import pytest

import workloads as W
from oracle import chebyshev as C
from oracle import dacp as DA
from oracle import hamiltonian as Hm
from oracle import metrics as MT
from oracle import params as P
from tests.conftest import read_golden


@pytest.fixture(scope="module")
def small():
    m = W.random_model(8, seed=21)
    H = Hm.dense_h(m)
    E, V = np.linalg.eigh(H)
    emax = Hm.pauli_norm_bound(m)
    return m, E, V, emax


def test_filter_coefficients(small):
    m, E, V, emax = small
    psi = W.start_vectors(8, 2, seed=1)
    a, K = 0.3 * emax / 4, 37
    out = DA.exp_semicircle_filter(m, psi, emax, a, K)
    c = V.T @ psi
    ref = C.filter_exact(E, emax, a, K)[:, None] * c
    ref /= np.linalg.norm(ref, axis=0)
    assert np.abs(V.T @ out - ref).max() < 1e-12


def test_moments_from_spectrum(small):
    m, E, V, emax = small
    psi = W.start_vectors(8, 2, seed=2)
    psi /= np.linalg.norm(psi, axis=0)
    kmax = 300
    mu, nu = DA.chebyshev_moments(m, psi, emax, kmax)
    c = V.T @ psi
    for k in (0, 1, 2, 17, 150, 299, 300):
        Tk = C.cheb_closed(k, E / emax)
        assert np.abs(mu[k] - c.T @ (Tk[:, None] * c)).max() < 1e-12, k
        assert np.abs(nu[k] - c.T @ ((E * Tk)[:, None] * c)).max() < 1e-11, k


def test_product_and_doubling_identities(small):
    m, E, V, emax = small
    psi = W.start_vectors(8, 1, seed=3)
    psi /= np.linalg.norm(psi)
    vecs = DA.chebyshev_vectors(m, psi, emax, 60)
    mu, _ = DA.chebyshev_moments(m, psi, emax, 120)
    rng = np.random.default_rng(0)
    for _ in range(20):
        i, j = rng.integers(0, 61, size=2)
        lhs = float(vecs[i][:, 0] @ vecs[j][:, 0])
        assert abs(lhs - 0.5 * (mu[i + j, 0, 0] + mu[abs(i - j), 0, 0])) < 1e-12
    for k in range(0, 60):
        # T_2k = 2 T_k^2 - 1 and T_{2k+1} = 2 T_{k+1} T_k - T_1
        assert abs(mu[2 * k, 0, 0] - (2 * vecs[k][:, 0] @ vecs[k][:, 0] - mu[0, 0, 0])) < 1e-12
        assert abs(mu[2 * k + 1, 0, 0] - (2 * vecs[k + 1][:, 0] @ vecs[k][:, 0] - mu[1, 0, 0])) < 1e-12


def test_assembly_equals_explicit_gram(small):
    m, E, V, emax = small
    b = 2
    psi = W.start_vectors(8, b, seed=4)
    psi /= np.linalg.norm(psi, axis=0)
    x = C.basis_orders(0.2, 4)
    vecs = DA.chebyshev_vectors(m, psi, emax, int(x[-1]))
    A = np.concatenate([vecs[k] for k in x], axis=1)   # column i*b + p
    mu, nu = DA.chebyshev_moments(m, psi, emax, int(2 * x[-1]))
    S, Hs = DA.assemble(mu, nu, x)
    assert np.abs(S - A.T @ A).max() < 1e-12
    assert np.abs(Hs - A.T @ Hm.apply_h(m, A)).max() < 1e-11


def test_complete_basis_gives_whole_spectrum():
    m = W.random_model(6, seed=9)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    emax = Hm.pauli_norm_bound(m)
    psi = W.start_vectors(6, 1, seed=5)
    # no filtering (K = 0) and a basis far larger than 2^6
    r = DA.dacp(m, psi, emax, a=0.5 * emax, K=0, n=60, n_eigs=64, window=emax)
    assert r["rank"] == 64
    assert np.abs(r["eigs"] - E).max() < 1e-10 * emax


def test_select_central():
    lams = np.array([-3.0, -0.5, -0.1, 0.2, 0.4, 2.0])
    assert np.allclose(DA.select_central(lams, 3, 1.0), [-0.1, 0.2, 0.4])
    assert np.allclose(DA.select_central(lams, 10, 1.0), [-0.5, -0.1, 0.2, 0.4])


def test_paper_constants(golden):
    consts = {r[0]: float(r[1]) for r in golden("paper_parameters.txt")}
    assert P.filter_order(1.0, 0.5, c=consts["filter_order_constant"]) == 36
    assert P.basis_half_size(100, 1, d_ratio=1.0, basis_ratio=consts["basis_ratio"]) == 75
    import inspect
    assert inspect.signature(DA.solve_gep).parameters["eps"].default == consts["rank_cutoff"]


def test_end_to_end_n10_chain_vs_dense():
    """N=10 mixed-field chain, 100 central eigenvalues, plain FP64: error <= 1e-9 * bandwidth."""
    m = W.chain(10)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    psi = W.start_vectors(10, 4, seed=0)
    emax = P.emax_bound(m, psi[:, 0])
    assert emax >= np.abs(E).max()
    mu = P.kpm_moments(m, psi[:, 0], emax, 256)
    a = P.kpm_window(mu, 1 << 10, emax, 2.0 * 100)
    n = P.basis_half_size(100, 4, d_ratio=2.0)
    K = P.filter_order(emax, a)
    r = DA.dacp(m, psi, emax, a, K, n, 100)
    assert len(r["eigs"]) == 100
    ex = MT.central_exact(E, 100)
    bandwidth = E[-1] - E[0]
    assert np.abs(r["eigs"] - ex).max() < 1e-9 * bandwidth


def test_planted_sign_error_is_caught(small):
    """A wrong sign in the evolution recurrence (2Gw + w_prev) breaks the moment pin."""
    m, E, V, emax = small
    psi = W.start_vectors(8, 1, seed=6)[:, 0]
    psi /= np.linalg.norm(psi)
    v0, v1 = psi, Hm.apply_h(m, psi) / emax
    for _ in range(2, 11):
        v0, v1 = v1, 2 * Hm.apply_h(m, v1) / emax + v0
    c = V.T @ psi
    ref = c @ (C.cheb_closed(10, E / emax) * c)
    assert abs(float(psi @ v1) - float(ref)) > 1e-3


def test_h2_moments_from_spectrum(small):
    """omega_k = <psi|H^2 T_k(G)|psi> = sum_i |c_i|^2 E_i^2 T_k(E_i/E_max) (Sec. II C <H^2>)."""
    m, E, V, emax = small
    psi = W.start_vectors(8, 2, seed=4)
    psi /= np.linalg.norm(psi, axis=0)
    om = DA.h2_moments(m, psi, emax, 120)
    c = V.T @ psi
    for k in (0, 1, 2, 3, 57, 119, 120):
        Tk = C.cheb_closed(k, E / emax)
        assert np.abs(om[k] - c.T @ ((E * E * Tk)[:, None] * c)).max() < 1e-10 * emax ** 2, k


def test_h2_moments_follow_from_mu(small):
    """G^2 T_k = (T_{k+2} + T_k + T_{|k-1|+1} + T_{||k-1|-1|})/4: omega is linear in mu.

    The GPU path derives omega this way from its moments; here both sides are
    recorded directly, so a wrong index in the identity fails."""
    m, E, V, emax = small
    psi = W.start_vectors(8, 2, seed=5)
    psi /= np.linalg.norm(psi, axis=0)
    mu, _ = DA.chebyshev_moments(m, psi, emax, 90)
    om = DA.h2_moments(m, psi, emax, 88)
    for k in (0, 1, 2, 3, 40, 88):
        k1 = abs(k - 1)
        k2 = abs(k1 - 1)
        ref = 0.25 * emax ** 2 * (mu[k + 2] + mu[k] + mu[k1 + 1] + mu[k2])
        assert np.abs(om[k] - ref).max() < 1e-10 * emax ** 2, k


@pytest.fixture(scope="module")
def ritz_case():
    N, b, ne = 8, 2, 30
    m = W.chain(N, J=1.0, hx=0.9045, hz=0.8090)
    Hd = Hm.dense_h(m)
    E = np.linalg.eigvalsh(Hd)
    emax = Hm.pauli_norm_bound(m)
    a = np.sort(np.abs(E))[2 * ne]
    K = int(np.ceil(18 * emax / a))
    psi_E = DA.exp_semicircle_filter(m, W.start_vectors(N, b, seed=0), emax, a, K)
    x = C.basis_orders(a / emax, 24)
    kmax = int(2 * x[-1])
    mu, nu = DA.chebyshev_moments(m, psi_E, emax, kmax)
    om = DA.h2_moments(m, psi_E, emax, kmax)
    S, H = DA.assemble(mu, nu, x)
    _, H2 = DA.assemble(mu, om, x)
    lam, Bc = DA.ritz_pairs(S, H)
    idx = DA.select_central_index(lam, ne, a)
    vecs = DA.chebyshev_vectors(m, psi_E, emax, int(x[-1]))
    basis = np.concatenate([vecs[xi] for xi in x], axis=1)     # column i*b + p = T_{x_i} psi_p
    return dict(m=m, Hd=Hd, E=E, emax=emax, a=a, S=S, H=H, H2=H2, lam=lam, Bc=Bc, idx=idx, basis=basis, ne=ne)


def test_ritz_pairs_are_s_normalised(ritz_case):
    rc = ritz_case
    B = rc["Bc"][:, rc["idx"]]
    lam = rc["lam"][rc["idx"]]
    assert np.abs(np.einsum("ij,ij->j", B, rc["S"] @ B) - 1.0).max() < 1e-9
    assert np.abs(np.einsum("ij,ij->j", B, rc["H"] @ B) - lam).max() < 1e-9 * rc["emax"]
    assert np.allclose(DA.select_central(rc["lam"], rc["ne"], rc["a"]), lam)


def test_residual_norms_match_explicit_ritz_vectors(ritz_case):
    """||r_j||^2 from H2 equals ||(H - lam_j) phi_j||^2 of the explicit Ritz vector,
    and ||r_j|| bounds the distance of lam_j to the exact spectrum (Sec. II C)."""
    rc = ritz_case
    idx = rc["idx"]
    lam = rc["lam"][idx]
    phi = rc["basis"] @ rc["Bc"][:, idx]
    assert np.abs(np.linalg.norm(phi, axis=0) - 1.0).max() < 1e-9
    r_ex = np.linalg.norm(rc["Hd"] @ phi - phi * lam, axis=0)
    r = DA.residual_norms(rc["Bc"], rc["lam"], rc["H2"])[idx]
    assert np.abs(r ** 2 - r_ex ** 2).max() < 1e-12 * rc["emax"] ** 2
    err = np.array([np.abs(rc["E"] - l).min() for l in lam])
    assert np.all(err <= r_ex * (1 + 1e-9) + 1e-13 * rc["emax"])
    assert np.all(err <= np.sqrt(r ** 2 + 1e-12 * rc["emax"] ** 2))


def test_residual_norms_flag_a_poor_basis(ritz_case):
    """With too few orders the levels near the window edge are not converged: their
    residuals grow while the well-converged central ones stay small."""
    rc = ritz_case
    m, emax, a = rc["m"], rc["emax"], rc["a"]
    psi_E = DA.exp_semicircle_filter(m, W.start_vectors(8, 2, seed=0), emax, a, int(np.ceil(18 * emax / a)))
    x = C.basis_orders(a / emax, 8)
    mu, nu = DA.chebyshev_moments(m, psi_E, emax, int(2 * x[-1]))
    om = DA.h2_moments(m, psi_E, emax, int(2 * x[-1]))
    S, H = DA.assemble(mu, nu, x)
    _, H2 = DA.assemble(mu, om, x)
    lam, Bc = DA.ritz_pairs(S, H)
    idx = DA.select_central_index(lam, rc["ne"], a)
    r = DA.residual_norms(Bc, lam, H2)[idx]
    err = np.array([np.abs(rc["E"] - l).min() for l in lam[idx]])
    assert r.max() > 1e3 * DA.residual_norms(rc["Bc"], rc["lam"], rc["H2"])[rc["idx"]].max()
    assert np.all(err <= np.sqrt(r ** 2 + 1e-12 * emax ** 2))


def test_end_to_end_random_field_heisenberg_vs_dense():
    """N=10 random-field Heisenberg chain (XX + YY + ZZ couplings, the many-body
    localization model), 80 central eigenvalues with b = 4: DACP through the
    pair-flip apply meets the float64 target against dense eigh."""
    m = W.heisenberg_chain(10, seed=4, W=2.0)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    psi = W.start_vectors(10, 4, seed=5)
    emax = P.emax_bound(m, psi[:, 0])
    assert emax >= np.abs(E).max()
    mu = P.kpm_moments(m, psi[:, 0], emax, 256)
    a = P.kpm_window(mu, 1 << 10, emax, 2.0 * 80)
    n = P.basis_half_size(80, 4, d_ratio=2.0)
    K = P.filter_order(emax, a)
    r = DA.dacp(m, psi, emax, a, K, n, 80)
    assert len(r["eigs"]) == 80
    ex = MT.central_exact(E, 80)
    assert np.abs(r["eigs"] - ex).max() < 1e-9 * (E[-1] - E[0])


def test_dacp_on_parity_sectors_gives_the_full_central_levels():
    """The oracle's DACP run on the two parity sectors of a shard (each an N - 1 spin model with
    z-fields and the global flip, reading 14; Sec. III heuristic parameters per sector, 32 levels
    each) and merged in plain numpy -- the n levels of smallest |E| of the union, within the smaller
    sector's largest returned |E| -- equals the full shard's 50 central levels of dense eigh to
    1e-9 of the width. This carries the global flip through the filter, the evolution and the
    subspace solve, not only through H.v."""
    m = W.spin_glass_shard(10, seed=17)
    full = np.linalg.eigvalsh(Hm.dense_h(m))
    n, n_sec = 50, 32
    got, radii = [], []
    for s_, ms in enumerate(Hm.parity_sector_models(m)):
        psi = W.start_vectors(9, 4, seed=3, r=s_)
        emax = P.emax_bound(ms, psi[:, 0])
        mu = P.kpm_moments(ms, psi[:, 0], emax, 256)
        a = P.kpm_window(mu, 1 << 9, emax, 2.0 * n_sec)
        r = DA.dacp(ms, psi, emax, a, P.filter_order(emax, a), P.basis_half_size(n_sec, 4, d_ratio=2.0), n_sec)
        assert len(r["eigs"]) == n_sec
        got.append(np.asarray(r["eigs"]))
        radii.append(np.abs(r["eigs"]).max())
    union = np.concatenate(got)
    union = union[np.abs(union) <= min(radii)]
    merged = np.sort(union[np.argsort(np.abs(union), kind="stable")[:n]])
    assert len(merged) == n
    assert np.abs(merged - MT.central_exact(full, n)).max() < 1e-9 * (full[-1] - full[0])
