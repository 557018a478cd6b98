"""Pins for the oracle's Hamiltonian (matrix-free apply and dense builder).

The bit-flip apply and the Kronecker-product builder are two independent
constructions; on top of their agreement, closed forms (N=1, N=2), trace
identities and symmetry-sector structure pin both against the mathematics.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from tests.conftest import read_golden


def test_apply_matches_kronecker_dense():
    m = W.random_model(7, seed=3)
    x = np.random.default_rng(1).standard_normal((1 << 7, 3))
    y = Hm.apply_h(m, x)
    ref = Hm.dense_h(m) @ x
    assert np.abs(y - ref).max() < 1e-13 * np.abs(ref).max()


def test_single_spin_closed_form():
    m = {"N": 1, "J": np.zeros((1, 1)), "h": np.array([0.7]), "gamma": np.array([1.3])}
    ev = np.linalg.eigvalsh(Hm.dense_h(m))
    r = np.hypot(0.7, 1.3)
    assert np.allclose(ev, [-r, r], atol=1e-15)
    # matrix-free: H^2 = (Gamma^2 + h^2) I
    x = np.array([0.3, -1.1])
    assert np.allclose(Hm.apply_h(m, Hm.apply_h(m, x)), r * r * x, atol=1e-14)


def test_two_spin_chain_golden():
    m = W.chain(2, J=1.0, hx=1.0, hz=0.0)
    ev = np.linalg.eigvalsh(Hm.dense_h(m))
    gold = np.array([float(r[0]) for r in read_golden("n2_chain_spectrum.txt")])
    assert np.allclose(ev, gold, atol=1e-14)


def test_traces():
    m = W.random_model(8, seed=5)
    H = Hm.dense_h(m)
    D = H.shape[0]
    assert abs(np.trace(H)) < 1e-11
    assert abs(np.trace(H @ H) / D - Hm.trace_h2_per_state(m)) < 1e-11
    assert abs(Hm.diagonal(m).sum()) < 1e-11


def test_symmetric_operator():
    m = W.random_model(9, seed=11)
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal((2, 1 << 9))
    assert abs(u @ Hm.apply_h(m, v) - Hm.apply_h(m, u) @ v) < 1e-11


def _sector_spectra(H, P):
    """Eigenvalues of H restricted to the +1 and -1 eigenspaces of an involution P."""
    w, V = np.linalg.eigh(P)
    out = []
    for sgn in (1.0, -1.0):
        B = V[:, np.isclose(w, sgn)]
        out.append((B.shape[1], np.linalg.eigvalsh(B.T @ H @ B)))
    return out


def test_parity_sectors_h0():
    m = W.spin_glass_shard(8, seed=4)        # h = 0 -> global spin flip is a symmetry
    H = Hm.dense_h(m)
    D = H.shape[0]
    P = np.zeros((D, D))
    P[np.arange(D) ^ (D - 1), np.arange(D)] = 1.0
    assert np.abs(P @ H - H @ P).max() < 1e-12
    (d1, e1), (d2, e2) = _sector_spectra(H, P)
    assert d1 == d2 == D // 2
    assert np.allclose(np.sort(np.concatenate([e1, e2])), np.linalg.eigvalsh(H), atol=1e-11)


def test_reflection_sectors_uniform_chain():
    N = 10
    m = W.chain(N)
    H = Hm.dense_h(m)
    D = 1 << N
    s = np.arange(D)
    rev = np.zeros(D, dtype=np.int64)
    for i in range(N):
        rev |= ((s >> i) & 1) << (N - 1 - i)
    R = np.zeros((D, D))
    R[rev, s] = 1.0
    assert np.abs(R @ H - H @ R).max() < 1e-12
    (dp, ep), (dm, em) = _sector_spectra(H, R)
    assert (dp, dm) == (528, 496)             # (2^N +- 2^ceil(N/2)) / 2
    assert np.allclose(np.sort(np.concatenate([ep, em])), np.linalg.eigvalsh(H), atol=1e-10)


def test_pauli_bound_holds():
    for seed in range(5):
        m = W.random_model(7, seed=seed)
        assert np.abs(np.linalg.eigvalsh(Hm.dense_h(m))).max() <= Hm.pauli_norm_bound(m) + 1e-12


def test_dense_limit():
    with pytest.raises(ValueError):
        Hm.dense_h(W.chain(13))


def test_planted_mistake_is_caught():
    """A transposed coupling (J_ji used as if it were J_ij+1) breaks the dense agreement."""
    m = W.random_model(6, seed=8)
    bad = dict(m)
    Jb = m["J"].copy()
    Jb[0, 2], Jb[1, 2] = Jb[1, 2], Jb[0, 2]
    bad["J"] = Jb
    x = np.random.default_rng(3).standard_normal(1 << 6)
    assert np.abs(Hm.apply_h(bad, x) - Hm.dense_h(m) @ x).max() > 1e-3


def test_row_apply_matches_full_apply():
    """The row-wise apply used for sampled parity at large N equals the full
    apply (itself pinned to the Kronecker builder) on every row it is given,
    including the first and last state, for one and several columns."""
    m = W.random_model(9, seed=11)
    rng = np.random.default_rng(4)
    for x in (rng.standard_normal(1 << 9), rng.standard_normal((1 << 9, 3))):
        full = Hm.apply_h(m, x)
        rows = np.concatenate([[0, (1 << 9) - 1], rng.integers(0, 1 << 9, size=60)])
        y, a = Hm.apply_h_rows(m, x, rows, with_abs=True)
        assert np.abs(y - full[rows]).max() < 1e-13 * np.abs(full).max()
        assert (a >= np.abs(y) - 1e-12).all()


def _pair_model(N, seed):
    m = W.random_model(N, seed=seed)
    rng = np.random.default_rng(seed + 100)
    m["Jxx"] = np.triu(rng.uniform(-1.0, 1.0, (N, N)), 1)
    m["Jyy"] = np.triu(rng.uniform(-1.0, 1.0, (N, N)), 1)
    return m


def test_pair_flips_match_kronecker_dense():
    """XX and YY couplings: the matrix-free pair flips with the -z_i z_j sign of
    Y_i Y_j equal the Kronecker products of the 2 x 2 Pauli matrices (Y complex,
    Y x Y real), on one and several columns and on sampled rows."""
    m = _pair_model(7, seed=5)
    H = Hm.dense_h(m)
    assert np.abs(H - H.T).max() == 0.0
    rng = np.random.default_rng(6)
    for x in (rng.standard_normal(1 << 7), rng.standard_normal((1 << 7, 3))):
        ref = H @ x
        assert np.abs(Hm.apply_h(m, x) - ref).max() < 1e-13 * np.abs(ref).max()
        rows = rng.integers(0, 1 << 7, size=40)
        assert np.abs(Hm.apply_h_rows(m, x, rows) - ref[rows]).max() < 1e-13 * np.abs(ref).max()


def test_heisenberg_two_spins_closed_form():
    """J (XX + YY + ZZ) on two spins: sigma_1 . sigma_2 = 2 S(S+1) - 3, so the
    triplet sits at J (three times) and the singlet at -3J."""
    J = 0.7
    m = {"N": 2, "J": np.array([[0.0, J], [0.0, 0.0]]), "h": np.zeros(2), "gamma": np.zeros(2),
         "Jxx": np.array([[0.0, J], [0.0, 0.0]]), "Jyy": np.array([[0.0, J], [0.0, 0.0]])}
    assert np.allclose(np.linalg.eigvalsh(Hm.dense_h(m)), [-3 * J, J, J, J], atol=1e-15)
    # matrix-free: the singlet (|01> - |10>)/sqrt2 is an eigenvector with -3J
    singlet = np.array([0.0, 1.0, -1.0, 0.0]) / np.sqrt(2.0)
    assert np.allclose(Hm.apply_h(m, singlet), -3 * J * singlet, atol=1e-15)


def test_pair_terms_traces_and_bound():
    m = _pair_model(8, seed=9)
    H = Hm.dense_h(m)
    D = H.shape[0]
    assert abs(np.trace(H)) < 1e-11                       # pair flips are off-diagonal
    assert abs(np.trace(H @ H) / D - Hm.trace_h2_per_state(m)) < 1e-11
    assert np.abs(np.linalg.eigvalsh(H)).max() <= Hm.pauli_norm_bound(m) + 1e-12


def test_xx_plus_yy_conserves_magnetization():
    """With Jxx = Jyy and no x-field the coupling only swaps unequal bits, so
    H maps each Hamming-weight sector into itself."""
    m = W.heisenberg_chain(9, seed=2)
    s = np.arange(1 << 9)
    weight = np.array([bin(v).count("1") for v in s])
    x = np.where(weight == 4, np.random.default_rng(1).standard_normal(1 << 9), 0.0)
    y = Hm.apply_h(m, x)
    assert np.abs(y[weight != 4]).max() == 0.0 and np.abs(y[weight == 4]).max() > 0.1


def test_planted_yy_sign_mistake_is_caught():
    """Y_i Y_j with +z_i z_j instead of -z_i z_j (i.e. XX - YY pairing terms)
    changes the spectrum of the XX chain, so the free-fermion pin catches it."""
    m = W.heisenberg_chain(6, seed=3, delta=0.0)
    bad = dict(m)
    bad["Jyy"] = -m["Jyy"]
    assert np.abs(np.linalg.eigvalsh(Hm.dense_h(bad)) - np.linalg.eigvalsh(Hm.dense_h(m))).max() > 1e-3


def test_reflection_sector_blocks_reproduce_the_spectrum():
    """The even / odd mirror-sector blocks (formed with the matrix-free apply)
    have dimensions (2^N +- 2^ceil(N/2)) / 2 and together carry H's spectrum:
    the mixed-field chain at N = 10 and a Heisenberg chain in a uniform field
    at N = 9."""
    m = W.chain(10)
    He, Ho = Hm.reflection_sector_matrices(m, chunk=128)
    assert He.shape == (528, 528) and Ho.shape == (496, 496)
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(He), np.linalg.eigvalsh(Ho)]))
    assert np.abs(ev - np.linalg.eigvalsh(Hm.dense_h(m))).max() < 1e-12
    h = W.heisenberg_chain(9, seed=1, W=0.0)
    h["h"] = np.full(9, 0.3)
    He, Ho = Hm.reflection_sector_matrices(h, chunk=64)
    assert He.shape[0] + Ho.shape[0] == 512 and He.shape[0] == (512 + 32) // 2
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(He), np.linalg.eigvalsh(Ho)]))
    assert np.abs(ev - np.linalg.eigvalsh(Hm.dense_h(h))).max() < 1e-12


def test_reflection_sectors_refuse_an_asymmetric_model():
    with pytest.raises(ValueError):
        Hm.reflection_sector_matrices(W.random_model(6, seed=2))


def test_global_flip_matches_kronecker_products_and_trace():
    """The global flip c X_0 ... X_{N-1}: the matrix-free apply, the row-wise apply and the
    Kronecker builder agree, and Tr H^2 / D gains c^2 (Pauli strings are orthonormal)."""
    m = dict(W.random_model(6, seed=4))
    m["gflip"] = 0.731
    Hd = Hm.dense_h(m)
    x = W.start_vectors(6, 2, seed=1)
    assert np.abs(Hm.apply_h(m, x) - Hd @ x).max() < 1e-13 * np.abs(Hd).max() * np.abs(x).max() * 64
    y, _ = Hm.apply_h_rows(m, x, np.arange(64), with_abs=True)
    assert np.abs(y - Hd @ x).max() < 1e-12
    assert abs(np.trace(Hd @ Hd) / 64 - Hm.trace_h2_per_state(m)) < 1e-12
    assert np.abs(Hd - Hd.T).max() == 0.0


@pytest.mark.parametrize("N,seed", [(8, 3), (10, 7)])
def test_parity_sectors_split_the_spectrum(N, seed):
    """The two (N-1)-spin sector models of a spin-glass shard (h = 0) have spectra whose union is
    the full spectrum (dense eigh of both sides), 2^(N-1) levels each."""
    m = W.spin_glass_shard(N, seed=seed)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    sp, sm = Hm.parity_sector_models(m)
    assert sp["N"] == sm["N"] == N - 1 and sp["gflip"] == -sm["gflip"] == m["gamma"][N - 1]
    Ep = np.linalg.eigvalsh(Hm.dense_h(sp))
    Em = np.linalg.eigvalsh(Hm.dense_h(sm))
    assert len(Ep) == len(Em) == 1 << (N - 1)
    assert np.abs(np.sort(np.concatenate([Ep, Em])) - E).max() < 1e-10 * np.abs(E).max()
    # a z-field breaks the symmetry and is refused
    bad = dict(m)
    bad["h"] = np.full(N, 0.1)
    with pytest.raises(ValueError):
        Hm.parity_sector_models(bad)
