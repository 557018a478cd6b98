"""Pins for the Jordan-Wigner closed form: agreement with dense diagonalisation."""

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from oracle import jordan_wigner as JW
from tests.conftest import read_golden


def _random_chain(N, seed):
    rng = np.random.default_rng(seed)
    m = W.chain(N, J=1.0, hx=1.0, hz=0.0)
    for i in range(N - 1):
        m["J"][i, i + 1] = rng.uniform(-2.0, 2.0)
    m["gamma"] = rng.uniform(0.05, 2.0, size=N)
    return m


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 10])
def test_jw_matches_dense(N):
    m = _random_chain(N, seed=N)
    ev = np.linalg.eigvalsh(Hm.dense_h(m))
    assert np.abs(JW.spectrum(m) - ev).max() < 1e-12 * max(1.0, np.abs(ev).max())


def test_jw_uniform_chain_and_golden():
    m = W.chain(2, J=1.0, hx=1.0, hz=0.0)
    gold = np.array([float(r[0]) for r in read_golden("n2_chain_spectrum.txt")])
    assert np.allclose(JW.spectrum(m), gold, atol=1e-14)
    m10 = W.chain(10, J=1.0, hx=1.0, hz=0.0)
    assert np.allclose(JW.spectrum(m10), np.linalg.eigvalsh(Hm.dense_h(m10)), atol=1e-11)


def test_jw_rejects_non_chain():
    with pytest.raises(ValueError):
        JW.spectrum(W.chain(4))                  # h_z != 0
    with pytest.raises(ValueError):
        JW.spectrum(W.spin_glass_shard(4, 0))    # all-to-all couplings


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_xx_chain_free_fermions_match_dense(N):
    """Open XX chain in random z-fields (XXZ with delta = 0): the subset sums of
    the hopping matrix's eigenvalues equal the dense spectrum; this pins the
    pair flips and the sign of Y_i Y_j."""
    m = W.heisenberg_chain(N, seed=N, J=0.8, delta=0.0, W=1.5)
    t = [m["Jxx"][i, i + 1] for i in range(N - 1)]
    ev = np.linalg.eigvalsh(Hm.dense_h(m))
    assert np.abs(JW.hopping_chain_spectrum(t, m["h"]) - ev).max() < 1e-12 * max(1.0, np.abs(ev).max())
