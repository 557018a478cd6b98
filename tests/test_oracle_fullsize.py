"""The oracle's whole DACP pipeline at the benchmark size, against exact levels.

One shard of the 256-shard N = 14 batch (realization 0), 500 central levels,
b = 4, the paper's parameters (c = 18, window ratio 2, basis ratio 1.5): the
float64 oracle's filter, directly recorded moments, assembly and generalized
eigensolve, against the dense-eigh levels in
tests/golden/shard14_dense_central_levels.txt. About 80 000 float64 H.v on
one core, several minutes, so it runs only with DACP_ORACLE_FULL=1.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import dacp as DA
from oracle import hamiltonian as Hm
from oracle import params as P
from tests.conftest import read_golden


@pytest.mark.skipif(not os.environ.get("DACP_ORACLE_FULL"), reason="several minutes; set DACP_ORACLE_FULL=1")
def test_oracle_dacp_on_a_benchmark_shard_vs_dense():
    rows = read_golden("shard14_dense_central_levels.txt")
    emin, emax_exact = [(float(r[1]), float(r[2])) for r in rows if len(r) == 3 and r[0] == "0"][0]
    lv = np.array([float(r[1]) for r in rows if len(r) == 2 and r[0] == "0"])
    n_eigs = 500
    exact = np.sort(lv[np.argsort(np.abs(lv), kind="stable")[:n_eigs]])
    m = W.spin_glass_shard(14, seed=0)
    psi = W.start_vectors(14, 4, seed=0, r=0)
    diag = Hm.diagonal(m)
    emax = P.emax_bound(m, psi[:, 0], diag=diag)
    assert emax >= max(-emin, emax_exact)
    mu = P.kpm_moments(m, psi[:, 0], emax, 256, diag=diag)
    a = P.kpm_window(mu, 1 << 14, emax, 2.0 * n_eigs)
    K = P.filter_order(emax, a)
    n = P.basis_half_size(n_eigs, 4)
    r = DA.dacp(m, psi, emax, a, K, n, n_eigs)
    assert len(r["eigs"]) == n_eigs
    # the float64 target: 1e-9 of the spectral width
    assert np.abs(r["eigs"] - exact).max() < 1e-9 * (emax_exact - emin)
