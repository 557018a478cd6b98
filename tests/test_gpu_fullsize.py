"""Parity at the benchmark's full size (GPU).

The configuration bench.py times: 256 spin-glass shards, N = 14, b = 4, 500 central levels each,
double-float vectors, E_max by the Ritz-residual rule, the tile size the autotuner picks, the learned
parameters when their weights exist (heuristic otherwise), and dacp_solve / dacp_solve_learned. The CPU oracle cannot run the whole batch, so it checks
sampled outputs and properties that hold at any size:

  * one realization's filtered state against the oracle's filter, run with the GPU's parameters;
  * that realization's first moment rows, against the oracle's direct record of <psi_E|T_k(G)|psi_E>
    on the oracle's own filtered state (doubling identities against direct products, at full size);
  * |mu_j| <= mu_0 and the requested count, for sampled realizations;
  * sampled realizations' levels against float64 DACP with the paper's parameters, within 1e-2 of the
    local mean spacing. That float64 run is itself pinned to the oracle and to dense spectra by the other
    parity tests;
  * every one of the 500 levels of realizations 0, 64, 128 and 192 against their exact levels (dense
    float64 eigh of the 16384 x 16384 matrices, tests/golden/shard14_dense_central_levels.txt, written
    by an oracle-only script), within 1e-2 of the local mean spacing: the accuracy measure of Sec. III
    (Fig. 2 judges DACP's levels against exact ones) at the batched target.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import dacp as DA
from oracle import metrics as MT
from tests.conftest import read_golden

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")
from paper_2011_02107_gb300 import train_mlp as TM  # noqa: E402

N, R, B, NE = 14, 256, 4, 500


@pytest.fixture(scope="module")
def batch():
    models = [W.spin_glass_shard(N, seed=r) for r in range(R)]
    psis = [W.start_vectors(N, B, seed=0, r=r) for r in range(R)]
    mlp = None
    if os.path.exists(TM.DEFAULT_PATH) and str(np.load(TM.DEFAULT_PATH)["precision"]) == "df32":
        mlp = TM.load()
    d = P.Dacp(models, psis, block_b=B, precision=P.DACP_DF32)
    try:
        d.set_emax_rule(1)
        d.choose_params(NE)
        d.autotune(64)
        eigs, nf, rank, nfb = d.solve(NE, mlp=mlp)
        p = d.params()
        pick = [0, 77, 128, 255]
        mom = {r: d.moments(r) for r in pick}
        psiE = d.filtered(0)
    finally:
        d.close()
        if mlp is not None:
            P.dacp_mlp_destroy(mlp)
    return dict(models=models, psis=psis, eigs=eigs, nf=nf, rank=rank, p=p, mom=mom, psiE=psiE, pick=pick)


def test_fullsize_counts_and_moment_bounds(batch):
    assert all(int(n) == NE for n in batch["nf"])
    for r, mu in batch["mom"].items():
        diag = np.einsum("jpp->jp", mu)
        m0 = diag[0]
        assert np.allclose(m0, 1.0, atol=1e-12)                 # normalised columns
        assert np.all(np.abs(diag) <= m0 * (1 + 1e-9)), r      # |T_j| <= 1 on the spectrum
    for r in range(R):
        e = np.asarray(batch["eigs"][r])
        assert np.all(np.diff(e) >= 0) and np.abs(e).max() <= batch["p"]["a"][r] * (1 + 1e-12)


def test_fullsize_filter_and_moments_vs_oracle(batch):
    m, psi, p = batch["models"][0], batch["psis"][0], batch["p"]
    emax, a, K = float(p["emax"][0]), float(p["a"][0]), int(p["K"][0])
    ref = DA.exp_semicircle_filter(m, psi, emax, a, K)
    got = batch["psiE"]
    # double-float round-off u = 2^-44 per operation over K ~ 10^3 orders gives ~K u ~ 1e-10 relative;
    # 1e-7 leaves room for the filter's amplification and is far below float32's ~1e-4
    assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max()
    kmax = 60
    mu_ref, _ = DA.chebyshev_moments(m, ref, emax, kmax)
    mu_ref = 0.5 * (mu_ref + np.transpose(mu_ref, (0, 2, 1)))
    mu = batch["mom"][0][:kmax + 1]
    assert np.abs(mu - mu_ref).max() < 1e-7                    # |mu| <= 1; inherits the psi_E difference


def test_fullsize_sampled_levels_vs_float64_dacp(batch):
    pick = batch["pick"]
    d = P.Dacp([batch["models"][r] for r in pick], [batch["psis"][r] for r in pick], block_b=B,
               precision=P.DACP_FP64)
    try:
        d.choose_params(NE, c_order=18.0)
        ref, nf, _ = d.run(NE)
    finally:
        d.close()
    for j, r in enumerate(pick):
        assert nf[j] == NE
        ok, err = TM.accurate(np.asarray(batch["eigs"][r])[:NE], np.asarray(ref[j])[:NE])
        assert ok, (r, err)


def test_fullsize_levels_vs_exact_levels(batch):
    """All 500 central levels of the four shards with a stored dense spectrum, level by level."""
    exact = {}
    for row in read_golden("shard14_dense_central_levels.txt"):
        if len(row) == 2:
            exact.setdefault(int(row[0]), []).append(float(row[1]))
    assert sorted(exact) == [0, 64, 128, 192]
    for r, lv in sorted(exact.items()):
        lv = np.sort(np.asarray(lv))                         # the 640 levels nearest E = 0
        ref = MT.central_exact(lv, NE)
        got = np.sort(np.asarray(batch["eigs"][r]))
        assert len(got) == NE, r
        first = int(np.searchsorted(lv, ref[0]))            # ref is a contiguous run of lv
        assert np.array_equal(lv[first:first + NE], ref)
        spacing = np.array([MT.local_spacing(lv, first + i) for i in range(NE)])
        err = np.abs(got - ref) / spacing
        assert err.max() <= 1e-2, (r, float(err.max()), int(np.argmax(err)))
