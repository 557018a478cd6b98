"""The Ritz-residual E_max rule (dacp_set_emax_rule(h, 1)) on the GPU.

Sec. II A needs E_max to bound |E|: a level beyond it grows exponentially in
both recurrences. Sec. III cites a Lanczos upper-bound estimator; rule 1 adds
only the largest residual of any Ritz pair to the extreme Ritz value, where
rule 0 adds the whole residual norm. Rule 1 is a bound in practice, not in
theory, so it is checked here where the exact spectral radius is known: the
four N = 14 benchmark shards and the N = 16 mixed-field chain, whose extreme
levels are stored in tests/golden (dense eigh, oracle-only scripts).

  * E_max from the device (64 Lanczos steps on column 0 of the start block:
    rule 1 runs the recurrence on past rule 0's 20 steps; eigenvector-free
    interlacing form) equals oracle.params.emax_bound(rule="ritz", steps=64)
    to 1e-5 relative, and is never below the exact radius (1.08 and 1.066
    times it on the shards and the chain). The tolerance is the recurrence's
    own sensitivity: without reorthogonalisation the Lanczos vectors lose
    orthogonality, and a start vector perturbed by 1e-15 relative moves the
    64-step bound of the uniform chain by 1.0e-6 relative (of the shards by
    8e-15); the interlacing form itself matches eigh of the same tridiagonal
    to rounding (dacp_test_emax_rule). Rule 0's 20-step bound matches the
    oracle to 1e-9;
  * it is smaller than rule 0's bound, so the filter order K and the last
    basis order k_n shrink with it;
  * the levels computed with it still meet the float64 target: within 1e-9
    of the spectral width of the exact levels.
"""

import numpy as np
import pytest

import workloads as W
from oracle import metrics as MT
from oracle import params as OP
from tests.conftest import read_golden

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")


def _shard_golden():
    bounds, levels = {}, {}
    for row in read_golden("shard14_dense_central_levels.txt"):
        if len(row) == 3:
            bounds[int(row[0])] = (float(row[1]), float(row[2]))
        else:
            levels.setdefault(int(row[0]), []).append(float(row[1]))
    return bounds, {k: np.sort(np.asarray(v)) for k, v in levels.items()}


def _params(models, psis, rule, n_eigs):
    d = P.Dacp(models, psis, block_b=4, precision=P.DACP_FP64)
    try:
        d.set_emax_rule(rule)
        d.choose_params(n_eigs)
        return d.params()
    finally:
        d.close()


def _run_rule1(models, psis, n_eigs):
    d = P.Dacp(models, psis, block_b=4, precision=P.DACP_FP64)
    try:
        d.set_emax_rule(1)
        d.choose_params(n_eigs)
        eigs, nf, _ = d.run(n_eigs)
        return d.params(), eigs, nf
    finally:
        d.close()


def _check_bounds(models, psis, p1, p0, radii):
    for r, m in enumerate(models):
        ref = OP.emax_bound(m, psis[r][:, 0], steps=64, rule="ritz")
        ref0 = OP.emax_bound(m, psis[r][:, 0], steps=20, rule="residual")
        assert abs(p0["emax"][r] - ref0) <= 1e-9 * ref0, (r, p0["emax"][r], ref0)
        assert abs(p1["emax"][r] - ref) <= 1e-5 * ref, (r, p1["emax"][r], ref)
        assert p1["emax"][r] >= radii[r], (r, p1["emax"][r], radii[r])
        assert p1["emax"][r] < p0["emax"][r]
        assert p1["K"][r] < p0["K"][r] and p1["kn"][r] < p0["kn"][r]


def test_ritz_rule_on_benchmark_shards():
    bounds, levels = _shard_golden()
    seeds = sorted(bounds)
    models = [W.spin_glass_shard(14, seed=s) for s in seeds]
    psis = [W.start_vectors(14, 4, seed=0, r=s) for s in seeds]   # the benchmark's start vectors
    p0 = _params(models, psis, 0, 500)
    p1, eigs, nf = _run_rule1(models, psis, 500)
    radii = [max(-bounds[s][0], bounds[s][1]) for s in seeds]
    _check_bounds(models, psis, p1, p0, radii)
    for j, s in enumerate(seeds):
        assert nf[j] == 500
        ref = MT.central_exact(levels[s], 500)
        width = bounds[s][1] - bounds[s][0]
        err = np.abs(np.sort(np.asarray(eigs[j])) - ref)
        assert err.max() <= 1e-9 * width, (s, float(err.max() / width))


def test_ritz_rule_on_n16_chain():
    rows = read_golden("chain16_dense_central_levels.txt")
    emin, emax = float(rows[0][0]), float(rows[0][1])
    lv = np.sort(np.array([float(r[0]) for r in rows[1:]]))
    models = [W.chain(16)]
    psis = [W.start_vectors(16, 4, seed=0)]
    p0 = _params(models, psis, 0, 1000)
    p1, eigs, nf = _run_rule1(models, psis, 1000)
    _check_bounds(models, psis, p1, p0, [max(-emin, emax)])
    assert nf[0] == 1000
    err = np.abs(np.sort(np.asarray(eigs[0])) - MT.central_exact(lv, 1000))
    assert err.max() <= 1e-9 * (emax - emin), float(err.max() / (emax - emin))
