"""GPU parity of the staged float32 launch (launch mode 2).

Mode 2 stages every HBM read of a tile -- the vector tile H acts on, the
recurrence's previous vectors and the diagonal -- in shared memory by bulk
copies before the CTA computes. The arithmetic, its order and the reductions
are those of the per-order launches (mode 0), so at the same tile size the two
give bit-identical filtered states and moments; the filtered state is also held
against the float64 oracle (Sec. II A, Eq. filter) at the float32 tolerance of
the other parity tests.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dacp as DA
from oracle import hamiltonian as Hm
from oracle import metrics as MT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2011_02107_gb300")


def _run(models, psis, b, mode, tile, n_eigs=None, params=None):
    d = P.Dacp(models, psis, block_b=b, precision=P.DACP_FP32)
    try:
        if params is None:
            d.choose_params(n_eigs)
        else:
            d.set_params(*params)
        d.set_launch(mode, tile)
        assert d.launch() == (mode, tile)
        d.filter()
        d.basis_moments()
        filt = [d.filtered(r) for r in range(len(models))]
        mus = [d.moments(r) for r in range(len(models))]
        eigs = d.central_eigs(n_eigs)[:2] if n_eigs else None
        return filt, mus, eigs
    finally:
        d.close()


@pytest.mark.parametrize("b", [1, 2, 4])
def test_staged_matches_graph_replay_on_ragged_batch(b):
    """Uneven N with tiny realizations (N = 1, 2: scalar path and tiles below one
    16-byte diagonal line, read without staging) between tiled ones (several
    tiles per realization at 8 KB): mode 2 equals mode 0 bit for bit, and the
    filtered states match the oracle."""
    models = [W.spin_glass_shard(11, seed=1), W.random_model(1, seed=2), W.chain(9),
              W.random_model(2, seed=3), W.spin_glass_shard(12, seed=4), W.random_model(3, seed=5)]
    psis = [W.start_vectors(m["N"], b, seed=7, r=i) for i, m in enumerate(models)]
    emax = np.array([Hm.pauli_norm_bound(m) for m in models])
    params = (emax, 0.3 * emax, 8, 3)
    f0, m0, _ = _run(models, psis, b, 0, 8192, params=params)
    f2, m2, _ = _run(models, psis, b, 2, 8192, params=params)
    for r, m in enumerate(models):
        assert np.array_equal(f0[r], f2[r]), r
        assert np.array_equal(m0[r], m2[r]), r
        ref = DA.exp_semicircle_filter(m, psis[r], emax[r], 0.3 * emax[r], 8)
        assert np.abs(f2[r] - ref).max() <= 1e-4


@pytest.mark.parametrize("tile", [16384, 32768, 65536])
def test_staged_end_to_end_at_benchmark_tiles(tile):
    """Spin-glass shards (N = 10, b = 4) with the heuristic parameters at the
    tile sizes the autotuner weighs: bit-identical to mode 0, and the central
    levels within the float32 bound of the other parity tests (no ghost or
    missing level, error below 5e-2 of the local spacing)."""
    models = [W.spin_glass_shard(10, seed=s) for s in range(3)]
    psis = [W.start_vectors(10, 4, seed=9, r=i) for i in range(3)]
    f0, m0, e0 = _run(models, psis, 4, 0, tile, n_eigs=60)
    f2, m2, e2 = _run(models, psis, 4, 2, tile, n_eigs=60)
    assert np.array_equal(e0[0], e2[0], equal_nan=True) and np.array_equal(e0[1], e2[1])
    for r, m in enumerate(models):
        assert np.array_equal(m0[r], m2[r])
        E = np.linalg.eigvalsh(Hm.dense_h(m))
        assert e2[1][r] == 60
        mt = MT.match(e2[0][r], E)
        assert mt["n_unmatched"] == 0
        assert mt["spacing_err"].max() < 5e-2


def test_autotune_may_pick_staged_and_keeps_results():
    """The float32 autotuner weighs mode 2 beside modes 0 and 1; whatever it picks,
    the moments equal those of mode 0 at the same tile size."""
    models = [W.spin_glass_shard(12, seed=s) for s in range(4)]
    psis = [W.start_vectors(12, 4, seed=5, r=i) for i in range(4)]
    emax = np.array([Hm.pauli_norm_bound(m) for m in models])
    params = (emax, 0.25 * emax, 10, 4)
    d = P.Dacp(models, psis, block_b=4, precision=P.DACP_FP32)
    try:
        d.set_params(*params)
        d.autotune(orders=40)
        mode, tile = d.launch()
        assert mode in (0, 1, 2)
        d.filter()
        d.basis_moments()
        mt = [d.moments(r) for r in range(4)]
    finally:
        d.close()
    _, m0, _ = _run(models, psis, 4, 0, tile, params=params)
    for a, b in zip(mt, m0):
        assert np.array_equal(a, b)


def test_staged_mode_argument_errors():
    """Mode 2 is refused for float64 / double-float vectors and for tiles whose
    staged copies exceed shared memory (128 KB at b = 4: 3 tiles + diagonal)."""
    m = W.spin_glass_shard(14, seed=0)
    for prec in (P.DACP_FP64, P.DACP_DF32):
        d = P.Dacp([m], [W.start_vectors(14, 4, seed=0)], block_b=4, precision=prec)
        try:
            with pytest.raises(P.DacpError) as e:
                d.set_launch(2, 32768)
            assert e.value.status == 1
        finally:
            d.close()
    d = P.Dacp([m], [W.start_vectors(14, 4, seed=0)], block_b=4, precision=P.DACP_FP32)
    try:
        with pytest.raises(P.DacpError) as e:
            d.set_launch(2, 131072)
        assert e.value.status == 1
        d.set_launch(2, 65536)
        assert d.launch() == (2, 65536)
    finally:
        d.close()
