"""What the trained parameter network gains over the method without it (GPU).

Held-out spin-glass shards (seeds the training never saw, sizes at and just
beyond the training range) are solved three ways on the GPU:

  * reference: plain float64 DACP with the paper's parameters (c = 18,
    window ratio 2, basis ratio 1.5 -- Sec. II A, II B);
  * heuristic: double-float DACP with the same heuristic parameters;
  * learned:   double-float DACP with the network's window / order / basis
    (dacp_choose_params_mlp), heuristic fallback for short realizations.

The learned run must keep every requested level within 1e-2 of the local
mean spacing of the reference, and cost less than the heuristic run: at
least 10 % less in the GB300 cost model (stencil value-orders + M^3 subspace
term), and less in the measured T_F + T_E + T_D of the library's own CUDA
events. At N = 16 (beyond the training range, 1000 levels) the evolution's
k_n = n pi E_max / a hardly moves (the network narrows window and basis
together; on 16 N = 18 shards with 2000 levels it ran 840838 orders against
840152), so the gain there is in the filter and the solve: the learned run
must still cost less in the model and in the measured path.
"""

import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")
from paper_2011_02107_gb300 import train_mlp as TM  # noqa: E402

WEIGHTS = TM.DEFAULT_PATH


def _run(models, psis, prec, n_eigs, mlp=None, **kw):
    """Both arms through the same call (dacp_solve, solves overlapped with the evolution)."""
    d = P.Dacp(models, psis, block_b=4, precision=prec)
    try:
        if mlp is not None:
            eigs, nf, rank, nfb = d.solve(n_eigs, mlp=mlp)
        else:
            d.choose_params(n_eigs, **kw)
            eigs, nf, rank = d.run(n_eigs)
            nfb = 0
        p = d.params()
        ms = d.timings()
    finally:
        d.close()
    return eigs, nf, p, ms, nfb


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained weights")
def test_learned_parameters_keep_accuracy_and_cut_cost():
    z = np.load(WEIGHTS)
    if str(z["precision"]) != "df32":
        pytest.skip("weights trained for another precision")
    mlp = TM.load(WEIGHTS)
    try:
        for N, ne, seeds in ((12, 100, range(900_000, 900_006)), (13, 200, range(910_000, 910_004)),
                             (16, 1000, range(920_000, 920_002))):
            models = [W.spin_glass_shard(N, seed=s) for s in seeds]
            psis = [W.start_vectors(N, 4, seed=77, r=i) for i in range(len(models))]
            ref, nf_ref, _, _, _ = _run(models, psis, P.DACP_FP64, ne, c_order=18.0)
            heu, nf_h, p_h, ms_h, _ = _run(models, psis, P.DACP_DF32, ne)
            lrn, nf_l, p_l, ms_l, nfb = _run(models, psis, P.DACP_DF32, ne, mlp=mlp)
            for r in range(len(models)):
                assert nf_ref[r] == ne and nf_l[r] == ne
                ok, err = TM.accurate(np.asarray(lrn[r])[:ne], ref[r][:ne])
                assert ok, (N, r, err)
            cost_h = sum(TM.cost(N, 4, p_h, r) for r in range(len(models)))
            cost_l = sum(TM.cost(N, 4, p_l, r) for r in range(len(models)))
            # the eligible knob settings all keep the basis ratio 1.5: the gain comes from the
            # window and the filter order (at most ~25 %)
            assert cost_l < (0.9 if N < 16 else 1.0) * cost_h, (N, cost_l, cost_h)
            # whole measured path: the learned knobs keep the basis ratio (so T_E is alike) and
            # save in the filter and the subspace solve
            assert sum(ms_l) < sum(ms_h), (N, ms_l, ms_h)
    finally:
        P.dacp_mlp_destroy(mlp)


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained weights")
def test_learned_parameters_on_parity_sectors():
    """The benchmark's use of the network: held-out N = 14 shards solved as their parity
    sectors (255 of 500 levels per sector, E_max rule 1), learned knobs against the
    heuristic. The merged levels of the learned run must match plain float64 DACP on
    the full shards within 1e-2 of the local spacing, and the learned run must cost
    less, in the GB300 cost model and in the measured T_F + T_E + T_D of a second run
    (the first run of each kind in a process also pays one-time set-up: module loads,
    graph captures). Measured on GB300 with 8 and 64 shards: 560 against 603 ms and
    1749 against 1928 ms, modelled cost 0.74 of the heuristic's."""
    z = np.load(WEIGHTS)
    if str(z["precision"]) != "df32":
        pytest.skip("weights trained for another precision")
    mlp = TM.load(WEIGHTS)
    N, ne, n_sec = 14, 500, 255
    models = [W.spin_glass_shard(N, seed=s) for s in range(930_000, 930_016)]
    full_psis = [W.start_vectors(N, 4, seed=77, r=i) for i in range(len(models))]
    sec_psis = [p for i in range(len(models)) for p in W.sector_start_vectors(N, 4, seed=77, r=i)]

    def sectors(learned):
        d = P.Dacp.parity_sectors(models, sec_psis, block_b=4, precision=P.DACP_DF32)
        try:
            d.set_emax_rule(1)
            if learned:
                eigs, nf, _, _ = d.solve(n_sec, mlp=mlp)
            else:
                d.choose_params(n_sec)
                eigs, nf, _ = d.run(n_sec)
            p, ms = d.params(), d.timings()
        finally:
            d.close()
        merged, nfm = P.merge_sector_levels(eigs, nf, ne)
        return merged, nfm, sum(TM.cost(N - 1, 4, p, r) for r in range(2 * len(models))), sum(ms)

    try:
        ref, nf_ref, _, _, _ = _run(models, full_psis, P.DACP_FP64, ne, c_order=18.0)
        sectors(False)
        sectors(True)
        _, _, cost_h, ms_h = sectors(False)
        lrn, nf_l, cost_l, ms_l = sectors(True)
        for r in range(len(models)):
            assert nf_ref[r] == ne and nf_l[r] == ne
            ok, err = TM.accurate(np.asarray(lrn[r])[:ne], np.asarray(ref[r])[:ne])
            assert ok, (r, err)
        assert cost_l < cost_h, (cost_l, cost_h)
        assert ms_l < ms_h, (ms_l, ms_h)
    finally:
        P.dacp_mlp_destroy(mlp)
