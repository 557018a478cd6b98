"""Host side of the parity-sector path (CPU only): dacp_merge_sectors and the refusals of
dacp_create_parity_sectors, both before any device use.

The merge returns, per realization, the n_eigs levels of smallest |E| of the union of its two
sectors' levels, but only up to the smaller of the two sectors' largest |E|: beyond that radius a
sector may hold levels it did not return, so the union cannot vouch for them.
"""

import numpy as np
import pytest

P = pytest.importorskip("paper_2011_02107_gb300")


def test_merge_takes_the_central_union_within_both_radii():
    a = np.array([-0.30, -0.10, 0.05, 0.20])          # sector +1, its 4 levels nearest 0
    b = np.array([-0.21, -0.02, 0.12, 0.25])          # sector -1
    eigs, nf = P.dacp_merge_sectors(np.stack([a, b]), np.array([4, 4]), 5)
    assert nf[0] == 5
    assert np.allclose(eigs[0], [-0.10, -0.02, 0.05, 0.12, 0.20])   # |0.20| < |0.21|
    # asking for more than the radii cover: sector +1 reaches |E| = 0.30, sector -1 only 0.25
    eigs, nf = P.dacp_merge_sectors(np.stack([a, b]), np.array([4, 4]), 8)
    assert nf[0] == 7 and np.allclose(eigs[0, :7], [-0.21, -0.10, -0.02, 0.05, 0.12, 0.20, 0.25])


def test_merge_passes_a_failed_sector_on_and_handles_short_sectors():
    x = np.zeros((4, 3))
    x[0] = [-0.1, 0.2, 0.3]
    x[1] = [-0.05, 0.0, 0.0]                           # sector -1 of realization 0 found one level
    x[2] = [0.0, 0.0, 0.0]
    x[3] = [0.01, 0.02, 0.03]
    eigs, nf = P.dacp_merge_sectors(x, np.array([3, 1, -4, 3]), 2)
    assert nf[0] == 1 and eigs[0, 0] == -0.05          # the short sector's radius is 0.05
    assert nf[1] == -4                                 # DACP_ERR_NUMERIC of sector +1 of realization 1


def test_parity_sectors_refuse_z_fields_and_tiny_models():
    n = np.array([4], dtype=np.int32)
    J = np.zeros(16)
    for h, nsp in ((np.full(4, 0.1), n), (np.zeros(1), np.array([1], dtype=np.int32))):
        with pytest.raises(P.DacpError) as e:
            P.dacp_create_parity_sectors(nsp, J[:nsp[0] ** 2], h[:nsp[0]], np.ones(nsp[0]), 1, 0,
                                         np.zeros(2 * (1 << max(nsp[0] - 1, 0))))
        assert e.value.status == 1


def test_merge_of_dense_sector_spectra_gives_the_full_central_levels():
    """The library's host merge on real spectra: each sector's n_sec levels of smallest |E| (dense
    eigh of the oracle's sector models, reading of the global-flip split) merge to exactly the full
    model's n central levels (dense eigh of the full model)."""
    import workloads as W
    from oracle import hamiltonian as Hm
    from oracle import metrics as MT
    for N, n, seed in ((8, 30, 1), (9, 50, 2), (10, 60, 3)):
        m = W.spin_glass_shard(N, seed=seed)
        full = np.linalg.eigvalsh(Hm.dense_h(m))
        n_sec = n // 2 + 6
        rows, nfs = [], []
        for ms in Hm.parity_sector_models(m):
            E = np.linalg.eigvalsh(Hm.dense_h(ms))
            rows.append(np.sort(E[np.argsort(np.abs(E), kind="stable")[:n_sec]]))
            nfs.append(n_sec)
        eigs, nf = P.dacp_merge_sectors(np.stack(rows), np.array(nfs), n)
        assert nf[0] == n
        assert np.abs(eigs[0] - MT.central_exact(full, n)).max() < 1e-12 * (full[-1] - full[0])


def test_sector_level_rule_covers_the_sector_split():
    """The benchmark asks each sector for half of n_eigs plus 1 % (at least 5 levels). On 24 shards
    at N = 10 (60 levels) and 8 at N = 11 (120 levels) the larger sector's share of the central
    levels, from dense sector spectra, stays at least 2 levels inside that rule."""
    import os
    import sys
    import workloads as W
    from oracle import hamiltonian as Hm
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench as B
    for N, n, seeds in ((10, 60, range(24)), (11, 120, range(8))):
        worst = 0
        for s in seeds:
            m = W.spin_glass_shard(N, seed=100 + s)
            sp = [np.linalg.eigvalsh(Hm.dense_h(ms)) for ms in Hm.parity_sector_models(m)]
            lab = np.concatenate([np.zeros(len(sp[0])), np.ones(len(sp[1]))])
            idx = np.argsort(np.abs(np.concatenate(sp)), kind="stable")[:n]
            worst = max(worst, int(max((lab[idx] == 0).sum(), (lab[idx] == 1).sum())))
        assert worst + 2 <= B.sector_levels(n), (N, n, worst, B.sector_levels(n))
