"""GPU parity of the global-flip term and of the parity-sector path.

  * H.v with the global flip c X_0 ... X_{N-1} (dacp_set_global_flips) against the oracle's
    apply (pinned to Kronecker products), in float64, float32 and double-float with b = 1, 2, 4,
    for realizations of one tile and of several (8 KB tiles);
  * the parity sectors of spin-glass shards (dacp_create_parity_sectors; h = 0): sector levels
    merged by dacp_merge_sectors against the full models' dense spectra, float64, within 1e-9 of
    the width; the merge is exact because the union of the sector spectra is the spectrum (the
    oracle's pin, test_oracle_hamiltonian);
  * the benchmark's sector path (double-float, E_max rule 1, the shipped parameter network,
    255 levels per sector, dacp_solve_sectors merging to 500) on the four shards with stored exact
    levels, within 1e-2 of the local mean spacing (Sec. III accuracy measure);
  * dacp_solve_sectors re-solving short merges, and its refusals.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from oracle import metrics as MT
from tests.conftest import df32_pack, df32_unpack, read_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")


def _with_flip(m, c):
    m = dict(m)
    m["gflip"] = c
    return m


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df32"])
@pytest.mark.parametrize("b", [1, 2, 4])
def test_apply_h_with_global_flip(prec, b):
    models = [_with_flip(W.random_model(N, seed=30 + N), 0.37 * (-1) ** N) for N in (1, 2, 9, 13)]
    code = {"fp64": P.DACP_FP64, "fp32": P.DACP_FP32, "df32": P.DACP_DF32}[prec]
    psis = [W.start_vectors(m["N"], b, seed=5, r=i) for i, m in enumerate(models)]
    d = P.Dacp(models, psis, block_b=b, precision=code)
    try:
        d.set_launch(0, 8192)
        for r, m in enumerate(models):
            x = W.start_vectors(m["N"], b, seed=9, r=r)
            if prec == "fp64":
                xd, xin = torch.from_numpy(x).cuda(), x
            elif prec == "fp32":
                xd, xin = torch.from_numpy(x.astype(np.float32)).cuda(), x.astype(np.float32).astype(np.float64)
            else:
                pk = df32_pack(x)
                xd, xin = torch.from_numpy(pk).cuda(), df32_unpack(pk, b)
            yd = torch.zeros_like(xd)
            torch.cuda.synchronize()
            d.apply_h(r, xd.data_ptr(), yd.data_ptr())
            torch.cuda.synchronize()
            got = yd.double().cpu().numpy()
            if prec == "df32":
                got = df32_unpack(got, b)
            N = m["N"]
            ref, scale = Hm.apply_h_rows(m, xin, np.arange(1 << N), with_abs=True)
            assert np.abs(Hm.apply_h(m, xin) - ref).max() <= 1e-12 * np.abs(ref).max()
            unit = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "df32": 2.0 ** -44}[prec]
            dscale = (np.abs(np.triu(m["J"], 1)).sum() + np.abs(m["h"]).sum()) * np.abs(xin)
            tol = 4 * ((N + 4) * unit * scale + (N * (N + 1) // 2 + 1) * 2.0 ** -53 * dscale)
            err = np.abs(got.reshape(ref.shape) - ref)
            assert (err <= tol).all(), (r, N, float(err.max()), float((err / scale).max()))
    finally:
        d.close()


def _sector_starts(models, b, seed):
    return [p for r, m in enumerate(models) for p in W.sector_start_vectors(m["N"], b, seed=seed, r=r)]


def test_sectors_end_to_end_fp64_against_dense():
    models = [W.spin_glass_shard(10, seed=s) for s in (11, 12)]
    n_eigs, n_sec = 60, 36
    d = P.Dacp.parity_sectors(models, _sector_starts(models, 4, 3), block_b=4, precision=P.DACP_FP64)
    try:
        assert d.N == [9, 9, 9, 9]
        d.choose_params(n_sec)
        e, nf, rank = d.run(n_sec)
    finally:
        d.close()
    eigs, nf2 = P.merge_sector_levels(e, nf, n_eigs)
    for r, m in enumerate(models):
        E = np.linalg.eigvalsh(Hm.dense_h(m))
        assert nf2[r] == n_eigs
        ref = MT.central_exact(E, n_eigs)
        assert np.abs(eigs[r] - ref).max() <= 1e-9 * (E[-1] - E[0])


def test_sector_path_at_the_benchmark_size_against_exact_levels():
    exact = {}
    for row in read_golden("shard14_dense_central_levels.txt"):
        if len(row) == 2:
            exact.setdefault(int(row[0]), []).append(float(row[1]))
    seeds = sorted(exact)
    models = [W.spin_glass_shard(14, seed=s) for s in seeds]
    # the benchmark's start vectors are keyed by the shard's index in its batch, which is its seed
    psis = [p for s in seeds for p in W.sector_start_vectors(14, 4, seed=0, r=s)]
    n_eigs, n_sec = 500, 255
    from paper_2011_02107_gb300 import train_mlp as TM
    mlp = TM.load() if os.path.exists(TM.DEFAULT_PATH) else None
    d = P.Dacp.parity_sectors(models, psis, block_b=4, precision=P.DACP_DF32)
    try:
        d.set_emax_rule(1)
        d.choose_params(n_sec)
        d.autotune(64)
        eigs, nf2, _ = d.solve_sectors(n_eigs, n_sec, mlp=mlp)
    finally:
        d.close()
        if mlp is not None:
            P.dacp_mlp_destroy(mlp)
    for j, s in enumerate(seeds):
        lv = np.sort(np.asarray(exact[s]))
        ref = MT.central_exact(lv, n_eigs)
        assert nf2[j] == n_eigs
        first = int(np.searchsorted(lv, ref[0]))
        spacing = np.array([MT.local_spacing(lv, first + i) for i in range(n_eigs)])
        err = np.abs(eigs[j] - ref) / spacing
        assert err.max() <= 1e-2, (s, float(err.max()))


def test_apply_h_with_global_flip_tile_specialised_kernel():
    """Double-float b = 4 with 64 KB tiles (11 in-tile bits, the benchmark's kernel): the flip's
    partner load takes a free early slot when fewer than three bits lie beyond the tile (N = 12,
    13) and is issued late otherwise (N = 14, 15)."""
    models = [_with_flip(W.random_model(N, seed=40 + N), 0.53 * (-1) ** N) for N in (12, 13, 14, 15)]
    psis = [W.start_vectors(m["N"], 4, seed=6, r=i) for i, m in enumerate(models)]
    d = P.Dacp(models, psis, block_b=4, precision=P.DACP_DF32)
    try:
        d.set_launch(0, 65536)
        for r, m in enumerate(models):
            N = m["N"]
            x = W.start_vectors(N, 4, seed=10, r=r)
            pk = df32_pack(x)
            xd, xin = torch.from_numpy(pk).cuda(), df32_unpack(pk, 4)
            yd = torch.zeros_like(xd)
            torch.cuda.synchronize()
            d.apply_h(r, xd.data_ptr(), yd.data_ptr())
            torch.cuda.synchronize()
            got = df32_unpack(yd.cpu().numpy(), 4)
            rows = np.random.default_rng(N).choice(1 << N, size=4096, replace=False)
            ref, scale = Hm.apply_h_rows(m, xin, rows, with_abs=True)
            dscale = (np.abs(np.triu(m["J"], 1)).sum() + np.abs(m["h"]).sum()) * np.abs(xin[rows])
            tol = 4 * ((N + 4) * 2.0 ** -44 * scale + (N * (N + 1) // 2 + 1) * 2.0 ** -53 * dscale)
            err = np.abs(got[rows] - ref)
            assert (err <= tol).all(), (N, float(err.max()), float((err / scale).max()))
    finally:
        d.close()


def test_solve_sectors_resolves_short_merges():
    """dacp_solve_sectors: with n_sector well below n_eigs / 2 every model's merge comes up short and
    both its sectors are solved again (each asked for all n_eigs levels): the levels still match
    dense eigh to 1e-9 of the width. With a comfortable n_sector nothing is redone and the result
    equals run + merge. A handle that is not a parity-sector handle, and n_sector > n_eigs, are
    refused."""
    models = [W.spin_glass_shard(10, seed=s) for s in (21, 22)]
    n_eigs = 60
    dense = [np.linalg.eigvalsh(Hm.dense_h(m)) for m in models]
    for n_sec, redone in ((20, 2), (36, 0)):
        d = P.Dacp.parity_sectors(models, _sector_starts(models, 4, 3), block_b=4, precision=P.DACP_FP64)
        try:
            eigs, nf, nre = d.solve_sectors(n_eigs, n_sec)
            assert nre == redone and all(int(x) == n_eigs for x in nf)
            if redone == 0:
                d.choose_params(n_sec)
                e, nfr, _ = d.run(n_sec)
                ref, _ = P.merge_sector_levels(e, nfr, n_eigs)
                for a, b in zip(eigs, ref):
                    assert np.array_equal(a, b)
            with pytest.raises(P.DacpError) as err:
                d.solve_sectors(n_eigs, n_eigs + 1)
            assert err.value.status == 1
        finally:
            d.close()
        for r, E in enumerate(dense):
            assert np.abs(eigs[r] - MT.central_exact(E, n_eigs)).max() <= 1e-9 * (E[-1] - E[0])
    d = P.Dacp(models, [W.start_vectors(10, 4, seed=3, r=i) for i in range(2)], block_b=4, precision=P.DACP_FP64)
    try:
        with pytest.raises(P.DacpError) as err:
            P.dacp_solve_sectors(d.handle, None, 1, n_eigs, 36)
        assert err.value.status == 1
    finally:
        d.close()
