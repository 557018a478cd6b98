"""GPU parity with two-body flip couplings (XX and YY terms; dacp_set_pair_couplings).

H gains sum_{i<j} (Jxx_ij X_i X_j + Jyy_ij Y_i Y_j): the XXZ / Heisenberg
chains, and the paper's native sigma^x sigma^x couplings (Sec. III) without the
rotation. The oracle's pair-flip apply is pinned by Kronecker products and the
free-fermion XX chain (tests/test_oracle_*). Tolerances:
  * H.v: 4 (terms + 3) u sum_k |term_k| per row, u the path's unit round-off
    (2^-53 float64, 2^-24 float32 with the float32-rounded input, 2^-44
    double-float), plus the float64 diagonal's own (N(N+1)/2 + 1) 2^-53
    (sum|J| + sum|h|) |x[s]|, as in the maximum-size parity test;
  * central eigenvalues: the float64 target 1e-9 of the spectral width, and
    for double-float 1e-8 of the width and 1e-2 of the local mean spacing.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from oracle import metrics as MT
from tests.conftest import df32_pack, df32_unpack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2011_02107_gb300")


def _all_pairs(N, seed):
    m = W.random_model(N, seed=seed)
    rng = np.random.default_rng(seed + 7)
    m["Jxx"] = np.triu(rng.uniform(-1.0, 1.0, (N, N)), 1)
    m["Jyy"] = np.triu(rng.uniform(-1.0, 1.0, (N, N)), 1)
    return m


def _batch():
    # pairs inside and beyond 8 KB tiles, a realization without pairs, N = 2
    return [W.heisenberg_chain(10, seed=1), _all_pairs(12, seed=2), W.random_model(9, seed=3),
            W.heisenberg_chain(2, seed=4), _all_pairs(11, seed=5)]


def _to_dev(x, prec):
    if prec == "fp64":
        return torch.from_numpy(x).cuda(), x
    if prec == "fp32":
        return torch.from_numpy(x.astype(np.float32)).cuda(), x.astype(np.float32).astype(np.float64)
    packed = df32_pack(x)
    return torch.from_numpy(packed).cuda(), df32_unpack(packed, x.shape[1])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df32"])
@pytest.mark.parametrize("b", [1, 2, 4])
def test_apply_h_with_pair_couplings(prec, b):
    models = _batch()
    code = {"fp64": P.DACP_FP64, "fp32": P.DACP_FP32, "df32": P.DACP_DF32}[prec]
    psis = [W.start_vectors(m["N"], b, seed=11, r=i) for i, m in enumerate(models)]
    d = P.Dacp(models, psis, block_b=b, precision=code)
    try:
        d.set_launch(0, 8192)
        for r, m in enumerate(models):
            x = W.start_vectors(m["N"], b, seed=12, r=r)
            xd, xin = _to_dev(x, prec)
            yd = torch.zeros_like(xd)
            d.apply_h(r, xd.data_ptr(), yd.data_ptr())
            torch.cuda.synchronize()
            got = yd.double().cpu().numpy()
            if prec == "df32":
                got = df32_unpack(got, b)
            rows = np.arange(1 << m["N"])
            ref, scale = Hm.apply_h_rows(m, xin, rows, with_abs=True)
            assert np.abs(Hm.apply_h(m, xin) - ref).max() <= 1e-12 * np.abs(ref).max()
            N = m["N"]
            Jxx, Jyy = Hm.pair_couplings(m)
            terms = N + int(np.count_nonzero((Jxx != 0) | (Jyy != 0)))
            unit = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "df32": 2.0 ** -44}[prec]
            dscale = (np.abs(np.triu(m["J"], 1)).sum() + np.abs(m["h"]).sum()) * np.abs(xin)
            tol = 4 * ((terms + 3) * unit * scale + (N * (N + 1) // 2 + 1) * 2.0 ** -53 * dscale)
            err = np.abs(got - ref)
            assert (err <= tol).all(), (r, N, float(err.max()), float((err / scale).max()))
    finally:
        d.close()


@pytest.mark.parametrize("prec", ["fp64", "df32"])
def test_heisenberg_end_to_end_vs_dense(prec):
    """Random-field Heisenberg chains (XX + YY + ZZ) in a batch with a plain
    Ising chain: heuristic parameters, filter, evolution and subspace solve all
    run with the pair flips. The central levels are checked against dense
    eigh."""
    models = [W.heisenberg_chain(10, seed=4, W=2.0), W.heisenberg_chain(9, seed=7, W=2.0), W.chain(9)]
    psis = [W.start_vectors(m["N"], 4, seed=5, r=i) for i, m in enumerate(models)]
    code = P.DACP_FP64 if prec == "fp64" else P.DACP_DF32
    d = P.Dacp(models, psis, block_b=4, precision=code)
    try:
        d.choose_params(60)
        p = d.params()
        d.filter()
        d.basis_moments()
        eigs, nf, rank = d.central_eigs(60)
        for r, m in enumerate(models):
            E = np.linalg.eigvalsh(Hm.dense_h(m))
            assert p["emax"][r] >= np.abs(E).max()
            assert nf[r] == 60, (r, nf[r])
            err = np.abs(eigs[r] - MT.central_exact(E, 60)).max()
            width = E[-1] - E[0]
            if prec == "fp64":
                assert err < 1e-9 * width, (r, err)
            else:
                assert err < 1e-8 * width, (r, err)
                mt = MT.match(eigs[r], E)
                assert mt["n_unmatched"] == 0 and mt["spacing_err"].max() < 1e-2
    finally:
        d.close()


def test_pair_couplings_reset_state_and_can_be_removed():
    m = W.heisenberg_chain(8, seed=2)
    psi = W.start_vectors(8, 1, seed=3)
    d = P.Dacp([m], [psi], block_b=1, precision=P.DACP_FP64)
    try:
        d.choose_params(20)
        z = np.zeros(64)
        P.dacp_set_pair_couplings(d.handle, z, z)       # all zero: the plain zz / z / x operator
        with pytest.raises(P.DacpError) as e:
            d.filter()                                   # parameters were reset
        assert e.value.status == 6
        x = W.start_vectors(8, 1, seed=4)
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        d.apply_h(0, xd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        plain = {k: v for k, v in m.items() if k not in ("Jxx", "Jyy")}
        ref = Hm.apply_h(plain, x)
        assert np.abs(yd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
        bad = np.full(64, np.nan)
        with pytest.raises(P.DacpError) as e:
            P.dacp_set_pair_couplings(d.handle, bad, z)
        assert e.value.status == 1
    finally:
        d.close()
