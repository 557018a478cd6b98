"""GPU parity of H.v at the largest sizes the library takes (N up to 26 spins).

These vectors have many beyond-tile bits: 16 at N = 26 with 8 KB float64 tiles,
13 at N = 24 with the double-float b = 4 tiles of the benchmark. So the flips
past the compile-time-unrolled ones run too, along with the 64-bit offsets and
the 32-bit per-state offsets of the double-float pass. The oracle evaluates
sampled output rows one by one from the definition (``apply_h_rows``). The
samples are the first and last states, each side of several tile boundaries,
and random states. The tolerances are the summation bounds of the path's
arithmetic, with a factor 4 of margin:
  * the row sum: (N + 3) u sum_k |term_k|, with u = 2^-53 (float64), 2^-24
    (float32: the oracle sees the float32-rounded input; the couplings and the
    diagonal are rounded to float32 on the device) or 2^-44 (double-float,
    about 2^-44 per error-free step);
  * the diagonal, a float64 sum of N(N+1)/2 terms formed in different orders
    on the two sides: (N(N+1)/2 + 1) 2^-53 (sum|J| + sum|h|) |x[s]|.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from tests.conftest import df32_pack, df32_unpack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2011_02107_gb300")


def _rows(N, tile_states, seed):
    D = 1 << N
    rng = np.random.default_rng(seed)
    t = np.array([1, 2, 3, 5, 7, (D // tile_states) - 1]) * tile_states
    edges = np.concatenate([t - 1, t])
    return np.unique(np.concatenate([[0, 1, D - 2, D - 1], edges, rng.integers(0, D, size=3000)]))


@pytest.mark.parametrize("N,b,prec,tile", [
    (26, 1, "fp64", 8192),      # kMaxSpins; 10 tile bits, 16 beyond
    (25, 2, "fp32", 8192),      # 10 tile bits, 15 beyond
    (24, 4, "df32", 65536),     # the benchmark's vector format: 11 tile bits, 13 beyond
])
def test_apply_h_at_maximum_size(N, b, prec, tile):
    m = W.random_model(N, seed=90 + N)
    code = {"fp64": P.DACP_FP64, "fp32": P.DACP_FP32, "df32": P.DACP_DF32}[prec]
    esz = {"fp64": 8, "fp32": 4, "df32": 8}[prec]
    x = W.start_vectors(N, b, seed=3)
    d = P.Dacp([m], [x], block_b=b, precision=code)
    try:
        d.set_launch(0, tile)
        tile_states = tile // (b * esz)
        rows = _rows(N, tile_states, seed=N)
        if prec == "fp64":
            xd = torch.from_numpy(x).cuda()
            xin = x
        elif prec == "fp32":
            xd = torch.from_numpy(x.astype(np.float32)).cuda()
            xin = x.astype(np.float32).astype(np.float64)
        else:
            packed = df32_pack(x)
            xd = torch.from_numpy(packed).cuda()
            xin = df32_unpack(packed, b)
            del packed
        yd = torch.zeros_like(xd)
        d.apply_h(0, xd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        idx = torch.from_numpy(rows).cuda()
        got = yd[idx].double().cpu().numpy()
        if prec == "df32":
            got = df32_unpack(got, b)
        del xd, yd
        ref, scale = Hm.apply_h_rows(m, xin, rows, with_abs=True)
        unit = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "df32": 2.0 ** -44}[prec]
        # the diagonal is a float64 sum of N(N+1)/2 terms on both sides, in different orders
        dscale = (np.abs(np.triu(m["J"], 1)).sum() + np.abs(m["h"]).sum()) * np.abs(xin[rows])
        tol = 4 * ((N + 3) * unit * scale + (N * (N + 1) // 2 + 1) * 2.0 ** -53 * dscale)
        err = np.abs(got - ref)
        assert (err <= tol).all(), (prec, float(err.max()), float((err / scale).max()))
    finally:
        d.close()
