"""The exact central levels of four benchmark shards, and the benchmark's check against them.

``tests/golden/shard14_dense_central_levels.txt`` holds, for realizations 0, 64,
128 and 192 of the 256-shard N = 14 batch, the 640 levels nearest E = 0 from
dense float64 eigh, written by ``tests/golden/make_shard_dense_levels.py``. That
script uses only the oracle's matrix-free apply (pinned to Kronecker products)
and LAPACK. Here the fixture is checked for its shape and for bounds that the
mathematics fixes. ``bench.exact_accuracy``, which the benchmark line uses to
report the timed path's error against these levels, is checked on exact and
perturbed inputs.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from tests.conftest import read_golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _levels():
    out = {}
    for row in read_golden("shard14_dense_central_levels.txt"):
        d = out.setdefault(int(row[0]), {"v": []})
        if len(row) == 3:
            d["emin"], d["emax"] = float(row[1]), float(row[2])
        else:
            d["v"].append(float(row[1]))
    return out


def test_fixture_shape_and_bounds():
    lv = _levels()
    assert sorted(lv) == [0, 64, 128, 192]
    for seed, d in lv.items():
        v = np.array(d["v"])
        assert len(v) == 640 and np.all(np.diff(v) >= 0)
        assert v[0] < 0 < v[-1]                              # the window around E = 0
        m = W.spin_glass_shard(14, seed=seed)
        assert -Hm.pauli_norm_bound(m) <= d["emin"] < v[0] and v[-1] < d["emax"] <= Hm.pauli_norm_bound(m)
        # Tr H^2 / D = sum J^2 + sum Gamma^2 bounds the extreme levels: E_max^2 <= D Tr H^2 / D
        assert max(-d["emin"], d["emax"]) ** 2 <= (1 << 14) * Hm.trace_h2_per_state(m)
        # the central spacing is of the order the Gaussian density of states gives, 1/rho(0)
        sigma = np.sqrt(Hm.trace_h2_per_state(m))
        spacing = np.sqrt(2 * np.pi) * sigma / (1 << 14)
        assert 0.3 * spacing < np.mean(np.diff(v)) < 3.0 * spacing


@pytest.fixture(scope="module")
def bench():
    lib = os.path.join(ROOT, "paper_2011_02107_gb300", "libdacp.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    import bench as B
    return B


def test_exact_accuracy_reports_errors_in_spacings(bench):
    lv = _levels()
    n = 500
    central = {s: np.sort(np.array(d["v"])[np.argsort(np.abs(d["v"]), kind="stable")[:n]]) for s, d in lv.items()}
    last = [np.array([]) for _ in range(256)]
    for s, c in central.items():
        last[s] = c.copy()
    wl = bench.WORKLOADS["c3"]
    out = bench.exact_accuracy(wl, 0, last, n)
    assert out["realizations"] == [0, 64, 128, 192] and out["max_spacing_err"] == 0.0 and out["within_1e-2"] == 4
    # shift one level of shard 64 by half its local mean spacing (+-10 levels)
    c = central[64]
    i = 250
    sp = (c[i + 10] - c[i - 10]) / 20
    last[64] = c.copy()
    last[64][i] += 0.5 * sp
    out = bench.exact_accuracy(wl, 0, last, n)
    assert abs(out["max_spacing_err"] - 0.5) < 1e-9 and out["within_1e-2"] == 3
    assert out["median_spacing_err"] == 0.0 and out["p99_spacing_err"] < 0.5
    # a short list counts as a miss; other workloads and ranks are not checked
    last[0] = central[0][:10]
    assert bench.exact_accuracy(wl, 0, last, n)["max_spacing_err"] == float("inf")
    assert bench.exact_accuracy(bench.WORKLOADS["c1"], 0, last, n) is None
    assert bench.exact_accuracy(wl, 1, last, n) is None


def test_chain16_fixture_shape_and_bounds():
    """The N = 16 mixed-field chain's exact central levels (two mirror-sector
    blocks, tests/golden/make_chain16_dense_levels.py): 1100 sorted levels
    around E = 0 inside the Pauli bound, with the Gaussian-density spacing."""
    rows = read_golden("chain16_dense_central_levels.txt")
    emin, emax = float(rows[0][0]), float(rows[0][1])
    v = np.array([float(r[0]) for r in rows[1:]])
    m = W.chain(16)
    assert len(v) == 1100 and np.all(np.diff(v) >= 0) and v[0] < 0 < v[-1]
    assert -Hm.pauli_norm_bound(m) <= emin < v[0] and v[-1] < emax <= Hm.pauli_norm_bound(m)
    assert max(-emin, emax) ** 2 <= (1 << 16) * Hm.trace_h2_per_state(m)
    spacing = np.sqrt(2 * np.pi) * np.sqrt(Hm.trace_h2_per_state(m)) / (1 << 16)
    assert 0.3 * spacing < np.mean(np.diff(v)) < 3.0 * spacing


def test_exact_accuracy_on_the_chain(bench):
    rows = read_golden("chain16_dense_central_levels.txt")
    v = np.array([float(r[0]) for r in rows[1:]])
    n = 1000
    central = np.sort(v[np.argsort(np.abs(v), kind="stable")[:n]])
    out = bench.exact_accuracy(bench.WORKLOADS["c2"], 0, [central], n)
    assert out["realizations"] == [0] and out["max_spacing_err"] == 0.0 and out["within_1e-2"] == 1
