"""Write the exact central levels of four benchmark shards (N = 14) to a text fixture.

The benchmark batch is 256 spin-glass shards, N = 14 (workloads.spin_glass_shard,
seeds 0..255). For realizations 0, 64, 128 and 192 this script forms the dense
16384 x 16384 matrix column block by column block with the oracle's matrix-free
apply (oracle.hamiltonian.apply_h, itself pinned to Kronecker products), takes
every eigenvalue with LAPACK eigvalsh, and keeps the 640 levels nearest E = 0
(the 500 central levels of the benchmark plus context for local spacings).
It calls nothing but oracle/ and numpy; about a minute or two per shard on
eight cores.

  python tests/golden/make_shard_dense_levels.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import hamiltonian as Hm  # noqa: E402

N = 14
SEEDS = (0, 64, 128, 192)
KEEP = 640
OUT = os.path.join(HERE, "shard14_dense_central_levels.txt")


def dense_from_apply(m):
    D = 1 << m["N"]
    diag = Hm.diagonal(m)
    H = np.empty((D, D))
    step = 1024
    for c0 in range(0, D, step):
        E = np.zeros((D, step))
        E[np.arange(c0, c0 + step), np.arange(step)] = 1.0
        H[:, c0:c0 + step] = Hm.apply_h(m, E, diag)
    return H


def main():
    rows = []
    for seed in SEEDS:
        m = W.spin_glass_shard(N, seed=seed)
        ev = np.linalg.eigvalsh(dense_from_apply(m))
        idx = np.sort(np.argsort(np.abs(ev), kind="stable")[:KEEP])
        rows.append((seed, ev[idx], ev[0], ev[-1]))
        print(f"shard {seed}: E in [{ev[0]:.6f}, {ev[-1]:.6f}]", flush=True)
    write(rows)


def write(rows):
    """rows: (seed, central levels ascending, E_min, E_max) per shard."""
    with open(OUT, "w") as f:
        f.write("# Exact central levels of spin-glass shards N = 14 (workloads.spin_glass_shard(14, seed)),\n")
        f.write("# the benchmark batch's realizations 0, 64, 128, 192: the 640 levels nearest E = 0, ascending.\n")
        f.write("# Written by tests/golden/make_shard_dense_levels.py (oracle apply_h -> dense -> LAPACK eigvalsh).\n")
        f.write("# rows of three columns: seed, E_min, E_max; rows of two: seed, level\n")
        for seed, lv, emin, emax in rows:
            f.write(f"{seed} {emin:.17g} {emax:.17g}\n")
            for v in lv:
                f.write(f"{seed} {v:.17g}\n")


if __name__ == "__main__":
    main()
