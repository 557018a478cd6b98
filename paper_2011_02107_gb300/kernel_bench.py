"""Kernel-level benchmark of the recurrences on a synthetic batch.

Runs a fixed number of filter and evolution orders (explicit parameters, no
heuristic) on a batch of spin-glass shards and prints the per-order times
from the library's CUDA events and the algorithmic bandwidth. Used for tile /
launch-mode studies and as a short, fixed-length command for profiler captures.

  python -m paper_2011_02107_gb300.kernel_bench [--N 14] [--R 256] [--b 4]
      [--precision fp32] [--orders 200] [--mode -1] [--tile 0] [--sectors]
--sectors: the 2 R parity sectors (N - 1 spins each, with the global flip) of the R shards.
mode 0: graph replay of per-order launches, 1: persistent launch, 2: graph
replay with staged tiles (float32); mode -1 / tile 0: let dacp_autotune choose.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_2011_02107_gb300 as P  # noqa: E402
import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=14)
    ap.add_argument("--R", type=int, default=256)
    ap.add_argument("--b", type=int, default=4)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "df32"])
    ap.add_argument("--orders", type=int, default=200)
    ap.add_argument("--mode", type=int, default=-1)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--sectors", action="store_true")
    args = ap.parse_args()
    prec = {"fp32": P.DACP_FP32, "df32": P.DACP_DF32}.get(args.precision, P.DACP_FP64)
    esz = 4 if prec == P.DACP_FP32 else 8
    models = [W.spin_glass_shard(args.N, seed=r) for r in range(args.R)]
    if args.sectors:
        psis = [p for r in range(args.R) for p in W.sector_start_vectors(args.N, args.b, seed=0, r=r)]
        d = P.Dacp.parity_sectors(models, psis, block_b=args.b, precision=prec)
    else:
        psis = [W.start_vectors(args.N, args.b, seed=0, r=r) for r in range(args.R)]
        d = P.Dacp(models, psis, block_b=args.b, precision=prec)
    try:
        # a Pauli-norm bound per realization: a sector's fields and flip are the full model's
        # couplings to spin N - 1 and its x-field, so the full model's bound serves both
        emax = np.array([sum(abs(m["J"][np.triu_indices(args.N, 1)])) + sum(m["gamma"]) for m in models])
        emax = np.repeat(emax, d.R // args.R)
        a = 0.015 * emax
        # choose n so that k_n + 1 ~ orders (k_n = floor(n pi / a_r))
        n = max(1, int(math.floor((args.orders - 1) * 0.015 / math.pi)))
        d.set_params(emax, a, args.orders, n)
        if args.mode < 0 or args.tile <= 0:
            d.autotune(64)
        else:
            d.set_launch(args.mode, args.tile)
        mode, tile = d.launch()
        d.filter()
        d.basis_moments()
        ms = d.timings()
        p = d.params()
        vec = sum(1 << nr for nr in d.N) * args.b * esz
        evo_orders = int(p["kn"].max()) + 2          # mu up to 2 k_n + 3
        out = {"N": args.N, "R": args.R, "sectors": bool(args.sectors), "b": args.b, "precision": args.precision, "mode": mode, "tile_bytes": tile,
               "filter_orders": args.orders, "evolution_orders": evo_orders,
               "filter_us_per_order": 1e3 * ms[0] / args.orders, "evolution_us_per_order": 1e3 * ms[1] / evo_orders,
               "evolution_algorithmic_GBps": 3 * vec * evo_orders / (ms[1] / 1e3) / 1e9,
               "filter_algorithmic_GBps": 6 * vec * args.orders / (ms[0] / 1e3) / 1e9,
               "launches": d.launch_count()}
        print(json.dumps(out), flush=True)
    finally:
        d.close()


if __name__ == "__main__":
    main()
