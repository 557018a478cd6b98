"""DACP against the exp-semicircle filter + Lanczos method (Appendix D), on the same GPU kernels.

Appendix D argues that combining the exp-semicircle filter with the Lanczos
method costs at least 2R filter runs of 36 E_max / a H.v each for R central
levels (72 R E_max / a H.v in all), plus the reorthogonalisation of every new
vector against all earlier ones, while DACP's evolution takes about
pi R E_max / a H.v. This script runs both on the same realization and
parameters (E_max, a, K from the Sec. III heuristic) and reports, per method,
the time, the H.v applied, the levels returned and, for the levels both
return, their largest difference; DACP's own residual norms (Sec. II C) bound
its levels' errors. The Lanczos variant is given m = steps_ratio * R Krylov
directions (the appendix's minimum is 2R) and one start vector (column 0 of
DACP's block).

  python -m paper_2011_02107_gb300.compare_lanczos [--model chain|shard] [--N 12] [--n-eigs 100]
      [--steps-ratio 2.0] [--b 4]
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_2011_02107_gb300 as P  # noqa: E402
import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="chain", choices=["chain", "shard"])
    ap.add_argument("--N", type=int, default=12)
    ap.add_argument("--n-eigs", type=int, default=100)
    ap.add_argument("--steps-ratio", type=float, default=2.0)
    ap.add_argument("--b", type=int, default=4)
    args = ap.parse_args()
    m = W.chain(args.N) if args.model == "chain" else W.spin_glass_shard(args.N, seed=0)
    psi = W.start_vectors(args.N, args.b, seed=0)
    R = args.n_eigs
    d = P.Dacp([m], [psi], block_b=args.b, precision=P.DACP_FP64)
    try:
        d.choose_params(R)
        p = d.params()
        t0 = time.perf_counter()
        eigs, nf, rank = d.run(R)
        t_dacp = time.perf_counter() - t0
        ph = d.timings()
        lev, resid, nfr = d.residuals(0, R)
        kn, K = int(p["kn"][0]), int(p["K"][0])
        hv_dacp = 2 * args.b * K + args.b * (kn + 2)          # filter (2 H.v per order) + evolution, per column
        steps = max(1, int(round(args.steps_ratio * R)))
        t1 = time.perf_counter()
        lz, dim, ms, hv_lz = P.dacp_lanczos_filtered(d.handle, 0, steps, R)
        t_lz = time.perf_counter() - t1
    finally:
        d.close()
    got = np.asarray(eigs[0])
    both = [x for x in lz if len(got) and np.min(np.abs(got - x)) < 1e-6 * float(p["emax"][0])]
    diff = max((float(np.min(np.abs(got - x))) for x in both), default=None)
    out = {
        "model": args.model, "N": args.N, "n_eigs": R, "emax": float(p["emax"][0]), "a": float(p["a"][0]), "K": K,
        "dacp": {"b": args.b, "seconds": t_dacp, "phase_ms": {"T_F": ph[0], "T_E": ph[1], "T_D": ph[2]},
                 "h_v": hv_dacp, "levels": int(nf[0]), "basis": int(args.b * (2 * int(p["n"][0]) + 1)),
                 "max_residual_over_emax": float(np.max(resid) / p["emax"][0]) if nfr > 0 else None},
        "lanczos_filter": {"steps": steps, "dimension": dim, "seconds": t_lz,
                           "phase_ms": {"filter": ms[0], "reorthogonalisation": ms[1], "rayleigh_ritz": ms[2]},
                           "h_v": hv_lz, "converged_levels": len(lz)},
        "common_levels": len(both), "max_difference_common": diff,
        "h_v_ratio": hv_lz / hv_dacp, "time_ratio": t_lz / t_dacp,
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
