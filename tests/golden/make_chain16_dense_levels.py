"""Write the exact central levels of the N = 16 mixed-field Ising chain to a text fixture.

The chain is workloads.chain(16): J = 1, h_x = 0.9045, h_z = 0.8090, open, of
dimension 65536. A dense float64 matrix of that size (34 GB) is more than dense
eigh can take here. The chain is its own mirror image, though, so the oracle
splits H into its even and odd reflection sectors
(oracle.hamiltonian.reflection_sector_matrices: 32896 and 32640 states, formed
with the matrix-free apply). LAPACK eigvalsh then diagonalises each block. The
fixture keeps the 1100 levels nearest E = 0 of the union: the 1000 central
levels of that workload plus context for local spacings. The script calls
nothing but oracle/ and numpy; it needs about 30 GB of memory and tens of
minutes on eight cores.

  python tests/golden/make_chain16_dense_levels.py
  python tests/golden/make_chain16_dense_levels.py --integrable-check   # the sector split vs Jordan-Wigner

The check printed: max |sector levels - Jordan-Wigner| = 1.148e-12 over all 65536 levels.
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import hamiltonian as Hm  # noqa: E402

KEEP = 1100
OUT = os.path.join(HERE, "chain16_dense_central_levels.txt")


def main():
    m = W.chain(16)
    t0 = time.time()
    He, Ho = Hm.reflection_sector_matrices(m)
    print(f"sector blocks {He.shape[0]} + {Ho.shape[0]} formed in {time.time() - t0:.0f}s", flush=True)
    ev = []
    for Hs in (He, Ho):
        t0 = time.time()
        ev.append(np.linalg.eigvalsh(Hs))
        print(f"eigvalsh of {Hs.shape[0]} in {time.time() - t0:.0f}s", flush=True)
    del He, Ho
    ev = np.sort(np.concatenate(ev))
    idx = np.sort(np.argsort(np.abs(ev), kind="stable")[:KEEP])
    with open(OUT, "w") as f:
        f.write("# Exact central levels of the N = 16 mixed-field Ising chain (workloads.chain(16): J = 1,\n")
        f.write("# h_x = 0.9045, h_z = 0.8090, open): the 1100 levels nearest E = 0, ascending. Written by\n")
        f.write("# tests/golden/make_chain16_dense_levels.py (oracle reflection-sector blocks -> LAPACK eigvalsh).\n")
        f.write("# first row: E_min, E_max; then one level per row\n")
        f.write(f"{ev[0]:.17g} {ev[-1]:.17g}\n")
        for v in ev[idx]:
            f.write(f"{v:.17g}\n")
    print("wrote", OUT, flush=True)


def integrable_check():
    """The same sector split on the integrable chain (h_z = 0, h_x = 1): the
    central levels against the Jordan-Wigner closed form, at full size."""
    from oracle import jordan_wigner as JW
    m = W.chain(16, J=1.0, hx=1.0, hz=0.0)
    He, Ho = Hm.reflection_sector_matrices(m)
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(He), np.linalg.eigvalsh(Ho)]))
    del He, Ho
    ex = JW.spectrum(m)
    print(f"integrable N = 16: max |sector levels - Jordan-Wigner| = {np.abs(ev - ex).max():.3e} "
          f"over all {len(ev)} levels", flush=True)


if __name__ == "__main__":
    if "--integrable-check" in sys.argv:
        integrable_check()
    else:
        main()
