"""Lanczos on the exp-semicircle-filtered operator (Appendix D), plain float64 (oracle).

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module; it shares no code with the CUDA path.

Appendix D weighs DACP against the simpler route of combining the
exp-semicircle filter with the Lanczos method: the filter A = T_K(F),
F = (H^2 - E_c)/E_0 (Sec. II A, Eqs. F, chevo, filter), maps the central
levels of H to the largest eigenvalues of A, and a Krylov method then finds
them. Each Lanczos step applies the filter once (2K H.v), at least 2R steps are
needed for R levels, and every new vector is reorthogonalised against all the
previous ones (the D R^2 cost the appendix names). Steps, in that order:

  1. v_0 = psi / |psi|;
  2. for j = 0 .. m-2: w = A v_j (the filter of exp_semicircle_filter, then
     normalised: the Krylov space does not depend on the scale), full
     reorthogonalisation against v_0 .. v_j (classical Gram-Schmidt, twice),
     v_{j+1} = w / |w|; a breakdown (|w| below 1e-8 of |A v_j|) ends the space;
  3. Rayleigh-Ritz of H in the space: H_m = V^T H V, its eigenpairs
     (theta_i, z_i), and the residual norms |H V z_i - theta_i V z_i|;
  4. of the converged Ritz values (residual at most res_tol E_max), the n_eigs
     of smallest |E| inside [-a, a], ascending (the selection of
     oracle.dacp.select_central).

Readings (the appendix gives no algorithm, only the combination and its cost):
the breakdown threshold 1e-8 sits above the filter's own rounding (a start
vector inside an invariant subspace left residuals of 6.5e-11 after 2K = 60
float64 H.v) and below any direction the space needs. Unconverged Ritz values
of a Krylov space fall anywhere, central window included, so only converged
ones are kept (the residual test Sec. II C applies to DACP's levels, res_tol
1e-8 by default: a converged level's error is of order res^2 / gap). The Ritz values come
from H itself in the Krylov space of A, not from the
tridiagonal of A, because T_K(F(E)) is even in E and many-to-one outside the
window, so the eigenvalues of A cannot be mapped back to E. A consequence the
pins below fix: the space holds, for levels E and -E, only the combination the
start vector gives them, so exactly symmetric pairs (+-E) are not resolved.
"""

from __future__ import annotations

import numpy as np

from .dacp import exp_semicircle_filter, select_central
from .hamiltonian import apply_h, diagonal


def krylov_filtered(model, psi, emax: float, a: float, K: int, m: int, diag=None):
    """Orthonormal basis (D x m', m' <= m) of the Krylov space of T_K(F) from psi."""
    if diag is None:
        diag = diagonal(model)
    v = np.asarray(psi, dtype=np.float64).ravel()
    V = [v / np.linalg.norm(v)]
    for _ in range(m - 1):
        w = exp_semicircle_filter(model, V[-1], emax, a, K, diag=diag)[:, 0]    # A v_j / |A v_j|
        Q = np.stack(V, axis=1)
        for _ in range(2):
            w = w - Q @ (Q.T @ w)
        nrm = np.linalg.norm(w)
        if nrm < 1e-8:
            break
        V.append(w / nrm)
    return np.stack(V, axis=1)


def ritz_pairs(model, V, diag=None):
    """Eigenvalues theta (ascending) of V^T H V and the residual norms |H y - theta y| of their
    Ritz vectors y = V z."""
    HV = apply_h(model, V, diag)
    Hm = V.T @ HV
    th, Z = np.linalg.eigh(0.5 * (Hm + Hm.T))
    R = HV @ Z - (V @ Z) * th
    return th, np.linalg.norm(R, axis=0)


def lanczos_filtered(model, psi, emax: float, a: float, K: int, m: int, n_eigs: int, res_tol: float = 1e-8,
                     diag=None):
    """The n_eigs converged Ritz values of smallest |E| inside [-a, a] from an m-dimensional Krylov
    space of the filtered operator, and the dimension reached."""
    if diag is None:
        diag = diagonal(model)
    V = krylov_filtered(model, psi, emax, a, K, m, diag)
    th, res = ritz_pairs(model, V, diag)
    return select_central(th[res <= res_tol * emax], n_eigs, a), V.shape[1]
