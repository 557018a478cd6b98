"""Closed-form spectrum of the open transverse-field Ising chain with h_z = 0 (oracle).

H = sum_{i=0}^{N-2} J_i Z_i Z_{i+1} + sum_i Gamma_i X_i is exactly solvable
(Sec. III: the paper's Ising model "is exactly solvable by Jordan-Wigner
transformation", used for the exact eigenvalues of Fig. 2a).

Pairing the Majorana operators of each site, H becomes a free-fermion
quadratic form whose single-particle energies are 2*sigma_k, with sigma_k the
singular values of the N x N upper-bidiagonal matrix M (M_ii = Gamma_i,
M_{i,i+1} = J_i). Every many-body level is therefore sum_k s_k sigma_k with
s in {+1, -1}^N: 2^N levels, enumerated exactly here. The formula is pinned
against dense diagonalisation for N <= 10 in the tests (N=1: +-|Gamma|;
N=2, J = Gamma = 1: {+-sqrt5, +-1}).
"""

from __future__ import annotations

import numpy as np


def chain_couplings(model):
    """(J_i, Gamma_i) of an open chain model; raises if it is not one with h = 0."""
    N = model["N"]
    J = model["J"]
    off = J.copy()
    for i in range(N - 1):
        off[i, i + 1] = 0.0
    if np.any(off != 0.0) or np.any(model["h"] != 0.0):
        raise ValueError("not an open zz chain with h_z = 0")
    return np.array([J[i, i + 1] for i in range(N - 1)]), model["gamma"].copy()


def single_particle(model) -> np.ndarray:
    """sigma_k: singular values of the bidiagonal coupling matrix."""
    Jc, G = chain_couplings(model)
    N = model["N"]
    M = np.diag(G)
    for i in range(N - 1):
        M[i, i + 1] = Jc[i]
    return np.linalg.svd(M, compute_uv=False)


def spectrum(model) -> np.ndarray:
    """All 2^N eigenvalues, sorted ascending (N <= 26)."""
    sig = single_particle(model)
    levels = np.zeros(1)
    for s in sig:
        levels = np.concatenate([levels + s, levels - s])
    return np.sort(levels)


def hopping_chain_spectrum(t, hz) -> np.ndarray:
    """All 2^N levels of the open XX chain in a z-field (free fermions).

    H = sum_i t_i (X_i X_{i+1} + Y_i Y_{i+1}) + sum_i hz_i Z_i. With
    sigma^+- = (X +- iY)/2, t (XX + YY) = 2t (sigma^+_i sigma^-_{i+1} + h.c.),
    and the Jordan-Wigner map turns it into nearest-neighbour hopping of
    amplitude 2 t_i (the string cancels between neighbours; the sign of a
    hopping on an open chain is a gauge choice). With n_i = (1 - Z_i)/2,
    hz_i Z_i = hz_i - 2 hz_i n_i. So H = sum_i hz_i + c^T A c with A the
    tridiagonal matrix (A_ii = -2 hz_i, A_{i,i+1} = 2 t_i), and every level is
    sum_i hz_i + the sum of a subset of A's eigenvalues.
    """
    t = np.asarray(t, dtype=np.float64)
    hz = np.asarray(hz, dtype=np.float64)
    N = len(hz)
    A = np.diag(-2.0 * hz)
    for i in range(N - 1):
        A[i, i + 1] = A[i + 1, i] = 2.0 * t[i]
    eps = np.linalg.eigvalsh(A)
    levels = np.zeros(1)
    for e in eps:
        levels = np.concatenate([levels, levels + e])
    return np.sort(levels + hz.sum())
