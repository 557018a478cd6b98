"""Spin-1/2 two-body Hamiltonian, matrix-free and dense (oracle).

H = sum_{i<j} J_ij Z_i Z_j + sum_i h_i Z_i + sum_i Gamma_i X_i on 2^N basis
states s; Z_i acts on bit i with z_i(s) = 1 - 2*bit_i(s) and X_i flips bit i.
Models may also carry two-body flip couplings ``Jxx`` and ``Jyy`` (N x N, i<j
used): + sum_{i<j} (Jxx_ij X_i X_j + Jyy_ij Y_i Y_j). Both flip bits i and j;
with Y|b> = i z(b) |b XOR 1>, the pair Y_i Y_j carries -z_i(s) z_j(s), which is
real, so every such H stays a real symmetric matrix (XXZ and Heisenberg chains,
the paper's native sigma^x sigma^x couplings of Sec. III without rotation).

A model may also carry ``gflip`` (a number c): + c X_0 X_1 ... X_{N-1}, every
spin flipped at once. That is the term a parity sector keeps of the x-field of
the spin it removes (parity_sector_models below).

The paper works in matrix-free mode (Sec. II intro): H is a function taking a
state to a state, each Pauli term "represented by a specific function"
(Sec. III). ``apply_h`` is that function written out term by term.
``dense_h`` builds the same operator independently, as a sum of Kronecker
products of 2x2 Pauli matrices, for N <= 12.
"""

from __future__ import annotations

import numpy as np


def z_signs(N: int) -> np.ndarray:
    """z_i(s) = 1 - 2*bit_i(s) as an (N, 2^N) float64 array."""
    s = np.arange(1 << N)
    return np.stack([1.0 - 2.0 * ((s >> i) & 1) for i in range(N)])


def pair_couplings(model):
    """(Jxx, Jyy) as upper-triangular N x N arrays; zeros when the model has none."""
    N = model["N"]
    z = np.zeros((N, N))
    Jxx = np.triu(np.asarray(model.get("Jxx", z), dtype=np.float64), 1)
    Jyy = np.triu(np.asarray(model.get("Jyy", z), dtype=np.float64), 1)
    return Jxx, Jyy


def diagonal(model) -> np.ndarray:
    """diag(s) = sum_{i<j} J_ij z_i z_j + sum_i h_i z_i for every basis state."""
    N = model["N"]
    z = z_signs(N)
    d = np.zeros(1 << N)
    for i in range(N):
        d += model["h"][i] * z[i]
        for j in range(i + 1, N):
            if model["J"][i, j] != 0.0:
                d += model["J"][i, j] * z[i] * z[j]
    return d


def apply_h(model, x: np.ndarray, diag: np.ndarray | None = None) -> np.ndarray:
    """y = H x. x has shape (2^N,) or (2^N, b); columns are independent vectors."""
    N = model["N"]
    D = 1 << N
    if diag is None:
        diag = diagonal(model)
    s = np.arange(D)
    dd = diag if x.ndim == 1 else diag[:, None]
    y = dd * x
    for i in range(N):
        g = model["gamma"][i]
        if g != 0.0:
            y = y + g * x[s ^ (1 << i)]
    Jxx, Jyy = pair_couplings(model)
    for i in range(N):
        for j in range(i + 1, N):
            if Jxx[i, j] != 0.0 or Jyy[i, j] != 0.0:
                # <s| (Jxx X_i X_j + Jyy Y_i Y_j) |s'> with s' = s XOR (2^i + 2^j)
                zz = (1.0 - 2.0 * ((s >> i) & 1)) * (1.0 - 2.0 * ((s >> j) & 1))
                c = Jxx[i, j] - Jyy[i, j] * zz
                y = y + (c if x.ndim == 1 else c[:, None]) * x[s ^ ((1 << i) | (1 << j))]
    gf = float(model.get("gflip", 0.0))
    if gf != 0.0:
        y = y + gf * x[s ^ (D - 1)]
    return y


def apply_h_rows(model, x: np.ndarray, states, with_abs: bool = False):
    """Rows `states` of y = H x, one row at a time from the definition: y[s] =
    diag(s) x[s] + sum_i Gamma_i x[s XOR 2^i]. Only the listed states' diagonal
    is formed, so this reaches any N the vectors fit in memory (the full
    ``diagonal`` is O(2^N N^2)). With ``with_abs`` also returns sum_k |term_k|
    per row, the scale of the round-off a summation of those terms can make."""
    N = model["N"]
    st = np.asarray(states, dtype=np.int64)
    z = 1.0 - 2.0 * ((st[:, None] >> np.arange(N)[None, :]) & 1)          # z_i(s)
    Ju = np.triu(model["J"], 1)
    d = z @ model["h"] + np.einsum("si,ij,sj->s", z, Ju, z)
    xs = x[st]
    dd = d if x.ndim == 1 else d[:, None]
    y = dd * xs
    a = np.abs(dd * xs)
    for i in range(N):
        g = model["gamma"][i]
        if g != 0.0:
            t = g * x[st ^ (1 << i)]
            y = y + t
            a = a + np.abs(t)
    Jxx, Jyy = pair_couplings(model)
    for i in range(N):
        for j in range(i + 1, N):
            if Jxx[i, j] != 0.0 or Jyy[i, j] != 0.0:
                c = Jxx[i, j] - Jyy[i, j] * z[:, i] * z[:, j]
                t = (c if x.ndim == 1 else c[:, None]) * x[st ^ ((1 << i) | (1 << j))]
                y = y + t
                a = a + np.abs(t)
    gf = float(model.get("gflip", 0.0))
    if gf != 0.0:
        t = gf * x[st ^ ((1 << N) - 1)]
        y = y + t
        a = a + np.abs(t)
    return (y, a) if with_abs else y


_I2 = np.eye(2)
_X = np.array([[0.0, 1.0], [1.0, 0.0]])
_Y = np.array([[0.0, -1.0j], [1.0j, 0.0]])
_Z = np.array([[1.0, 0.0], [0.0, -1.0]])


def _site_op(N: int, ops: dict) -> np.ndarray:
    """Kronecker product with ops[i] on spin i and identity elsewhere.

    Spin i is bit i of the state index, so the factor for spin N-1 is leftmost.
    """
    out = np.ones((1, 1))
    for i in reversed(range(N)):
        out = np.kron(out, ops.get(i, _I2))
    return out


def dense_h(model) -> np.ndarray:
    """Dense 2^N x 2^N matrix of H from Kronecker products (N <= 12)."""
    N = model["N"]
    if N > 12:
        raise ValueError("dense_h is limited to N <= 12")
    D = 1 << N
    H = np.zeros((D, D))
    for i in range(N):
        if model["gamma"][i] != 0.0:
            H += model["gamma"][i] * _site_op(N, {i: _X})
        if model["h"][i] != 0.0:
            H += model["h"][i] * _site_op(N, {i: _Z})
        for j in range(i + 1, N):
            if model["J"][i, j] != 0.0:
                H += model["J"][i, j] * _site_op(N, {i: _Z, j: _Z})
    Jxx, Jyy = pair_couplings(model)
    for i in range(N):
        for j in range(i + 1, N):
            if Jxx[i, j] != 0.0:
                H += Jxx[i, j] * _site_op(N, {i: _X, j: _X})
            if Jyy[i, j] != 0.0:
                yy = _site_op(N, {i: _Y, j: _Y})          # complex Kronecker product
                assert np.abs(yy.imag).max() == 0.0
                H += Jyy[i, j] * yy.real
    gf = float(model.get("gflip", 0.0))
    if gf != 0.0:
        H += gf * _site_op(N, {i: _X for i in range(N)})
    return H


def pauli_norm_bound(model) -> float:
    """sum |J| + sum |h| + sum |Gamma|: a rigorous bound on the spectral radius."""
    N = model["N"]
    iu = np.triu_indices(N, 1)
    Jxx, Jyy = pair_couplings(model)
    return float(np.abs(model["J"][iu]).sum() + np.abs(model["h"]).sum()
                 + np.abs(model["gamma"]).sum() + np.abs(Jxx).sum() + np.abs(Jyy).sum()
                 + abs(float(model.get("gflip", 0.0))))


def trace_h2_per_state(model) -> float:
    """Tr(H^2)/2^N = sum J_ij^2 + sum h_i^2 + sum Gamma_i^2 (Pauli strings are orthonormal)."""
    N = model["N"]
    iu = np.triu_indices(N, 1)
    Jxx, Jyy = pair_couplings(model)
    return float((model["J"][iu] ** 2).sum() + (model["h"] ** 2).sum()
                 + (model["gamma"] ** 2).sum() + (Jxx ** 2).sum() + (Jyy ** 2).sum()
                 + float(model.get("gflip", 0.0)) ** 2)


def bit_reverse(N: int) -> np.ndarray:
    """rev(s): bit i of s moved to bit N-1-i, for every basis state (the mirror image of a chain)."""
    s = np.arange(1 << N)
    rev = np.zeros_like(s)
    for i in range(N):
        rev |= ((s >> i) & 1) << (N - 1 - i)
    return rev


def reflection_sector_matrices(model, chunk: int = 1024):
    """H restricted to the even and odd sectors of the reflection i -> N-1-i.

    For a model that is its own mirror image, H commutes with the permutation
    s -> rev(s), so H is block diagonal in the basis e_s (s = rev(s)) and
    (e_s + e_rev(s))/sqrt2 (even), (e_s - e_rev(s))/sqrt2 (odd). Each block is
    formed column by column with the matrix-free apply: two dense matrices of
    dimension (2^N +- 2^ceil(N/2))/2 whose spectra together are H's. This
    halves the size dense eigh has to handle (N = 16: two 32.9k blocks instead
    of one 65.5k matrix).
    """
    N = model["N"]
    Jxx, Jyy = pair_couplings(model)
    mirror = np.arange(N)[::-1]
    for name, M in (("J", np.triu(model["J"], 1)), ("Jxx", Jxx), ("Jyy", Jyy)):
        Ms = M + M.T
        if np.abs(Ms[np.ix_(mirror, mirror)] - Ms).max() > 0.0:
            raise ValueError(f"{name} is not mirror symmetric")
    for name in ("h", "gamma"):
        if np.abs(model[name][mirror] - model[name]).max() > 0.0:
            raise ValueError(f"{name} is not mirror symmetric")
    D = 1 << N
    s = np.arange(D)
    rev = bit_reverse(N)
    fixed = s[rev == s]
    lo = s[s < rev]                     # one state of each mirror pair
    diag = diagonal(model)
    out = []
    for sign in (1.0, -1.0):
        # sector basis: (state a, state b, weight): e_a for fixed states, (e_a + sign e_b)/sqrt2 for pairs
        a = np.concatenate([fixed, lo]) if sign > 0 else lo
        b = np.concatenate([fixed, rev[lo]]) if sign > 0 else rev[lo]
        w = np.concatenate([np.ones(len(fixed)), np.full(len(lo), 2 ** -0.5)]) if sign > 0 else np.full(len(lo), 2 ** -0.5)
        nf = len(fixed) if sign > 0 else 0
        d = len(a)
        Hs = np.empty((d, d))
        for c0 in range(0, d, chunk):
            c1 = min(d, c0 + chunk)
            cols = np.arange(c0, c1)
            V = np.zeros((D, c1 - c0))
            V[a[cols], cols - c0] = w[cols]
            pair = cols >= nf
            V[b[cols[pair]], cols[pair] - c0] += sign * w[cols[pair]]
            Wc = apply_h(model, V, diag)
            # project back: row k = <basis_k| H |col>
            Hs[:, c0:c1] = w[:, None] * Wc[a]
            Hs[nf:, c0:c1] += sign * w[nf:, None] * Wc[b[nf:]]
        out.append(Hs)
    return out[0], out[1]


def parity_sector_models(model):
    """The two parity sectors of a model without z-fields, as (N-1)-spin models (sigma = +1, -1).

    With h = 0 (and no pair terms) every term of H commutes with P = X_0 ... X_{N-1}: Z_i Z_j
    because P flips both signs, X_i trivially. Take as basis of sector sigma the states
    (e_s + sigma e_{s XOR (2^N - 1)}) / sqrt 2 with bit N-1 of s clear, labelled by s's lower
    N-1 bits. On them z_{N-1} = +1, so Z_i Z_{N-1} acts as Z_i; X_i (i < N-1) maps label s to
    s XOR 2^i; X_{N-1} maps e_s to e_{s XOR 2^(N-1)} = the partner of label s XOR (2^(N-1) - 1),
    i.e. sigma times that basis state. Hence sector sigma is: J_ij for i < j < N-1, z-fields
    h_i = J_{i,N-1}, x-fields Gamma_i (i < N-1) and gflip = sigma Gamma_{N-1}.
    """
    N = model["N"]
    if N < 2:
        raise ValueError("a parity sector needs N >= 2")
    if np.any(np.asarray(model["h"]) != 0.0):
        raise ValueError("z-fields break the parity symmetry")
    Jxx, Jyy = pair_couplings(model)
    if np.any(Jxx != 0.0) or np.any(Jyy != 0.0) or float(model.get("gflip", 0.0)) != 0.0:
        raise ValueError("only zz couplings and x-fields")
    J = np.triu(np.asarray(model["J"], dtype=np.float64), 1)
    out = []
    for sigma in (1.0, -1.0):
        out.append({"N": N - 1, "J": J[:N - 1, :N - 1].copy(), "h": J[:N - 1, N - 1].copy(),
                    "gamma": np.asarray(model["gamma"], dtype=np.float64)[:N - 1].copy(),
                    "gflip": sigma * float(model["gamma"][N - 1])})
    return out
