"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no Hamiltonian apply, no Chebyshev recurrence, no moments).

All Hamiltonians are written in the form

    H = sum_{i<j} J_ij Z_i Z_j + sum_i h_i Z_i + sum_i Gamma_i X_i

with Z_i acting on bit i of the basis-state index (z_i(s) = 1 - 2*bit_i(s)).
The paper's two models (Sec. III) use sigma^x sigma^x couplings and sigma^z
fields; a global Hadamard rotation (X <-> Z on every spin) maps them onto this
form without changing the spectrum, so the paper's couplings become the zz
couplings here and its z-fields become the x-fields (``paper_tfim`` and
``paper_spin_glass``).

A model is a dict with keys ``N`` (spins), ``J`` (N x N float64, only i<j
used), ``h`` (N float64) and ``gamma`` (N float64). Models with two-body flip
couplings (``heisenberg_chain``) also carry ``Jxx`` and ``Jyy`` (N x N, i<j
used) for + sum_{i<j} (Jxx_ij X_i X_j + Jyy_ij Y_i Y_j).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "chain",
    "spin_glass_shard",
    "paper_tfim",
    "paper_spin_glass",
    "random_model",
    "heisenberg_chain",
    "start_vectors",
    "pack_models",
]


def _model(N, J, h, gamma):
    return {
        "N": int(N),
        "J": np.ascontiguousarray(J, dtype=np.float64),
        "h": np.ascontiguousarray(h, dtype=np.float64),
        "gamma": np.ascontiguousarray(gamma, dtype=np.float64),
    }


def chain(N: int, J: float = 1.0, hx: float = 0.9045, hz: float = 0.8090):
    """Uniform open mixed-field Ising chain: J sum Z_i Z_{i+1} + hx sum X_i + hz sum Z_i.

    The defaults are the mixed-field chain of the N=10, N=16 and N=20 workloads
    (J=1, h_x=0.9045, h_z=0.8090); hz=0, hx=1 gives the integrable variant.
    """
    Jm = np.zeros((N, N))
    for i in range(N - 1):
        Jm[i, i + 1] = J
    return _model(N, Jm, np.full(N, hz), np.full(N, hx))


def spin_glass_shard(N: int, seed: int, j_scale: float = 1.0,
                     gamma_lo: float = 0.6, gamma_hi: float = 1.4):
    """All-to-all shard: J_ij ~ U[-j_scale, j_scale] (i<j), Gamma_i ~ U[lo, hi], h = 0.

    Draw order from numpy PCG64(seed): the J_ij row-major over i<j, then Gamma.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    Jm = np.zeros((N, N))
    iu = np.triu_indices(N, 1)
    Jm[iu] = rng.uniform(-j_scale, j_scale, size=len(iu[0]))
    gamma = rng.uniform(gamma_lo, gamma_hi, size=N)
    return _model(N, Jm, np.zeros(N), gamma)


def paper_tfim(N: int, seed: int, Jc: float = 10.0, Gamma: float = 1.0):
    """Disordered transverse-field Ising chain of Sec. III, rotated to the zz/x form.

    Paper: (1/4) sum J_{i,i+1} sx sx + (1/2) sum Gamma_i sz with
    J_{i,i+1} ~ U[-Jc/sqrt(N), Jc/sqrt(N)], Gamma_i ~ U[0, Gamma].
    Here: zz coupling J_{i,i+1}/4 and x-field Gamma_i/2, h = 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = Jc / np.sqrt(N)
    Jm = np.zeros((N, N))
    for i in range(N - 1):
        Jm[i, i + 1] = rng.uniform(-w, w) / 4.0
    gamma = rng.uniform(0.0, Gamma, size=N) / 2.0
    return _model(N, Jm, np.zeros(N), gamma)


def paper_spin_glass(N: int, seed: int, Jc: float = 10.0, Gamma: float = 1.0):
    """Spin-glass shards of Sec. III with the Ising parameters, rotated to the zz/x form."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = Jc / np.sqrt(N)
    Jm = np.zeros((N, N))
    iu = np.triu_indices(N, 1)
    Jm[iu] = rng.uniform(-w, w, size=len(iu[0]))
    gamma = rng.uniform(0.0, Gamma, size=N)
    return _model(N, Jm, np.zeros(N), gamma)


def random_model(N: int, seed: int, density: float = 1.0, scale: float = 1.0):
    """Generic disordered model with all three kinds of terms (test input)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Jm = np.zeros((N, N))
    iu = np.triu_indices(N, 1)
    vals = rng.uniform(-scale, scale, size=len(iu[0]))
    keep = rng.uniform(size=len(iu[0])) < density
    Jm[iu] = vals * keep
    h = rng.uniform(-scale, scale, size=N)
    gamma = rng.uniform(0.2 * scale, scale, size=N)
    return _model(N, Jm, h, gamma)


def heisenberg_chain(N: int, seed: int, J: float = 1.0, delta: float = 1.0, W: float = 3.0,
                     gamma: float = 0.0):
    """Open random-field XXZ chain (the standard many-body-localization model):
    J sum (X_i X_{i+1} + Y_i Y_{i+1} + delta Z_i Z_{i+1}) + sum h_i Z_i + gamma sum X_i,
    h_i ~ U[-W, W] from numpy PCG64(seed). delta = 1 is the Heisenberg chain.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.uniform(-W, W, size=N)
    Jz = np.zeros((N, N))
    Jp = np.zeros((N, N))
    for i in range(N - 1):
        Jz[i, i + 1] = J * delta
        Jp[i, i + 1] = J
    m = _model(N, Jz, h, np.full(N, float(gamma)))
    m["Jxx"] = Jp.copy()
    m["Jyy"] = Jp.copy()
    return m


def start_vectors(N: int, b: int, seed: int, r: int = 0) -> np.ndarray:
    """b real Gaussian N(0,1) start vectors of length 2^N, layout [state][column].

    Drawn from numpy PCG64 keyed by (seed, r) so that realization r of a batch
    gets its own stream.
    """
    rng = np.random.Generator(np.random.PCG64([seed, r]))
    return np.ascontiguousarray(rng.standard_normal((1 << N, b)))


def sector_start_vectors(N: int, b: int, seed: int, r: int = 0):
    """Start blocks of the two parity sectors (+1, -1) of an N-spin realization r: two draws of
    start_vectors(N - 1, b, seed, ...) keyed 2 r and 2 r + 1."""
    return [start_vectors(N - 1, b, seed, 2 * r), start_vectors(N - 1, b, seed, 2 * r + 1)]


def pack_models(models):
    """Concatenate a list of models into the flat arrays the C ABI takes.

    Returns (n_spins int32[R], J float64[sum N_r^2], h float64[sum N_r],
    gamma float64[sum N_r]).
    """
    n_spins = np.array([m["N"] for m in models], dtype=np.int32)
    J = np.concatenate([m["J"].ravel() for m in models]).astype(np.float64)
    h = np.concatenate([m["h"] for m in models]).astype(np.float64)
    g = np.concatenate([m["gamma"] for m in models]).astype(np.float64)
    return n_spins, J, h, g
