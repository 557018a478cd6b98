"""Python binding of the DACP C ABI (include/dacp.h), argument marshalling only.

DACP -- dual application of Chebyshev polynomial (arXiv 2011.02107) -- finds
thousands of central eigenvalues of spin-1/2 Hamiltonians
H = sum J_ij Z_i Z_j + sum h_i Z_i + sum Gamma_i X_i. Every step runs in the
CUDA library libdacp.so built in-tree by ``paper_2011_02107_gb300.build``;
importing this module fails loudly when that library is missing. There is no
CPU fallback.

The module-level functions carry the C names (``dacp_create``,
``dacp_filter``, ...); ``Dacp`` bundles them around one handle.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdacp.so")

DACP_FP64 = 0
DACP_FP32 = 1
DACP_DF32 = 2

_STATUS = {0: "DACP_OK", 1: "DACP_ERR_ARG", 2: "DACP_ERR_CUDA", 3: "DACP_ERR_NOMEM", 4: "DACP_ERR_NUMERIC",
           5: "DACP_ERR_TIMEOUT", 6: "DACP_ERR_STATE", 7: "DACP_ERR_NOT_CONVERGED", 8: "DACP_ERR_LIBRARY"}

EXPORTS = ["dacp_create", "dacp_set_params", "dacp_choose_params", "dacp_get_params", "dacp_filter",
           "dacp_basis_moments", "dacp_central_eigs", "dacp_get_moments", "dacp_get_filtered", "dacp_residuals", "dacp_solve", "dacp_eigenvectors",
           "dacp_apply_h", "dacp_get_timings", "dacp_get_launch_count", "dacp_last_error", "dacp_status_string",
           "dacp_destroy", "dacp_mlp_create", "dacp_mlp_set_normalization", "dacp_mlp_set_output_range", "dacp_mlp_get_weights",
           "dacp_mlp_set_weights", "dacp_mlp_forward", "dacp_mlp_gradients", "dacp_mlp_train",
           "dacp_mlp_get_launch_count", "dacp_mlp_last_error", "dacp_mlp_destroy", "dacp_choose_params_mlp",
           "dacp_get_features", "dacp_autotune", "dacp_set_launch", "dacp_get_launch",
           "dacp_test_poison_barrier", "dacp_moments_noalloc", "dacp_set_solver", "dacp_set_pair_couplings",
           "dacp_set_emax_rule", "dacp_test_emax_rule", "dacp_solve_learned",
           "dacp_lanczos_filtered", "dacp_set_global_flips", "dacp_create_parity_sectors",
           "dacp_merge_sectors", "dacp_test_fail_alloc", "dacp_solve_sectors"]

N_FEATURES = 40
N_KNOBS = 3


class DacpError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libdacp.so not found at {LIB_PATH}: build it first with "
            "`python -c \"import __graft_entry__ as g; g.build()\"` (the CUDA library is required; "
            "there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    L = ctypes.c_int64
    sig = {
        "dacp_create": [ctypes.POINTER(P), I, P, P, P, P, I, I, P, P],
        "dacp_set_params": [P, P, P, P, P],
        "dacp_choose_params": [P, I, D, D, D, I, I],
        "dacp_get_params": [P, P, P, P, P, P],
        "dacp_filter": [P],
        "dacp_basis_moments": [P],
        "dacp_central_eigs": [P, I, D, D, P, P, P],
        "dacp_get_moments": [P, I, P, L, ctypes.POINTER(L)],
        "dacp_get_filtered": [P, I, P, L],
        "dacp_residuals": [P, I, I, D, D, P, P, P],
        "dacp_solve": [P, I, D, D, P, P, P],
        "dacp_solve_learned": [P, P, I, D, D, P, P, P, P],
        "dacp_solve_sectors": [P, P, I, I, P, P, P],
        "dacp_lanczos_filtered": [P, I, I, I, D, P, P, P, P, ctypes.POINTER(L)],
        "dacp_set_global_flips": [P, P],
        "dacp_create_parity_sectors": [ctypes.POINTER(P), I, P, P, P, P, I, I, P, P],
        "dacp_merge_sectors": [I, I, P, P, I, P, P],
        "dacp_eigenvectors": [P, I, I, D, D, P, P, L, P],
        "dacp_apply_h": [P, I, P, P],
        "dacp_set_pair_couplings": [P, P, P],
        "dacp_set_emax_rule": [P, I],
        "dacp_test_emax_rule": [I, P, P, I, ctypes.POINTER(D)],
        "dacp_get_timings": [P, P],
        "dacp_get_launch_count": [P, ctypes.POINTER(L)],
        "dacp_mlp_create": [ctypes.POINTER(P), I, I, I, I, P, ctypes.c_uint64, P],
        "dacp_mlp_set_normalization": [P, P, P, P, P],
        "dacp_mlp_set_output_range": [P, P, P],
        "dacp_mlp_get_weights": [P, P, L, ctypes.POINTER(L)],
        "dacp_mlp_set_weights": [P, P, L],
        "dacp_mlp_forward": [P, P, I, P],
        "dacp_mlp_gradients": [P, P, P, I, P, ctypes.POINTER(D)],
        "dacp_mlp_train": [P, P, P, I, I, I, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(D)],
        "dacp_mlp_get_launch_count": [P, ctypes.POINTER(L)],
        "dacp_choose_params_mlp": [P, P, I, I, I],
        "dacp_get_features": [P, P, L],
        "dacp_autotune": [P, I, ctypes.POINTER(I)],
        "dacp_set_launch": [P, I, I],
        "dacp_test_poison_barrier": [P],
        "dacp_test_fail_alloc": [L],
        "dacp_set_solver": [P, I],
        "dacp_moments_noalloc": [I, P, P, P, D, P, I, P, P],
        "dacp_get_launch": [P, ctypes.POINTER(I), ctypes.POINTER(I)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.dacp_last_error.argtypes = [P]
    lib.dacp_last_error.restype = ctypes.c_char_p
    lib.dacp_status_string.argtypes = [I]
    lib.dacp_status_string.restype = ctypes.c_char_p
    lib.dacp_destroy.argtypes = [P]
    lib.dacp_destroy.restype = None
    lib.dacp_mlp_last_error.argtypes = [P]
    lib.dacp_mlp_last_error.restype = ctypes.c_char_p
    lib.dacp_mlp_destroy.argtypes = [P]
    lib.dacp_mlp_destroy.restype = None
    return lib


_lib = _load()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(h, status):
    if status != 0:
        msg = _lib.dacp_last_error(h).decode() if h else ""
        raise DacpError(status, msg)


# ---- C-named functions -----------------------------------------------------

def dacp_create(n_spins, J, h, gamma, block_b, precision, psi0, stream=None):
    n_spins = np.ascontiguousarray(n_spins, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    psi0 = np.ascontiguousarray(psi0, dtype=np.float64)
    out = ctypes.c_void_p()
    st = _lib.dacp_create(ctypes.byref(out), len(n_spins), _ptr(n_spins), _ptr(J), _ptr(h), _ptr(gamma),
                          int(block_b), int(precision), _ptr(psi0),
                          ctypes.c_void_p(stream) if stream else None)
    _check(None, st)
    return out.value


def dacp_set_params(hd, emax, a, K, n):
    emax = np.ascontiguousarray(emax, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.int32)
    n = np.ascontiguousarray(n, dtype=np.int32)
    _check(hd, _lib.dacp_set_params(hd, _ptr(emax), _ptr(a), _ptr(K), _ptr(n)))


def dacp_choose_params(hd, n_eigs, d_ratio=2.0, basis_ratio=1.5, c_order=0.0, lanczos_steps=20,
                       kpm_moments=256):
    _check(hd, _lib.dacp_choose_params(hd, int(n_eigs), float(d_ratio), float(basis_ratio), float(c_order),
                                       int(lanczos_steps), int(kpm_moments)))


def dacp_get_params(hd, R):
    emax = np.zeros(R)
    a = np.zeros(R)
    K = np.zeros(R, dtype=np.int32)
    n = np.zeros(R, dtype=np.int32)
    kn = np.zeros(R, dtype=np.int32)
    _check(hd, _lib.dacp_get_params(hd, _ptr(emax), _ptr(a), _ptr(K), _ptr(n), _ptr(kn)))
    return {"emax": emax, "a": a, "K": K, "n": n, "kn": kn}


def dacp_filter(hd):
    _check(hd, _lib.dacp_filter(hd))


def dacp_basis_moments(hd):
    _check(hd, _lib.dacp_basis_moments(hd))


def dacp_central_eigs(hd, R, n_eigs, window=0.0, eps=0.0):
    eigs = np.zeros(R * n_eigs)
    nf = np.zeros(R, dtype=np.int32)
    rank = np.zeros(R, dtype=np.int32)
    _check(hd, _lib.dacp_central_eigs(hd, int(n_eigs), float(window), float(eps), _ptr(eigs), _ptr(nf),
                                      _ptr(rank)))
    return eigs.reshape(R, n_eigs), nf, rank


def dacp_solve(hd, R, n_eigs, window=0.0, eps=0.0):
    eigs = np.zeros(R * n_eigs)
    nf = np.zeros(R, dtype=np.int32)
    rank = np.zeros(R, dtype=np.int32)
    _check(hd, _lib.dacp_solve(hd, int(n_eigs), float(window), float(eps), _ptr(eigs), _ptr(nf), _ptr(rank)))
    return eigs.reshape(R, n_eigs), nf, rank


def dacp_solve_learned(hd, m, R, n_eigs, window=0.0, eps=0.0):
    """Network parameters, overlapped solve, heuristic re-run of short realizations (all in the
    library). Returns (eigs [R, n_eigs], n_found, rank, n_fallback)."""
    eigs = np.zeros(R * n_eigs)
    nf = np.zeros(R, dtype=np.int32)
    rank = np.zeros(R, dtype=np.int32)
    nfb = ctypes.c_int(0)
    _check(hd, _lib.dacp_solve_learned(hd, m, int(n_eigs), float(window), float(eps), _ptr(eigs), _ptr(nf),
                                       _ptr(rank), ctypes.byref(nfb)))
    return eigs.reshape(R, n_eigs), nf, rank, nfb.value


def dacp_solve_sectors(hd, m, n_models, n_eigs, n_sector):
    """Parity-sector handle: solve with n_sector levels per sector (network m or the heuristic),
    merge per model, re-solve the models whose merge came up short (all in the library).
    Returns (eigs [n_models, n_eigs], n_found, n_redone)."""
    eigs = np.zeros(n_models * n_eigs)
    nf = np.zeros(n_models, dtype=np.int32)
    nre = ctypes.c_int(0)
    _check(hd, _lib.dacp_solve_sectors(hd, m, int(n_eigs), int(n_sector), _ptr(eigs), _ptr(nf), ctypes.byref(nre)))
    return eigs.reshape(n_models, n_eigs), nf, nre.value


def dacp_lanczos_filtered(hd, r, steps, n_eigs, res_tol=0.0):
    """The Appendix D comparison method (see include/dacp.h). Returns (eigs, dim, ms[3], hv)."""
    eigs = np.zeros(n_eigs)
    nf = ctypes.c_int(0)
    dim = ctypes.c_int(0)
    ms = np.zeros(3)
    hv = ctypes.c_int64(0)
    _check(hd, _lib.dacp_lanczos_filtered(hd, int(r), int(steps), int(n_eigs), float(res_tol), _ptr(eigs),
                                          ctypes.byref(nf), ctypes.byref(dim), _ptr(ms), ctypes.byref(hv)))
    return eigs[:nf.value].copy(), dim.value, ms, hv.value


def dacp_set_global_flips(hd, coef):
    coef = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
    _check(hd, _lib.dacp_set_global_flips(hd, _ptr(coef) if coef is not None else None))


def dacp_create_parity_sectors(n_spins, J, h, gamma, block_b, precision, psi0, stream=None):
    n_spins = np.ascontiguousarray(n_spins, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    psi0 = np.ascontiguousarray(psi0, dtype=np.float64)
    out = ctypes.c_void_p()
    st = _lib.dacp_create_parity_sectors(ctypes.byref(out), len(n_spins), _ptr(n_spins), _ptr(J), _ptr(h), _ptr(gamma),
                                         int(block_b), int(precision), _ptr(psi0),
                                         ctypes.c_void_p(stream) if stream else None)
    _check(None, st)
    return out.value


def dacp_merge_sectors(eigs_in, n_found_in, n_eigs):
    """eigs_in [2 R, n_in], n_found_in [2 R] -> (eigs [R, n_eigs], n_found [R])."""
    eigs_in = np.ascontiguousarray(eigs_in, dtype=np.float64)
    n_found_in = np.ascontiguousarray(n_found_in, dtype=np.int32)
    R = len(n_found_in) // 2
    eigs = np.zeros(R * n_eigs)
    nf = np.zeros(R, dtype=np.int32)
    _check(None, _lib.dacp_merge_sectors(R, eigs_in.shape[1], _ptr(eigs_in), _ptr(n_found_in), int(n_eigs), _ptr(eigs),
                                         _ptr(nf)))
    return eigs.reshape(R, n_eigs), nf


def merge_sector_levels(eigs, n_found, n_eigs):
    """dacp_merge_sectors over per-realization level lists (as Dacp.run returns them): sector
    lists 2 r, 2 r + 1 -> the n_eigs central levels of model r. Returns (list, n_found)."""
    n_in = max(1, max((len(e) for e in eigs), default=1))
    buf = np.zeros((len(eigs), n_in))
    for i, e in enumerate(eigs):
        buf[i, :len(e)] = e
    out, nf = dacp_merge_sectors(buf, n_found, n_eigs)
    return [out[r, :max(nf[r], 0)].copy() for r in range(len(nf))], nf


def dacp_get_moments(hd, r, cap):
    mu = np.zeros(cap)
    cnt = ctypes.c_int64(0)
    _check(hd, _lib.dacp_get_moments(hd, int(r), _ptr(mu), int(cap), ctypes.byref(cnt)))
    return mu[:cnt.value]


def dacp_get_filtered(hd, r, n):
    out = np.zeros(n)
    _check(hd, _lib.dacp_get_filtered(hd, int(r), _ptr(out), int(n)))
    return out


def dacp_residuals(hd, r, n_eigs, window=0.0, eps=0.0):
    eigs = np.zeros(n_eigs)
    resid = np.zeros(n_eigs)
    nf = ctypes.c_int(0)
    _check(hd, _lib.dacp_residuals(hd, int(r), int(n_eigs), float(window), float(eps), _ptr(eigs), _ptr(resid),
                                   ctypes.byref(nf)))
    n = max(nf.value, 0)
    return eigs[:n], resid[:n], nf.value


def dacp_eigenvectors(hd, r, n_eigs, phi_dev_ptr, ld, window=0.0, eps=0.0):
    """Central levels of r and their Ritz vectors into the device buffer at
    phi_dev_ptr (column-major, leading dimension ld); returns (eigs, n_found)."""
    eigs = np.zeros(n_eigs)
    nf = ctypes.c_int(0)
    _check(hd, _lib.dacp_eigenvectors(hd, int(r), int(n_eigs), float(window), float(eps), _ptr(eigs),
                                      ctypes.c_void_p(phi_dev_ptr), int(ld), ctypes.byref(nf)))
    return eigs[:max(nf.value, 0)], nf.value


def dacp_set_pair_couplings(hd, Jxx, Jyy):
    Jxx = np.ascontiguousarray(Jxx, dtype=np.float64)
    Jyy = np.ascontiguousarray(Jyy, dtype=np.float64)
    _check(hd, _lib.dacp_set_pair_couplings(hd, _ptr(Jxx), _ptr(Jyy)))


def dacp_set_emax_rule(hd, rule):
    _check(hd, _lib.dacp_set_emax_rule(hd, int(rule)))


def dacp_test_emax_rule(alpha, beta2, rule):
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta2 = np.ascontiguousarray(beta2, dtype=np.float64)
    if len(beta2) != len(alpha):
        raise ValueError("beta2 needs one entry per Lanczos step (the last is the squared residual norm)")
    out = ctypes.c_double(0.0)
    _check(None, _lib.dacp_test_emax_rule(len(alpha), _ptr(alpha), _ptr(beta2), int(rule), ctypes.byref(out)))
    return out.value


def dacp_apply_h(hd, r, x_dev_ptr, y_dev_ptr):
    _check(hd, _lib.dacp_apply_h(hd, int(r), ctypes.c_void_p(x_dev_ptr), ctypes.c_void_p(y_dev_ptr)))


def dacp_get_timings(hd):
    ms = np.zeros(3)
    _check(hd, _lib.dacp_get_timings(hd, _ptr(ms)))
    return ms


def dacp_get_launch_count(hd):
    n = ctypes.c_int64(0)
    _check(hd, _lib.dacp_get_launch_count(hd, ctypes.byref(n)))
    return n.value


def dacp_destroy(hd):
    if hd:
        _lib.dacp_destroy(hd)


def dacp_last_error(hd):
    return _lib.dacp_last_error(hd).decode() if hd else ""


def dacp_status_string(s):
    return _lib.dacp_status_string(int(s)).decode()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _mcheck(m, status):
    if status != 0:
        raise DacpError(status, _lib.dacp_mlp_last_error(m).decode() if m else "")


def dacp_mlp_create(n_in, n_hidden, hidden_layers, n_out, weights=None, seed=0, stream=None):
    out = ctypes.c_void_p()
    w = _f32(weights) if weights is not None else None
    st = _lib.dacp_mlp_create(ctypes.byref(out), int(n_in), int(n_hidden), int(hidden_layers), int(n_out),
                              _ptr(w), int(seed), ctypes.c_void_p(stream) if stream else None)
    _mcheck(None, st)
    return out.value


def dacp_mlp_set_normalization(m, in_mean, in_std, out_mean, out_std):
    a, b, c_, d = _f32(in_mean), _f32(in_std), _f32(out_mean), _f32(out_std)
    _mcheck(m, _lib.dacp_mlp_set_normalization(m, _ptr(a), _ptr(b), _ptr(c_), _ptr(d)))


def dacp_mlp_set_output_range(m, lo, hi):
    a, b = _f32(lo), _f32(hi)
    _mcheck(m, _lib.dacp_mlp_set_output_range(m, _ptr(a), _ptr(b)))


def dacp_mlp_get_weights(m):
    cnt = ctypes.c_int64(0)
    _lib.dacp_mlp_get_weights(m, None, 0, ctypes.byref(cnt))
    w = np.zeros(cnt.value, dtype=np.float32)
    _mcheck(m, _lib.dacp_mlp_get_weights(m, _ptr(w), cnt.value, ctypes.byref(cnt)))
    return w


def dacp_mlp_set_weights(m, w):
    w = _f32(w)
    _mcheck(m, _lib.dacp_mlp_set_weights(m, _ptr(w), w.size))


def dacp_mlp_forward(m, x, n_out):
    x = _f32(x)
    y = np.zeros((x.shape[0], n_out), dtype=np.float32)
    _mcheck(m, _lib.dacp_mlp_forward(m, _ptr(x), x.shape[0], _ptr(y)))
    return y


def dacp_mlp_gradients(m, x, t, n_weights):
    x, t = _f32(x), _f32(t)
    g = np.zeros(n_weights, dtype=np.float32)
    loss = ctypes.c_double(0)
    _mcheck(m, _lib.dacp_mlp_gradients(m, _ptr(x), _ptr(t), x.shape[0], _ptr(g), ctypes.byref(loss)))
    return g, loss.value


def dacp_mlp_train(m, x, t, batch=64, epochs=100, lr=1e-3, seed=0):
    x, t = _f32(x), _f32(t)
    loss = ctypes.c_double(0)
    _mcheck(m, _lib.dacp_mlp_train(m, _ptr(x), _ptr(t), x.shape[0], int(batch), int(epochs), float(lr), int(seed),
                                   ctypes.byref(loss)))
    return loss.value


def dacp_mlp_get_launch_count(m):
    n = ctypes.c_int64(0)
    _mcheck(m, _lib.dacp_mlp_get_launch_count(m, ctypes.byref(n)))
    return n.value


def dacp_mlp_last_error(m):
    return _lib.dacp_mlp_last_error(m).decode() if m else ""


def dacp_mlp_destroy(m):
    if m:
        _lib.dacp_mlp_destroy(m)


def dacp_choose_params_mlp(hd, m, n_eigs, lanczos_steps=20, kpm_moments=256):
    _check(hd, _lib.dacp_choose_params_mlp(hd, m, int(n_eigs), int(lanczos_steps), int(kpm_moments)))


def dacp_autotune(hd, orders=64):
    tb = ctypes.c_int(0)
    _check(hd, _lib.dacp_autotune(hd, int(orders), ctypes.byref(tb)))
    return tb.value


def dacp_set_launch(hd, mode, tile_bytes):
    _check(hd, _lib.dacp_set_launch(hd, int(mode), int(tile_bytes)))


def dacp_moments_noalloc(model, emax, psi_dev_ptr, n_orders, mu_dev_ptr, stream=None):
    """Allocation-free moments of one realization (see include/dacp.h); device pointers in and out."""
    N = int(model["N"])
    J = np.ascontiguousarray(model["J"], dtype=np.float64).reshape(N, N)
    h = np.ascontiguousarray(model["h"], dtype=np.float64)
    g = np.ascontiguousarray(model["gamma"], dtype=np.float64)
    st = _lib.dacp_moments_noalloc(N, _ptr(J), _ptr(h), _ptr(g), float(emax), ctypes.c_void_p(psi_dev_ptr),
                                   int(n_orders), ctypes.c_void_p(mu_dev_ptr),
                                   ctypes.c_void_p(stream) if stream else None)
    if st != 0:
        raise DacpError(st, "dacp_moments_noalloc")


def dacp_set_solver(hd, mode):
    _check(hd, _lib.dacp_set_solver(hd, int(mode)))


def dacp_test_poison_barrier(hd):
    _check(hd, _lib.dacp_test_poison_barrier(hd))


def dacp_test_fail_alloc(after):
    _check(None, _lib.dacp_test_fail_alloc(int(after)))


def dacp_get_launch(hd):
    m, t = ctypes.c_int(0), ctypes.c_int(0)
    _check(hd, _lib.dacp_get_launch(hd, ctypes.byref(m), ctypes.byref(t)))
    return m.value, t.value


def dacp_get_features(hd, R):
    f = np.zeros((R, N_FEATURES), dtype=np.float32)
    _check(hd, _lib.dacp_get_features(hd, _ptr(f), f.size))
    return f


# ---- convenience wrapper ---------------------------------------------------

def _pack(models):
    n_spins = np.array([m["N"] for m in models], dtype=np.int32)
    J = np.concatenate([np.asarray(m["J"], dtype=np.float64).ravel() for m in models])
    h = np.concatenate([np.asarray(m["h"], dtype=np.float64) for m in models])
    g = np.concatenate([np.asarray(m["gamma"], dtype=np.float64) for m in models])
    return n_spins, J, h, g


class Dacp:
    """One handle over a batch of realizations (models from ``workloads``)."""

    def __init__(self, models, psi0_list, block_b=4, precision=DACP_FP64, stream=None):
        self.models = list(models)
        self.R = len(self.models)
        self.b = int(block_b)
        self.N = [m["N"] for m in self.models]
        n_spins = np.array(self.N, dtype=np.int32)
        J = np.concatenate([m["J"].ravel() for m in self.models])
        h = np.concatenate([m["h"] for m in self.models])
        g = np.concatenate([m["gamma"] for m in self.models])
        self.psi0_list = [np.ascontiguousarray(p, dtype=np.float64) for p in psi0_list]
        self.precision = precision
        self.stream = stream
        psi0 = np.concatenate([p.ravel() for p in self.psi0_list])
        self.handle = dacp_create(n_spins, J, h, g, block_b, precision, psi0, stream)
        if any("Jxx" in m or "Jyy" in m for m in self.models):
            z = [np.zeros((m["N"], m["N"])) for m in self.models]
            Jxx = np.concatenate([np.asarray(m.get("Jxx", zz), dtype=np.float64).ravel()
                                  for m, zz in zip(self.models, z)])
            Jyy = np.concatenate([np.asarray(m.get("Jyy", zz), dtype=np.float64).ravel()
                                  for m, zz in zip(self.models, z)])
            try:
                dacp_set_pair_couplings(self.handle, Jxx, Jyy)
            except Exception:
                dacp_destroy(self.handle)
                raise
        if any(float(m.get("gflip", 0.0)) != 0.0 for m in self.models):
            try:
                dacp_set_global_flips(self.handle, [float(m.get("gflip", 0.0)) for m in self.models])
            except Exception:
                dacp_destroy(self.handle)
                raise

    @classmethod
    def parity_sectors(cls, models, psi0_sectors, block_b=4, precision=DACP_FP64, stream=None):
        """A handle whose realizations 2r, 2r+1 are the parity sectors +1, -1 of models[r] (no
        z-fields; dacp_create_parity_sectors builds them in the library). psi0_sectors: 2 R start
        blocks of shape (2^(N_r - 1), b), in that order."""
        n_spins, J, h, g = _pack(models)
        psi0 = np.concatenate([np.ascontiguousarray(p, dtype=np.float64).ravel() for p in psi0_sectors])
        self = cls.__new__(cls)
        self.models = list(models)
        self.R = 2 * len(models)
        self.b = int(block_b)
        self.N = [m["N"] - 1 for m in models for _ in range(2)]
        self.precision = precision
        self.stream = stream
        self.psi0_list = [np.ascontiguousarray(p, dtype=np.float64) for p in psi0_sectors]
        self.handle = dacp_create_parity_sectors(n_spins, J, h, g, block_b, precision, psi0, stream)
        return self

    def set_params(self, emax, a, K, n):
        R = self.R
        dacp_set_params(self.handle, np.broadcast_to(emax, R), np.broadcast_to(a, R), np.broadcast_to(K, R),
                        np.broadcast_to(n, R))

    def choose_params(self, n_eigs, **kw):
        dacp_choose_params(self.handle, n_eigs, **kw)

    def choose_params_mlp(self, mlp, n_eigs, **kw):
        dacp_choose_params_mlp(self.handle, mlp, n_eigs, **kw)

    def autotune(self, orders=64):
        return dacp_autotune(self.handle, orders)

    def set_solver(self, mode):
        dacp_set_solver(self.handle, mode)

    def set_emax_rule(self, rule):
        dacp_set_emax_rule(self.handle, rule)

    def set_launch(self, mode, tile_bytes):
        dacp_set_launch(self.handle, mode, tile_bytes)

    def launch(self):
        return dacp_get_launch(self.handle)

    def features(self):
        return dacp_get_features(self.handle, self.R)

    def params(self):
        return dacp_get_params(self.handle, self.R)

    def filter(self):
        dacp_filter(self.handle)

    def basis_moments(self):
        dacp_basis_moments(self.handle)

    def central_eigs(self, n_eigs, window=0.0, eps=0.0):
        eigs, nf, rank = dacp_central_eigs(self.handle, self.R, n_eigs, window, eps)
        return [eigs[r, :max(nf[r], 0)].copy() for r in range(self.R)], nf, rank

    def solve(self, n_eigs, mlp=None, window=0.0, eps=0.0):
        """Whole path for the batch: parameters (network when given, else the
        heuristic), filter, evolution, subspace solve. With a network the
        library re-runs, with the heuristic, every realization whose learned
        parameters return fewer than n_eigs levels (dacp_solve_learned).
        Returns (eigs list, n_found, rank, n_fallback)."""
        if mlp is None:
            self.choose_params(n_eigs)
            eigs, nf, rank = self.run(n_eigs, window, eps)
            return eigs, nf, rank, 0
        e, nf, rank, nfb = dacp_solve_learned(self.handle, mlp, self.R, n_eigs, window, eps)
        return [e[r, :max(nf[r], 0)].copy() for r in range(self.R)], nf, rank, nfb

    def solve_sectors(self, n_eigs, n_sector, mlp=None):
        """Parity-sector handle (Dacp.parity_sectors): the levels of each model, merged from its two
        sectors, with short merges re-solved in the library (dacp_solve_sectors).
        Returns (eigs list per model, n_found, n_redone)."""
        nm = self.R // 2
        e, nf, nre = dacp_solve_sectors(self.handle, mlp, nm, n_eigs, n_sector)
        return [e[m, :max(nf[m], 0)].copy() for m in range(nm)], nf, nre

    def run(self, n_eigs, window=0.0, eps=0.0):
        """Filter, evolution and subspace solves with the solves overlapped (dacp_solve)."""
        eigs, nf, rank = dacp_solve(self.handle, self.R, n_eigs, window, eps)
        return [eigs[r, :max(nf[r], 0)].copy() for r in range(self.R)], nf, rank

    def moments(self, r):
        p = self.params()
        rows = 2 * int(p["kn"][r]) + 2
        mu = dacp_get_moments(self.handle, r, rows * self.b * self.b)
        return mu.reshape(rows, self.b, self.b)

    def residuals(self, r, n_eigs, window=0.0, eps=0.0):
        """Central levels of realization r and their residual norms (Sec. II C)."""
        return dacp_residuals(self.handle, r, n_eigs, window, eps)

    def eigenvectors(self, r, n_eigs, window=0.0, eps=0.0):
        """Central levels of r and their Ritz vectors (torch float64 tensor on the
        device, 2^N x n_found)."""
        import torch
        D = 1 << self.N[r]
        phi = torch.empty((n_eigs, D), dtype=torch.float64, device="cuda")   # column-major D x n_eigs
        torch.cuda.synchronize()                   # the library writes it on its own stream
        eigs, nf = dacp_eigenvectors(self.handle, r, n_eigs, phi.data_ptr(), D, window, eps)
        torch.cuda.synchronize()
        return eigs, phi[:max(nf, 0)].T, nf

    def filtered(self, r):
        n = (1 << self.N[r]) * self.b
        return dacp_get_filtered(self.handle, r, n).reshape(1 << self.N[r], self.b)

    def apply_h(self, r, x_ptr, y_ptr):
        dacp_apply_h(self.handle, r, x_ptr, y_ptr)

    def timings(self):
        return dacp_get_timings(self.handle)

    def launch_count(self):
        return dacp_get_launch_count(self.handle)

    def close(self):
        if self.handle:
            dacp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
