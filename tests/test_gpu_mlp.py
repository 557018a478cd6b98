"""GPU parity of the parameter network (float32 kernels) against the float64 MLP oracle.

Tolerances: forward 1e-5 and gradients 1e-4 of the largest value (float32
GEMMs over <= 256-term sums); one full-batch Adam step 1e-5 of lr.
"""

import numpy as np
import pytest

import workloads as W
from oracle import mlp as OM
from oracle import params as OP

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")

SIZES = [40, 64, 64, 64, 3]


def _net(seed=3):
    params = OM.init(SIZES, seed=seed)
    flat = OM.flatten(params).astype(np.float32)
    m = P.dacp_mlp_create(40, 64, 3, 3, weights=flat)
    return m, [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
               for W, b in params]


def test_forward_and_gradient_match_oracle():
    m, params = _net()
    try:
        rng = np.random.default_rng(0)
        x = rng.standard_normal((37, 40)).astype(np.float32)
        t = rng.standard_normal((37, 3)).astype(np.float32)
        y = P.dacp_mlp_forward(m, x, 3)
        y_ref, _ = OM.forward(params, x.astype(np.float64))
        assert np.abs(y - y_ref).max() <= 1e-5 * max(1.0, np.abs(y_ref).max())
        g, loss = P.dacp_mlp_gradients(m, x, t, sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:])))
        grads, loss_ref = OM.backward(params, x.astype(np.float64), t.astype(np.float64))
        g_ref = OM.flatten(grads)
        assert abs(loss - loss_ref) <= 1e-5 * loss_ref
        assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    finally:
        P.dacp_mlp_destroy(m)


def test_normalisation_is_applied():
    m, params = _net()
    try:
        mu_in = np.linspace(-1, 1, 40).astype(np.float32)
        sd_in = np.linspace(0.5, 2, 40).astype(np.float32)
        mu_out = np.array([0.3, 6.0, 1.5], np.float32)
        sd_out = np.array([0.2, 2.0, 0.3], np.float32)
        P.dacp_mlp_set_normalization(m, mu_in, sd_in, mu_out, sd_out)
        x = np.random.default_rng(1).standard_normal((5, 40)).astype(np.float32)
        y = P.dacp_mlp_forward(m, x, 3)
        z, _ = OM.forward(params, (x - mu_in) / sd_in)
        assert np.abs(y - (z * sd_out + mu_out)).max() <= 1e-5 * np.abs(z * sd_out + mu_out).max()
    finally:
        P.dacp_mlp_destroy(m)


def test_output_range_clamps_outputs():
    """dacp_mlp_set_output_range: each denormalised output is clamped to [lo, hi];
    inside the range the outputs are unchanged; lo > hi is rejected."""
    m, params = _net(seed=3)
    try:
        x = np.random.default_rng(4).standard_normal((64, 40)).astype(np.float32)
        y0 = P.dacp_mlp_forward(m, x, 3)
        lo = np.quantile(y0, 0.25, axis=0).astype(np.float32)
        hi = np.quantile(y0, 0.75, axis=0).astype(np.float32)
        P.dacp_mlp_set_output_range(m, lo, hi)
        y = P.dacp_mlp_forward(m, x, 3)
        assert np.array_equal(y, np.clip(y0, lo, hi))
        with pytest.raises(P.DacpError):
            P.dacp_mlp_set_output_range(m, hi + 1.0, lo)
    finally:
        P.dacp_mlp_destroy(m)


def test_one_full_batch_adam_step_matches_oracle():
    m, params = _net(seed=5)
    try:
        rng = np.random.default_rng(2)
        x = rng.standard_normal((16, 40)).astype(np.float32)
        t = rng.standard_normal((16, 3)).astype(np.float32)
        lr = 1e-2
        P.dacp_mlp_train(m, x, t, batch=16, epochs=1, lr=lr)
        w = P.dacp_mlp_get_weights(m)
        grads, _ = OM.backward(params, x.astype(np.float64), t.astype(np.float64))
        state = {}
        OM.adam_step(params, grads, state, lr=lr)
        w_ref = OM.flatten(params)
        # weights whose gradient is tiny move by less than lr; compare everywhere
        assert np.abs(w - w_ref).max() <= 1e-5 + 1e-3 * lr
    finally:
        P.dacp_mlp_destroy(m)


def test_training_fits_a_smooth_map():
    m = P.dacp_mlp_create(40, 64, 3, 3, seed=7)
    try:
        rng = np.random.default_rng(3)
        x = rng.standard_normal((512, 40)).astype(np.float32)
        t = np.stack([np.tanh(x[:, 0]), x[:, 1] * x[:, 2], 0.5 * x[:, 3]], axis=1).astype(np.float32)
        l0 = float(((P.dacp_mlp_forward(m, x, 3) - t) ** 2).sum() / (2 * len(x)))
        P.dacp_mlp_train(m, x, t, batch=64, epochs=200, lr=2e-3)
        l1 = float(((P.dacp_mlp_forward(m, x, 3) - t) ** 2).sum() / (2 * len(x)))
        assert l1 < 0.1 * l0
    finally:
        P.dacp_mlp_destroy(m)


def test_features_match_couplings_and_kpm():
    models = [W.spin_glass_shard(9, seed=2), W.chain(10)]
    psis = [W.start_vectors(m["N"], 2, seed=4, r=i) for i, m in enumerate(models)]
    d = P.Dacp(models, psis, block_b=2, precision=P.DACP_FP64)
    try:
        d.choose_params(50)
        f = d.features()
        em = d.params()["emax"]
        for r, m in enumerate(models):
            N = m["N"]
            assert f[r, 0] == N
            assert abs(f[r, 1] - (np.log(50) - N * np.log(2))) < 1e-5
            assert abs(f[r, 2] - m["gamma"].mean()) < 1e-6 and abs(f[r, 3] - m["gamma"].std()) < 1e-5
            J = m["J"][np.triu_indices(N, 1)]
            J = J[J != 0]
            assert abs(f[r, 4] - J.mean()) < 1e-6 and abs(f[r, 5] - J.std()) < 1e-5
            mu = OP.kpm_moments(m, psis[r][:, 0], em[r], 33)
            assert np.abs(f[r, 8:40] - mu[1:33]).max() < 1e-6
    finally:
        d.close()


def test_network_knobs_drive_the_parameters():
    """A network with zero weights outputs its output mean: the knobs must then
    give the same parameters as the heuristic called with those knobs."""
    sizes_w = sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))
    m = P.dacp_mlp_create(40, 64, 3, 3, weights=np.zeros(sizes_w, np.float32))
    knobs = np.array([np.log(1.7), 7.0, 1.2], np.float32)
    P.dacp_mlp_set_normalization(m, np.zeros(40, np.float32), np.ones(40, np.float32), knobs, np.ones(3, np.float32))
    models = [W.spin_glass_shard(9, seed=s) for s in range(3)]
    psis = [W.start_vectors(9, 2, seed=4, r=i) for i in range(3)]
    d1 = P.Dacp(models, psis, block_b=2, precision=P.DACP_FP32)
    d2 = P.Dacp(models, psis, block_b=2, precision=P.DACP_FP32)
    try:
        d1.choose_params_mlp(m, 60)
        d2.choose_params(60, d_ratio=float(np.float32(1.7)), basis_ratio=float(knobs[2]), c_order=float(knobs[1]))
        p1, p2 = d1.params(), d2.params()
        assert np.allclose(p1["a"], p2["a"], rtol=1e-6)
        assert np.array_equal(p1["K"], p2["K"]) and np.array_equal(p1["n"], p2["n"])
    finally:
        d1.close()
        d2.close()
        P.dacp_mlp_destroy(m)


def test_fallback_reruns_short_realizations_in_the_library():
    """dacp_solve_learned: knobs that cannot return the requested count fall back to the heuristic.

    The network's outputs are clamped to window ratio 1 and basis ratio 0.6 (dacp_mlp_set_output_range),
    so b(2n+1) < n_eigs and every realization comes back short. The library must then re-run all of
    them with the heuristic and return exactly what a heuristic run of the same batch returns."""
    import math
    models = [W.spin_glass_shard(10, seed=s) for s in (1, 2, 3)]
    psis = [W.start_vectors(10, 4, seed=5, r=i) for i in range(3)]
    n_eigs = 40
    m = P.dacp_mlp_create(40, 64, 3, 3, seed=7)
    try:
        lo = np.array([math.log(1.0), 9.0, 0.6], np.float32)
        P.dacp_mlp_set_output_range(m, lo, lo)
        d = P.Dacp(models, psis, block_b=4, precision=P.DACP_DF32)
        try:
            d.choose_params_mlp(m, n_eigs)
            assert all(4 * (2 * n + 1) < n_eigs for n in d.params()["n"])   # the learned basis is too small
            eigs, nf, rank, nfb = d.solve(n_eigs, mlp=m)
            p_fb = d.params()
        finally:
            d.close()
    finally:
        P.dacp_mlp_destroy(m)
    assert nfb == 3
    ref = P.Dacp(models, psis, block_b=4, precision=P.DACP_DF32)
    try:
        eref, nref, rref, nfb0 = ref.solve(n_eigs)
    finally:
        ref.close()
    assert nfb0 == 0
    for r in range(3):
        assert nf[r] == nref[r] == n_eigs and rank[r] == rref[r]
        assert np.array_equal(eigs[r], eref[r])
    assert all(4 * (2 * n + 1) < n_eigs for n in p_fb["n"])     # the handle keeps the learned run's state
