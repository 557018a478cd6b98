"""dacp_moments_noalloc through the C ABI, against the allocating path and the oracle.

Some callers cannot call cudaMalloc: engines whose device memory all comes
from their own pool or arena, and loops that must not enter an allocator.
They get the Chebyshev moments of one realization from dacp_moments_noalloc,
whose scratch is a static device array. Its moments must equal those of
dacp_basis_moments / dacp_get_moments for the same normalised start vector
(filter order 0) within the float64 moment tolerance of the other parity
tests (1e-9, |mu_j| <= mu_0 = 1), and the float64 oracle's directly recorded
moments (Appendix C) within the same tolerance.

The calls come in a row with different sizes, so state that one call leaves
in the shared array cannot leak into the next: N = 14 and 16 take 64 KB
tiles, several tiles per realization and the cross-tile partial sums and
counters inside the array (N = 16 is its edge); N = 12 and 9 take one tile.
A float64 handle with 8 KB tiles is created between the first and the second
call: the kernels' shared-memory limit must not fall below what the later
calls launch with. This file is collected last on purpose.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dacp as DA
from oracle import hamiltonian as Hm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")


def _reference(m, psi_n, emax, a, n):
    """Moments from the allocating path: K = 0 keeps psi_E = psi / |psi|."""
    d = P.Dacp([m], [psi_n[:, None]], block_b=1, precision=P.DACP_FP64)
    try:
        d.set_params(emax, a, 0, n)
        d.filter()
        d.basis_moments()
        kn = int(d.params()["kn"][0])
        return d.moments(0)[:, 0, 0], kn
    finally:
        d.close()


def test_noalloc_moments_match_allocating_path_and_oracle():
    small = None
    try:
        for i, (N, seed, n) in enumerate(((14, 3, 2), (16, 4, 1), (12, 1, 3), (9, 2, 3))):
            m = W.spin_glass_shard(N, seed=seed)
            psi = W.start_vectors(N, 1, seed=seed)[:, 0]
            psi_n = psi / np.linalg.norm(psi)
            emax = Hm.pauli_norm_bound(m)
            mu_ref, kn = _reference(m, psi_n, emax, 0.05 * emax, n)
            orders = kn + 1
            x = torch.from_numpy(psi_n.copy()).cuda()
            out = torch.full((2 * orders,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            P.dacp_moments_noalloc(m, emax, x.data_ptr(), orders, out.data_ptr())
            mu = out.cpu().numpy()
            assert np.isfinite(mu).all()
            assert mu.shape == mu_ref.shape
            assert abs(mu[0] - 1.0) < 1e-12
            assert np.abs(mu - mu_ref).max() < 1e-9, (N, np.abs(mu - mu_ref).max())
            mu_or, _ = DA.chebyshev_moments(m, psi_n, emax, 2 * orders - 1)
            assert np.abs(mu - mu_or[:, 0, 0]).max() < 1e-9, (N, np.abs(mu - mu_or[:, 0, 0]).max())
            if i == 0:
                ms = W.spin_glass_shard(10, seed=5)
                small = P.Dacp([ms], [W.start_vectors(10, 1, seed=5)], block_b=1, precision=P.DACP_FP64)
    finally:
        if small is not None:
            small.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    m = W.spin_glass_shard(17, seed=0)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.DacpError) as e:
        P.dacp_moments_noalloc(m, 10.0, x.data_ptr(), 4, x.data_ptr())
    assert e.value.status == 1
