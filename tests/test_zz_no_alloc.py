"""dacp_moments_noalloc against the allocating path, through the C ABI.

Callers that cannot allocate device memory (inside a stream capture, behind
their own memory pool, in allocation-free loops) get the Chebyshev moments of
one realization from dacp_moments_noalloc, whose scratch is a static device
array. Its moments must equal those of dacp_basis_moments / dacp_get_moments
for the same normalised start vector (filter order 0), within the float64
moment tolerance of the other parity tests (1e-9, |mu_j| <= mu_0 = 1), on two
calls in a row with different sizes so that state left by the first call
cannot leak into the second. This file is collected last on purpose.
"""

import numpy as np
import pytest

import workloads as W
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


def test_noalloc_moments_match_allocating_path_twice():
    for N, seed in ((12, 1), (9, 2)):
        m = W.spin_glass_shard(N, seed=seed)
        psi = W.start_vectors(N, 1, seed=seed)[:, 0]
        psi_n = psi / np.linalg.norm(psi)
        emax = Hm.pauli_norm_bound(m)
        mu_ref, kn = _reference(m, psi_n, emax, 0.05 * emax, 3)
        orders = kn + 1
        x = torch.from_numpy(psi_n.copy()).cuda()
        out = torch.full((2 * orders,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        P.dacp_moments_noalloc(m, emax, x.data_ptr(), orders, out.data_ptr())
        mu = out.cpu().numpy()
        assert np.isfinite(mu).all()
        assert mu.shape == mu_ref.shape
        assert abs(mu[0] - 1.0) < 1e-12
        assert np.abs(mu - mu_ref).max() < 1e-9


def test_noalloc_rejects_sizes_beyond_its_scratch():
    m = W.spin_glass_shard(17, seed=0)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.DacpError) as e:
        P.dacp_moments_noalloc(m, 10.0, x.data_ptr(), 4, x.data_ptr())
    assert e.value.status == 1
