"""GPU parity of the Appendix D comparison method (dacp_lanczos_filtered) against the oracle.

The Krylov space of the exp-semicircle-filtered operator is built with the
library's filter kernels and cuBLAS Gram-Schmidt, and Rayleigh-Ritz of H in it
gives converged Ritz values (residual test). A Krylov space depends on its
vectors' rounding only through its converged directions, so the comparison is
level by level on what both sides return as converged: each value within 1e-9
of the spectral width of the oracle's (oracle.lanczos) and of the dense
spectrum; the counts agree. The +-E case (a chain with a symmetric spectrum,
T_K(F) even in E) must come back short on both sides.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hamiltonian as Hm
from oracle import lanczos as LZ
from oracle import params as OP

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")


def _gpu(m, psi, emax, a, K, steps, n_eigs):
    d = P.Dacp([m], [psi], block_b=1, precision=P.DACP_FP64)
    try:
        d.set_params(emax, a, K, 1)
        return P.dacp_lanczos_filtered(d.handle, 0, steps, n_eigs)
    finally:
        d.close()


@pytest.mark.parametrize("N,seed", [(8, 15), (10, 3)])
def test_lanczos_filtered_matches_oracle_and_dense(N, seed):
    m = W.random_model(N, seed=seed)
    E = np.linalg.eigvalsh(Hm.dense_h(m))
    width = E[-1] - E[0]
    R = 6
    psi = W.start_vectors(N, 1, seed=4)
    emax = OP.emax_bound(m, psi[:, 0])
    a = np.sort(np.abs(E))[2 * R]
    K = OP.filter_order(emax, a)
    got, dim, ms, hv = _gpu(m, psi, emax, a, K, 4 * R, R)
    ref, dim_ref = LZ.lanczos_filtered(m, psi[:, 0], emax, a, K, 4 * R, R)
    assert dim == dim_ref == 4 * R
    assert hv == (dim - 1) * 2 * K + dim and np.all(ms >= 0)
    assert len(got) == len(ref) > 0
    assert np.abs(got - ref).max() <= 1e-9 * width
    assert max(np.min(np.abs(E - x)) for x in got) <= 1e-9 * width


def test_lanczos_filtered_does_not_resolve_plus_minus_pairs():
    """Integrable chain (symmetric spectrum): with a start vector in the span of one +-E pair the
    space is one-dimensional and its Ritz value (a mix of +-E) fails the residual test."""
    m = W.chain(6, J=1.0, hx=1.0, hz=0.0)
    E, Q = np.linalg.eigh(Hm.dense_h(m))
    k = int(np.argmin(np.where(E > 1e-6, E, np.inf)))
    j = int(np.argmin(np.abs(E + E[k])))
    assert abs(E[j] + E[k]) < 1e-10
    psi = (0.8 * Q[:, k] + 0.3 * Q[:, j])[:, None]
    emax = 1.05 * np.abs(E).max()
    got, dim, _, _ = _gpu(m, psi, emax, 3.0 * E[k], 20, 5, 5)
    assert dim == 1 and len(got) == 0
    ref, dim_ref = LZ.lanczos_filtered(m, psi[:, 0], emax, 3.0 * E[k], 20, 5, 5)
    assert dim_ref == 1 and len(ref) == 0


def test_lanczos_filtered_arguments():
    m = W.chain(6)
    d = P.Dacp([m], [W.start_vectors(6, 1, seed=0)], block_b=1, precision=P.DACP_FP64)
    try:
        with pytest.raises(P.DacpError) as e:
            P.dacp_lanczos_filtered(d.handle, 0, 4, 2)          # no parameters yet
        assert e.value.status == 6
        d.set_params(10.0, 1.0, 10, 1)
        for r, steps, n in ((1, 4, 2), (0, 0, 2), (0, 65, 2), (0, 4, 0)):
            with pytest.raises(P.DacpError) as e:
                P.dacp_lanczos_filtered(d.handle, r, steps, n)
            assert e.value.status == 1
    finally:
        d.close()
