"""The E_max bound arithmetic of the CUDA library, run on the host (no GPU).

dacp_test_emax_rule runs the same code as the device kernel for the
Ritz-residual rule (rule 1; the residual rule 0 is the same bisection arithmetic)
on a Lanczos tridiagonal. Here it is compared with the oracle's forms of both
rules (oracle.params: eigvalsh of the tridiagonal, ritz_last_components) on
Lanczos runs of shards, a chain and a Heisenberg chain.
"""

import numpy as np
import pytest

import workloads as W
from oracle import params as OP

P = pytest.importorskip("paper_2011_02107_gb300")


def _cases():
    out = []
    for m, seed in ((W.spin_glass_shard(10, seed=1), 0), (W.spin_glass_shard(11, seed=2), 1),
                    (W.chain(12), 2), (W.heisenberg_chain(10, seed=3), 3)):
        psi = W.start_vectors(m["N"], 1, seed=seed)[:, 0]
        for steps in (1, 2, 7, 20, 40):
            out.append(OP.lanczos_tridiagonal(m, psi, steps)[:2])
    return out


def test_both_rules_match_the_oracle():
    for al, be in _cases():
        k = len(al)
        T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
        th = np.linalg.eigvalsh(T)
        top = max(abs(th[0]), abs(th[-1]))
        res = top + be[k - 1]
        ritz = top + be[k - 1] * OP.ritz_last_components(al, be).max()
        got0 = P.dacp_test_emax_rule(al, be ** 2, 0)
        got1 = P.dacp_test_emax_rule(al, be ** 2, 1)
        assert abs(got0 - res) <= 1e-12 * res, (k, got0, res)
        assert abs(got1 - ritz) <= 1e-9 * ritz, (k, got1, ritz)
        assert top <= got1 <= got0 + 1e-12 * got0


def test_arguments_are_checked():
    with pytest.raises(P.DacpError):
        P.dacp_test_emax_rule(np.zeros(3), np.ones(3), 2)
    with pytest.raises(P.DacpError):
        P.dacp_test_emax_rule(np.zeros(65), np.ones(65), 0)
