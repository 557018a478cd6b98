"""Allocation failure, injected on the host (no GPU fault): dacp_test_fail_alloc makes the k-th
device allocation of the library fail as if cudaMalloc had run out of memory.

For every k up to the number of allocations one create + parameters + solve sequence makes, the call
that hit the failure returns DACP_ERR_NOMEM and the handle, if there is one, is destroyed. Afterwards
the device's free memory is back where it started, and a clean run gives the same levels as before
the injections.
"""

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2011_02107_gb300")


def _run(models, psis, n_eigs):
    d = None
    try:
        d = P.Dacp(models, psis, block_b=4, precision=P.DACP_FP64)
        d.choose_params(n_eigs)
        eigs, nf, _ = d.run(n_eigs)
        return eigs, nf
    finally:
        if d is not None:
            d.close()


def test_every_allocation_failure_is_reported_and_cleaned_up():
    models = [W.spin_glass_shard(8, seed=1), W.random_model(9, seed=2)]
    psis = [W.start_vectors(m["N"], 4, seed=3, r=i) for i, m in enumerate(models)]
    ref, nf_ref = _run(models, psis, 20)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    completed_at = None
    try:
        for k in range(400):
            P.dacp_test_fail_alloc(k)
            try:
                _run(models, psis, 20)
            except P.DacpError as e:
                assert e.status == 3, (k, str(e))          # DACP_ERR_NOMEM
                failures += 1
            else:
                completed_at = k                            # fewer than k + 1 allocations: never fired
                break
            finally:
                P.dacp_test_fail_alloc(-1)
    finally:
        P.dacp_test_fail_alloc(-1)
    assert completed_at is not None and failures == completed_at and failures >= 5, (failures, completed_at)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 64 << 20, (free0, free1)         # nothing left allocated
    got, nf = _run(models, psis, 20)
    assert list(nf) == list(nf_ref)
    for a, b in zip(got, ref):
        assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())
