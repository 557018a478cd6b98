"""Weak-scaling launch logic of bench.py on world_size 2 with the gloo backend (CPU only).

Each rank draws its own batch (seeds offset by rank, no data-path exchange), its full-model and its
parity-sector start vectors alike;
the timed region's length is the max over ranks and the found count the sum.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = dict(bench.WORKLOADS["c3"], N=6, R=3)
    models, psis = bench.make_inputs(wl, rank)
    sec = bench.sector_inputs(wl, rank)              # the parity-sector start blocks of the same batch
    assert len(sec) == 2 * wl["R"] and all(p.shape == (1 << (wl["N"] - 1), wl["b"]) for p in sec)
    sig = float(sum(m["J"].sum() for m in models) + sum(p.sum() for p in psis) + sum(p.sum() for p in sec))
    t = bench.reduce_across_ranks(1.0 + rank, "max", world)
    n = bench.reduce_across_ranks(10.0 * (rank + 1), "sum", world)
    sigs = [None] * world
    dist.all_gather_object(sigs, sig)
    out[rank] = (t, n, sigs)
    dist.destroy_process_group()


def test_two_rank_gloo_weak_scaling():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, n, sigs = out[r]
        assert t == 2.0 and n == 30.0
        assert len(set(np.round(sigs, 12))) == world      # every rank has its own batch
