"""Multi-rank path on CPU: location partitioning and the gather of per-rank
results, with two gloo ranks (the per-rank compute is the FP64 oracle on the
rank's slice, so no GPU is needed)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_1310_5182_gb300 import shard


def test_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    n = rng.integers(30, 101, 2000)
    Np = rng.integers(500, 2001, 2000)
    cost = shard.location_cost(n, Np, 6)
    for ws in (1, 2, 3, 8):
        parts = shard.partition(cost, ws)
        assert parts[0][0] == 0 and parts[-1][1] == 2000
        assert all(a[1] == b[0] for a, b in zip(parts[:-1], parts[1:]))
        loads = np.array([cost[lo:hi].sum() for lo, hi in parts])
        assert loads.max() <= cost.sum() / ws + cost.max() + 1e-6
    assert shard.partition(cost[:3], 8)[-1] == (3, 3)  # more ranks than locations


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    w = W.toy2d(seed=41, N=3000, M=37, Np=120, n=16)

    def compute(lo, hi):
        r = O.run_pipeline(w.X, w.Y, w.Xref[lo:hi], w.n0, 16, 120, w.d, w.g)
        return {"mean": r["mean"], "s2": r["s2"]}

    out = shard.run_sharded(compute, w.Xref, 16, 120, w.n0, rank, world)
    np.save(os.path.join(outdir, f"mean{rank}.npy"), out["mean"])
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_full_result(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    from oracle import oracle as O
    w = W.toy2d(seed=41, N=3000, M=37, Np=120, n=16)
    ref = O.run_pipeline(w.X, w.Y, w.Xref, w.n0, 16, 120, w.d, w.g)
    for r in range(2):
        got = np.load(tmp_path / f"mean{r}.npy")
        np.testing.assert_array_equal(got, ref["mean"])
