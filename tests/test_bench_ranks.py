"""bench.py's multi-rank bookkeeping on CPU, with two gloo ranks: each rank
draws its own reference locations, the timed seconds are MAX-reduced over the
ranks, the aggregate rate counts every rank's locations, and under the
reference arm only rank 0 runs and prints."""
import contextlib
import io
import os
import socket
import sys

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.workload_for_rank(rank, M=64)
    np.save(os.path.join(outdir, f"xref{rank}.npy"), w.Xref)
    t_local = [1.5, 4.0][rank]
    t_max = bench.max_over_ranks(t_local, world)
    rate = bench.aggregate_rate(w.M, world, 10, t_max)
    np.save(os.path.join(outdir, f"t{rank}.npy"), np.array([t_max, rate]))
    # the reference arm: rank 1 returns before any work and prints nothing
    if rank == 1:
        class A:
            warmup, steps, gpus = 1, 1, 2
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(A, rank, world)
        assert buf.getvalue() == ""
    dist.destroy_process_group()


def test_two_gloo_ranks_bench_bookkeeping(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    x0, x1 = np.load(tmp_path / "xref0.npy"), np.load(tmp_path / "xref1.npy")
    assert x0.shape == x1.shape == (64, 8)
    assert not np.array_equal(x0, x1)          # weak scaling: distinct locations per rank
    assert (x1 >= 0).all() and (x1 <= 1).all()  # in the borehole's unit cube
    for r in range(2):
        t_max, rate = np.load(tmp_path / f"t{r}.npy")
        assert t_max == 4.0                    # the slowest rank's time, on every rank
        assert rate == 64 * 2 * 10 / 4.0       # every rank's predictions over that time
