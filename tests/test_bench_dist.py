"""The bench's multi-rank path on the CPU: two gloo ranks each generate
their own batch of the same shape (weak scaling, no data-path collective)
and agree on the largest step time, which is what the bench reports."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    from paper_1311_2769_gb300 import synth
    w = synth.WORKLOADS["batch_4096_lognormal"]
    b = synth.generate(w, n_events=6, seed=bench.rank_seed(w, rank))
    t = bench.max_over_ranks(10.0 + rank, world, "cpu")
    q.put((rank, t, b.n_events, float(b.x[:64].astype("float64").sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_events_and_reduce_the_max():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1] == 11.0     # the largest time of the two ranks
    assert res[0][2] == res[1][2] == 6        # the same shape on every rank
    assert res[0][3] != res[1][3]             # but other events


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1311_2769_gb300 import synth
    w = synth.WORKLOADS["batch_4096_lognormal"]
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.rank_seed(w, 0) is None and bench.rank_seed(w, 2) == w.seed + 2000
