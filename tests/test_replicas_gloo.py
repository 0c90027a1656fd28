"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2) exercise the
max-over-ranks timing, the whole-job rate and the per-replica noise ids that keep the
replicas' diluted sources disjoint.  No GPU and no data-path collective is involved:
replicas only exchange their timings."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        seconds = 1.0 + rank                    # rank 1 is the slow one
        tmax = bench.aggregate_max(seconds, w)
        bench.barrier(w)
        ids = bench.replica_noise_ids(r, 2)
        gathered = [None] * w
        dist.all_gather_object(gathered, ids)
        rate = bench.whole_job_rate(256, w, tmax)
        out.put((rank, tmax, gathered, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, gathered, rate in res:
        assert tmax == 2.0                      # the max over ranks, seen by every rank
        assert gathered == [[0, 1], [2, 3]]     # disjoint noise ids
        assert rate == 256 * 2 / 2.0            # sources of all ranks / max rank time


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_max(3.5, 1) == 3.5
    assert bench.whole_job_rate(256, 1, 2.0) == 128.0
    assert bench.replica_noise_ids(0, 2) == [0, 1]
