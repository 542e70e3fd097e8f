"""The multi-GPU protocol of bench.py, run as two gloo ranks on the CPU:
each rank draws its own batch (no instance shared between ranks, no data-path
communication), the timings are reduced with MAX over ranks, and the whole-job
value is every rank's grid-point-steps over that maximum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1007_3470_gb300 import workloads as W
    insts, psis, _ = W.batch_1d(count=64, seed=bench.rank_seed(rank))
    sig = [round(i.w0, 12) for i in insts]
    gathered = [None] * world
    dist.all_gather_object(gathered, sig)
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    tmax, emax = bench.reduce_times_max([local_ms, 1.0 + rank], dist, "cpu")
    gps = float(sum(i.n[0] for i in insts) * 500)
    value = bench.aggregate_value(bench.reduce_sum(gps, dist, "cpu"), 3, tmax)
    out[rank] = (gathered, tmax, emax, value, gps)
    dist.destroy_process_group()


def test_two_ranks_shard_and_time_with_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (g0, t0, e0, v0, gps0), (g1, t1, e1, v1, gps1) = out[0], out[1]
    assert g0 == g1                        # every rank saw both batches
    assert set(g0[0]).isdisjoint(g0[1])    # the two batches share no instance
    assert t0 == t1 == 15.0 and e0 == e1 == 2.0
    assert gps0 != gps1                    # ranks carry different (independent) work
    assert v0 == v1 == pytest.approx((gps0 + gps1) * 3 / 15e-3)
