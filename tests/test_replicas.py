"""Host-side logic of the multi-GPU bench (one process per GPU, independent replicas of the workload:
weak scaling with no data-path collective): two gloo ranks on the CPU check the maximum-over-ranks
step time and the whole-job throughput, and that the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    r, w, l = bench._dist()
    ms = bench.replica_time(10.0 + 5.0 * rank, world)      # rank 1 is the slower replica
    val = bench.weak_value(1e9, world, ms)
    # the reference arm: every rank but 0 exits at once without work
    ref_rc = bench.run_reference(type("A", (), {"workload": "channel_q2_8x8x8", "warmup": 0, "steps": 1,
                                                 "ref_seconds": 1.0})()) if rank != 0 else 0
    out.put((rank, r, w, l, ms, val, ref_rc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, l, ms, val, ref_rc in res:
        assert (r, w, l) == (rank, 2, rank)
        assert ms == 15.0                                  # maximum over ranks
        assert abs(val - 2 * 1e9 / 15e-3 / 1e9) < 1e-9     # both replicas' units over the slowest time
        assert ref_rc == 0
