"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path does not shard: N > 1 runs independent replicas, each on its own designs, and the job's
time is the maximum over ranks. Checked here: the max-over-ranks reduction every rank sees, the
whole-job rate, that the replicas' design seeds are disjoint, and that the reference arm runs on
rank 0 alone (the other ranks return without work).
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 25.0 * rank            # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    seeds = bench.replica_design_seeds(rank, 3)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    rate = bench.whole_job_rate(world, 5, ms * 1e-3)

    class Args:
        warmup, steps, n, alpha, volfrac = 0, 1, 128, 1e4, 0.2
    ref_rc = bench.run_reference(Args, rank, world) if rank != 0 else None
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
        fh.write(repr((ms, gathered, rate, ref_rc)))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_aggregation_gloo_world2(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    results = [eval(open(tmp_path / ("rank%d.txt" % r)).read()) for r in range(world)]
    for ms, gathered, rate, ref_rc in results:
        assert ms == 125.0                                   # every rank sees the slowest rank's time
        assert rate == pytest.approx(world * 5 / 0.125)       # units of all ranks / max time
        assert set(gathered[0]).isdisjoint(gathered[1])       # replicas solve different designs
    assert results[1][3] == 0                                 # reference arm: rank 1 exits without work
