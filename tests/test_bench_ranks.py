"""Host-side logic of the multi-GPU bench path, on CPU with world_size-2 gloo ranks: the
job time is the slowest replica's, the job throughput counts every rank's work, and under
the reference arm only rank 0 runs and prints."""
import io
import json
import os
import socket
import sys
import tempfile
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_local = [12.5, 20.0][rank]             # rank 1 is the slow replica
    ms, value = bench.aggregate_ranks(ms_local, 1.0e6, world, allreduce_max)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "value": value}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        res = [json.load(open(os.path.join(d, f"r{r}.json"))) for r in range(2)]
    for r in res:
        assert r["ms"] == 20.0                          # max over ranks, seen by every rank
        assert r["value"] == pytest.approx(2 * 1.0e6 / 20.0e-3)   # both replicas' work / job time


def test_single_rank_needs_no_collective():
    import bench
    ms, value = bench.aggregate_ranks(8.0, 4.0e5, 1)
    assert ms == 8.0 and value == pytest.approx(4.0e5 / 8.0e-3)


def test_reference_arm_other_ranks_exit_without_work():
    import bench

    class A:
        warmup, steps, ref_step_seconds, gpus = 1, 1, 0.01, 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(A(), rank=1, world=2) == 0
    assert buf.getvalue() == ""
