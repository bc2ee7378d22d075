"""Host logic of the multi-GPU benchmark (independent replicas, one per rank),
run as world-size-2 process groups on the CPU (gloo): the job total is the sum
of the ranks' work over the slowest rank's time, and only rank 0 reports."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    work = 1000.0 * (rank + 1)          # rank 1 did twice the work ...
    ms = 10.0 + 5.0 * rank              # ... and took longer
    tot, tmax = bench.reduce_over_ranks(work, ms, w, "cpu")
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(rank=r, world=w, local=local, tot=tot, tmax=tmax), f)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_reduction_over_gloo(tmp_path, world):
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == world and d["local"] == r
        assert d["tot"] == 3000.0          # sum of the ranks' work
        assert d["tmax"] == 15.0           # the slowest rank's time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(123.0, 4.5, 1) == (123.0, 4.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the CPU reference arm runs and prints on rank 0 alone."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: called.append(1))
    args = argparse.Namespace(steps=1, warmup=3, gpus=2)
    assert bench.run_reference(args) == 0
    assert called == [] and capsys.readouterr().out == ""
