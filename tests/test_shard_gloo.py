"""Source sharding over ranks, run as a world-size-2 process group on the CPU
(gloo): each rank traces its share of the sources with the FP64 oracle, the
rate fields and budgets are summed with the package's all-reduce, and the sum
equals the unsharded trace (the rates of disjoint source sets add; Sec. 2.1
step iii, Eq. ion) to FP64 rounding."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import workloads as W
    return W.cosmic(n=24, nsrc=9, sigma_ln=1.5, seed=11)


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_1807_07094_gb300 import shard
    from helpers import oracle_trace
    import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _workload()
    mine = shard.partition_sources(w.src_ndot, world)[rank]
    o = oracle_trace(W.subset_sources(w, mine))
    g = torch.from_numpy(np.ascontiguousarray(o["gamma"]))
    h = torch.from_numpy(np.ascontiguousarray(o["heat"]))
    b = shard.allreduce_rates(g, h, o["budget"])
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), gamma=g.numpy(), heat=h.numpy(), budget=b,
             mine=mine)
    dist.destroy_process_group()


def test_partition_covers_every_source_once_and_balances():
    sys.path.insert(0, ROOT)
    from paper_1807_07094_gb300 import shard
    rng = np.random.Generator(np.random.PCG64(3))
    ndot = 10 ** rng.uniform(48, 51, (100, 3))
    for world in (1, 2, 3, 8):
        parts = shard.partition_sources(ndot, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(100))
        loads = [ndot[p].sum() for p in parts]
        # greedy bound: no rank exceeds the mean by more than the brightest source
        assert max(loads) <= np.mean(loads) + ndot.sum(axis=1).max() + 1e-6 * ndot.sum()


@pytest.mark.parametrize("world", [2])
def test_sharded_trace_sums_to_the_unsharded_one(tmp_path, world):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import oracle_trace
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert sorted(np.concatenate([r["mine"] for r in res]).tolist()) == list(range(9))
    assert all(len(r["mine"]) > 0 for r in res)
    full = oracle_trace(_workload())
    for r in res:
        for name in ("gamma", "heat"):
            ref = full[name]
            m = ref > 0
            assert np.array_equal(r[name] > 0, m)
            assert np.max(np.abs(r[name][m] - ref[m]) / ref[m]) < 1e-12
        em, ab, es = r["budget"]
        assert abs(em / full["budget"][0] - 1) < 1e-14
        # the absorbed photons are a long FP64 running sum per trace (one
        # addition per segment); summing per-rank totals reorders it
        assert abs(ab / full["budget"][1] - 1) < 1e-10
        assert abs(em - ab - es) <= 1e-9 * em
