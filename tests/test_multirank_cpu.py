"""The multi-rank path on CPU (gloo, world size 2).

Photon histories are independent (Section 2.4: one thread per history), so a
projection shards by history range: each rank runs its own range and the
only exchange is an element-wise int64 sum of the tallies, which is exact and
order-independent.  A scan shards by angle with no exchange at all.  Both
are checked here with the CPU oracle standing in for each rank's GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1204_6367_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = inputs.small_problem()
    lo, hi = n * rank // world, n * (rank + 1) // world
    tp, ts, _, _ = oracle.mc_run(prob, hi - lo, seed=13, history_offset=lo)
    t = torch.from_numpy(np.stack([tp, ts]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    # angle sharding: rank r projects angle r of the scan, no exchange
    ap, _, _, _ = oracle.mc_run(prob, 3000, seed=13, phi=0.5 * rank, angle_index=rank)
    if rank == 0:
        np.save(os.path.join(out_dir, "sum.npy"), t.numpy())
    np.save(os.path.join(out_dir, f"angle{rank}.npy"), ap)
    dist.barrier()
    dist.destroy_process_group()


def test_history_shards_sum_to_single_run(tmp_path):
    n, world = 60_000, 2
    oracle.build()
    mp.start_processes(_rank_main, args=(world, _free_port(), n, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    prob = inputs.small_problem()
    tp, ts, _, _ = oracle.mc_run(prob, n, seed=13)
    got = np.load(tmp_path / "sum.npy")
    np.testing.assert_array_equal(got[0], tp)
    np.testing.assert_array_equal(got[1], ts)
    for r in range(world):
        ap, _, _, _ = oracle.mc_run(prob, 3000, seed=13, phi=0.5 * r, angle_index=r)
        np.testing.assert_array_equal(np.load(tmp_path / f"angle{r}.npy"), ap)


def _bench_rank_main(rank, world, port, out_dir):
    # bench.py's rank plumbing with gloo on CPU: each rank's angle, the job
    # time as the slowest rank's, the whole-job rate from it
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["RANK"] = str(rank)
    os.environ["LOCAL_RANK"] = str(rank)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    step_ms = 10.0 + 5.0 * r                          # rank 1 is the slower one
    tot = bench.max_over_ranks(step_ms, w, device="cpu")
    rate = bench.job_rate(1000, w, 3, tot)
    np.save(os.path.join(out_dir, f"bench{r}.npy"), np.array([bench.rank_angle(r, w), tot, rate, local]))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rank_plumbing(tmp_path):
    world = 2
    mp.start_processes(_bench_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    got = [np.load(tmp_path / f"bench{r}.npy") for r in range(world)]
    angles = [g[0] for g in got]
    assert angles == [0.0, np.pi]                     # one projection angle per rank, an orbit split
    for r, g in enumerate(got):
        assert g[1] == 15.0                           # every rank reports the slowest rank's time
        assert g[2] == pytest.approx(1000 * 2 * 3 / 0.015)   # all ranks' histories over that time
        assert g[3] == r
