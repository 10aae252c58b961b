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
