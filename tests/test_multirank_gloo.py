"""World-size-2 checks of the multi-rank logic on CPU (gloo backend).

* bench.py's rank helper: barrier, max and sum reductions over ranks, as the
  benchmark uses them for its max-over-ranks timing and whole-job totals.
* Sharding of the particle work: each rank runs the oracle on an interleaved
  half of the release list; summing the counts and taking the maximum of the
  energy over ranks gives exactly the single-rank rasters (both reductions are
  order-independent and Philox streams are keyed by global cell indices).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), AWO_DIST_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2506_23364_gb300 import inputs

    R = bench.Ranks()
    assert R.world == world and R.rank == rank
    R.barrier()
    mx = R.reduce(10.0 + rank, "max")
    sm = R.reduce(1.0 + rank, "sum")

    z = inputs.fbm(72, 0.8, seed=6, relief=700.0, m=90)
    h = oracle.decode_u16(inputs.quantise_dm(z))
    _, t2, _ = oracle.normals(h, 10.0)
    _, cells = oracle.release(t2, 30.0, 45.0)
    p = oracle.SimParams(traj_per_cell=8, max_steps=300, seed=11)
    mine = cells[rank::world]
    c64, maxe, st = oracle.simulate(h, 10.0, mine, p)
    tc = torch.from_numpy(c64.astype(np.int64))
    tm = torch.from_numpy(maxe.copy())
    dist.all_reduce(tc, op=dist.ReduceOp.SUM)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    steps = R.reduce(float(st["total_steps"]), "sum")
    if rank == 0:
        ref_c, ref_m, ref_st = oracle.simulate(h, 10.0, cells, p)
        ok = (np.array_equal(tc.numpy(), ref_c.astype(np.int64)) and np.array_equal(tm.numpy(), ref_m)
              and steps == ref_st["total_steps"] and mx == 10.0 + world - 1
              and sm == sum(1.0 + r for r in range(world)))
        with open(os.path.join(out_dir, "result.txt"), "w") as f:
            f.write("ok" if ok else "mismatch")
    R.close()


def test_two_ranks_gloo(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    assert (tmp_path / "result.txt").read_text() == "ok"
