"""The multi-GPU path shards independent instances across ranks (weak scaling, no
data-path collective).  Checked on CPU with two gloo ranks: the shards are disjoint and
cover the union, per-rank results (FP64 oracle, one load step) equal a single-process
solve of the union, and the max-over-ranks timing reduction is correct."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, B, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2307_16894_gb300 import workload
    from gpu_helpers import OracleRun
    rom, mu, coef, paths = workload.shard("c2", B, rank, steps=2)
    o = OracleRun(rom, coef)
    r = o.step(paths[:, 0], tol_abs=rom["tol_abs"], start="prev")
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), mu=mu, P=r["Pbar"], iters=r["iters"], tmax=t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding(tmp_path):
    B, world = 3, 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, B, str(tmp_path)), nprocs=world, start_method="spawn")
    from paper_2307_16894_gb300 import workload
    from gpu_helpers import OracleRun
    rom, mu, coef, paths = workload.batch("c2", B=B * world, steps=2)
    ref = OracleRun(rom, coef).step(paths[:, 0], tol_abs=rom["tol_abs"], start="prev")
    parts = [np.load(os.path.join(tmp_path, "rank%d.npz" % r)) for r in range(world)]
    assert np.array_equal(np.concatenate([p["mu"] for p in parts]), mu)
    assert np.array_equal(np.concatenate([p["P"] for p in parts]), ref["Pbar"])
    assert np.array_equal(np.concatenate([p["iters"] for p in parts]), ref["iters"])
    assert all(float(p["tmax"][0]) == world for p in parts)
