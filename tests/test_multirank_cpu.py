"""The multi-rank path on CPU (gloo, world size 2): rays are sharded by
contiguous ray-id ranges, each rank traces its range with counter-based
streams, and an integer sum of images and tallies equals the single-process
result bit for bit.  The ranks use the CPU oracle as the tracer (no GPU here);
the sharding and reduction are the ones bench.py uses (offset = (step *
world + rank) * n)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, steps, out):
    import torch
    import torch.distributed as dist

    from oracle import binding as ob
    from paper_2503_16955_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.von_hamos_hapg()
    img = np.zeros((w["spec"]["det_ny"], w["spec"]["det_nx"]), dtype=np.int64)
    tal = np.zeros(3, dtype=np.int64)
    for step in range(steps):
        off = (step * world + rank) * n
        im, t, _ = ob.trace(w["spec"], w["source"], n, w["seed"], ray_offset=off, n_threads=2)
        img += im
        tal += np.array([t["emitted"], t["det_hits"], t["collisions"]], dtype=np.int64)
    ti = torch.from_numpy(img)
    tt = torch.from_numpy(tal)
    dist.all_reduce(ti, op=dist.ReduceOp.SUM)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out + ".img.npy", ti.numpy())
        np.save(out + ".tal.npy", tt.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_single_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    from oracle import binding as ob
    from paper_2503_16955_gb300 import workloads as W

    n, steps, world = 4000, 2, 2
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(world, _free_port(), n, steps, out), nprocs=world, join=True,
                       start_method="spawn")
    img = np.load(out + ".img.npy")
    tal = np.load(out + ".tal.npy")
    w = W.von_hamos_hapg()
    ref, t, _ = ob.trace(w["spec"], w["source"], n * steps * world, w["seed"], ray_offset=0)
    assert np.array_equal(img, ref)
    assert list(tal) == [t["emitted"], t["det_hits"], t["collisions"]]
