"""Multi-rank path on CPU: two gloo ranks each evaluate a contiguous shard of a
batch (here with the FP64 oracle standing in for the per-GPU evaluator: this
container has no GPU) and gather lnL; the result equals a single-process
evaluation row for row, and max_over_ranks returns the larger step time."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    from tests import cases
    from paper_2609_30145_gb300.shard import gather_rows, max_over_ranks, shard_rows
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.WORKLOADS["tiny_phot_16x4x512"]
    orc = cases.oracle_for(w)
    th = cases.theta_rows(w, 37, seed=90)
    sl = shard_rows(th.shape[0], rank, world)
    local = torch.from_numpy(orc.eval(th[sl], nthreads=1)["lnl"])
    full = gather_rows(local, th.shape[0], world)
    t = max_over_ranks(1.0 + rank)
    if rank == 0:
        np.save(os.path.join(out_dir, "lnl.npy"), full.numpy())
        np.save(os.path.join(out_dir, "t.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_rows_partition():
    from paper_2609_30145_gb300.shard import shard_rows
    for n in (0, 1, 7, 64, 1025):
        for world in (1, 2, 3, 8):
            parts = [shard_rows(n, k, world) for k in range(world)]
            assert parts[0].start == 0 and parts[-1].stop == n
            assert all(a.stop == b.start for a, b in zip(parts, parts[1:]))
            sizes = [p.stop - p.start for p in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_match_single_process(tmp_path):
    import synth
    from tests import cases
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    w = synth.WORKLOADS["tiny_phot_16x4x512"]
    orc = cases.oracle_for(w)
    th = cases.theta_rows(w, 37, seed=90)
    ref = orc.eval(th, nthreads=1)["lnl"]
    got = np.load(tmp_path / "lnl.npy")
    assert np.array_equal(got, ref)
    assert np.load(tmp_path / "t.npy")[0] == 2.0
