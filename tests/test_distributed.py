"""Data-parallel E-step over ranks (world size 2, gloo, CPU): the statistics
summed over the shards equal the statistics of the whole data set, and the
M-step from the summed statistics equals the single-process M-step."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1908_06843_gb300 import synth
from paper_1908_06843_gb300.distributed import allreduce_stats, shard_range


def test_shard_range_partitions():
    for N in [0, 1, 7, 1000, 200_003]:
        for world in [1, 2, 3, 8]:
            spans = [shard_range(N, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == N
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.bars(N=801, seed=1001)
    p = synth.init_bsc(d["Y"], 10, seed=2001, pi=0.5, normalise=False)
    a, b = shard_range(len(d["Y"]), rank, world)
    ref = oracle.estep(oracle.BSC, d["Y"][a:b], p["Wt"], p["pi"], p["sigma"], 6, 3)
    st = {k: torch.tensor(ref[k]) for k in ("At", "B", "scal")}
    allreduce_stats(st)
    if rank == 0:
        np.savez(out_path, **{k: v.numpy() for k, v in st.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_statistics_sum(tmp_path, orc):
    out = str(tmp_path / "st.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    d = synth.bars(N=801, seed=1001)
    p = synth.init_bsc(d["Y"], 10, seed=2001, pi=0.5, normalise=False)
    full = orc.estep(orc.BSC, d["Y"], p["Wt"], p["pi"], p["sigma"], 6, 3)
    np.testing.assert_allclose(got["At"], full["At"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(got["B"], full["B"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(got["scal"], full["scal"], rtol=1e-12)
    W1, pi1, s1, _, _ = orc.mstep(orc.BSC, 801, dict(got), p["Wt"], p["pi"], p["sigma"])
    W2, pi2, s2, _, _ = orc.mstep(orc.BSC, 801, full, p["Wt"], p["pi"], p["sigma"])
    np.testing.assert_allclose(W1, W2, rtol=1e-10, atol=1e-10)
    assert abs(pi1 - pi2) < 1e-12 and abs(s1 - s2) < 1e-12
