"""Data-parallel EM on the GPU (the paper's MPI design, Sec. 1, as
torch.distributed ranks): two ranks on one GPU, each E-steps its shard of the
bars data (kernels of different ranks never wait on one another), the
statistics are summed over gloo through host copies, and both ranks run the
same M-step.  The sums equal one process's statistics over all points, up to
the summation order of the FP32 partial sums of sum y<s>^T, and both ranks end
with bit-identical parameters.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _one_step(out, rank=0, world=1, port=0):
    import torch
    if world > 1:
        import torch.distributed as dist
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1908_06843_gb300 import BSC_ET, EM, LinearAnnealing, synth
    d = synth.bars(N=1001, seed=1001)          # odd N: unequal shards
    model = BSC_ET(25, 10, 6, 3)
    p = synth.init_bsc(d["Y"], 10, seed=2001, pi=0.5, normalise=False)
    params = model._pack(p["Wt"], p["pi"], p["sigma"])
    em = EM(model=model, anneal=LinearAnnealing(1), data={"y": d["Y"]}, lparams=params)
    em.run()
    torch.cuda.synchronize()
    st = {k: v.cpu().numpy() for k, v in model._st.items() if v is not None}
    np.savez(out, W=params["W"].cpu().numpy(), theta=params["theta"].cpu().numpy(),
             F=np.array(em.history), **st)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _worker(rank, world, port, prefix):
    _one_step(f"{prefix}_{rank}.npz", rank, world, port)


def test_two_ranks_sum_statistics_and_agree():
    import torch.multiprocessing as mp
    from parity import relfro
    with tempfile.TemporaryDirectory() as tmp:
        prefix = os.path.join(tmp, "rank")
        mp.start_processes(_worker, args=(2, _free_port(), prefix), nprocs=2, join=True,
                           start_method="spawn")
        _one_step(os.path.join(tmp, "single.npz"))
        r0 = np.load(prefix + "_0.npz")
        r1 = np.load(prefix + "_1.npz")
        one = np.load(os.path.join(tmp, "single.npz"))
        assert r0["scal"][3] == r1["scal"][3] == one["scal"][3] == 1001
        assert relfro(r0["B"], one["B"]) <= 1e-12
        assert relfro(r0["At"], one["At"]) <= 1e-6     # FP32 partial sums, other order
        assert abs(r0["scal"][0] - one["scal"][0]) <= 1e-12 * abs(one["scal"][0])
        np.testing.assert_array_equal(r0["W"], r1["W"])    # the same M-step on both ranks
        np.testing.assert_array_equal(r0["theta"], r1["theta"])
        assert relfro(r0["W"], one["W"]) <= 1e-5
        assert abs(r0["theta"][1] - one["theta"][1]) <= 1e-6 * one["theta"][1]
