"""Failure detection without a GPU fault: kernels flag problems in a device
status word that prosper_status reads; a bounded tensor-core wait that runs
out (its completion is never signalled) returns an error and leaves the
context usable.  Nothing here traps, faults or hangs the GPU."""
import os

import numpy as np
import pytest

from paper_1908_06843_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(precision=0):
    from paper_1908_06843_gb300 import Context
    d = synth.gabor(N=1000, seed=1002)
    ctx = Context(0, 256, 256, 10, 5, precision)
    W = torch.tensor(d["Wt"].astype(np.float32), device="cuda")
    theta = torch.tensor([4 / 256, 0.2, 0, 0], dtype=torch.float64, device="cuda")
    return ctx, ctx.params(W, theta), d["Y"], (W, theta)


def test_nonfinite_input_is_reported_and_context_stays_usable():
    from paper_1908_06843_gb300.binding import ProsperError
    ctx, P, Y, keep = _setup()
    Yb = Y.copy()
    Yb[17, 3] = np.nan
    st = ctx.alloc_stats()
    ctx.estep(P, torch.tensor(Yb, device="cuda"), st)
    with pytest.raises(ProsperError, match=r"\(-4\)"):
        ctx.status()
    with pytest.raises(ProsperError, match=r"\(-4\)"):      # host-buffer entry point too
        ctx.estep_host(P, Yb)
    ctx.estep(P, torch.tensor(Y, device="cuda"), st)         # clean data: no error left over
    ctx.status()
    assert np.isfinite(st["scal"].cpu().numpy()).all()


def test_indefinite_mstep_matrix_is_reported():
    from paper_1908_06843_gb300 import Context
    from paper_1908_06843_gb300.binding import ProsperError
    ctx = Context(0, 8, 4, 2, 1)
    W = torch.ones(4, 8, device="cuda")
    theta = torch.tensor([0.3, 1.0, 0, 0], dtype=torch.float64, device="cuda")
    P = ctx.params(W, theta)
    st = ctx.alloc_stats()
    B = np.eye(4)
    B[0, 1] = B[1, 0] = 2.0                                  # indefinite active block
    st["B"].copy_(torch.tensor(B * 10))
    st["scal"].copy_(torch.tensor([0, 5.0, 100.0, 10, 0, 0, 0, 0], dtype=torch.float64))
    ctx.mstep(st, 10, P)
    with pytest.raises(ProsperError, match=r"\(-4\)"):
        ctx.status()
    ctx.status()                                             # cleared


def test_tensor_core_wait_limit():
    """The BF16 projection waits for its MMA chain on an mbarrier with a time
    limit.  With the test hook the chain is never issued, so the wait runs out
    (50 ms), the kernel sets the timeout flag, frees its tensor memory and
    returns; prosper_status reports PROSPER_ETIMEOUT and a fresh context works."""
    from paper_1908_06843_gb300.binding import ProsperError
    os.environ["PROSPER_TEST_TC_NO_COMMIT_MS"] = "50"
    try:
        ctx, P, Y, keep = _setup(precision=1)
    finally:
        del os.environ["PROSPER_TEST_TC_NO_COMMIT_MS"]
    out = ctx.encode(P, torch.tensor(Y[:300], device="cuda"))
    with pytest.raises(ProsperError, match=r"\(-5\)"):
        ctx.status()
    ctx.close()
    ctx2, P2, Y2, keep2 = _setup(precision=1)
    ref = ctx2.encode(P2, torch.tensor(Y2[:300], device="cuda"))
    ctx2.status()
    assert int((ref["sel"] >= 0).all()) == 1
