"""prosper_encode_noalloc: the allocation-free BSC encode entry point.

It exists for callers that cannot call cudaMalloc when they encode (code past
a fixed start-up phase that must never allocate, a process whose device memory
belongs to a framework's caching allocator, or code that must not synchronise
the device).  Its scratch is a fixed device array inside the library.  This
test calls it through the C ABI twice in a row, with different inputs, and
checks each result against prosper_encode on a regular context.  It sits in a
file of its own that pytest collects last, and it works alone in a fresh
process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1908_06843_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _encode_noalloc(lib, D, H, Hp, gamma, W, theta, Y):
    N = Y.shape[0]
    dev = Y.device
    out = dict(sel=torch.full((N, Hp), -7, dtype=torch.int16, device=dev),
               s_mean=torch.full((N, Hp), -7.0, device=dev),
               map_idx=torch.full((N, gamma), -7, dtype=torch.int16, device=dev),
               map_p=torch.full((N,), -7.0, device=dev),
               logZ=torch.full((N,), -7.0, device=dev))
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.prosper_encode_noalloc(D, H, Hp, gamma, P(W), P(theta), P(Y), N, P(out["sel"]),
                                    P(out["s_mean"]), P(out["map_idx"]), P(out["map_p"]),
                                    P(out["logZ"]),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.prosper_last_error()
    return out


def test_noalloc_matches_encode_twice():
    from paper_1908_06843_gb300 import Context, binding
    lib = binding.load()
    D, H, Hp, gamma = 256, 256, 10, 5
    dev = torch.device("cuda")
    ctx = Context(0, D, H, Hp, gamma, 0)
    for call, (n, seed, pi, sigma) in enumerate([(4096, 1002, 4 / 256, 0.2), (1000, 1005, 0.03, 0.25)]):
        d = synth.gabor(N=n, seed=seed)
        W = torch.tensor(d["Wt"].astype(np.float32), device=dev)
        theta = torch.tensor([pi, sigma, 0.0, 0.0], dtype=torch.float64, device=dev)
        Y = torch.tensor(d["Y"], device=dev)
        got = _encode_noalloc(lib, D, H, Hp, gamma, W, theta, Y)
        ref = ctx.encode(ctx.params(W, theta), Y)
        torch.cuda.synchronize()
        # same kernels on the same inputs: the tolerance of the other parity tests holds
        # (1e-5 on posterior means and q(MAP), integers exact)
        assert torch.equal(got["sel"], ref["sel"]), call
        assert torch.equal(got["map_idx"], ref["map_idx"]), call
        assert float((got["s_mean"] - ref["s_mean"]).abs().max()) <= 1e-5, call
        assert float((got["map_p"] - ref["map_p"]).abs().max()) <= 1e-5, call
        assert float((got["logZ"] - ref["logZ"]).abs().max()) <= 1e-5 * float(ref["logZ"].abs().max()), call


@pytest.mark.parametrize("D,H,Hp,gamma,N", [(25, 10, 6, 3, 1000),   # bars shape: D % 4 != 0
                                             (30, 17, 5, 0, 300),     # gamma = 0: only s = 0
                                             (30, 17, 1, 1, 65)])     # Hprime = 1
def test_noalloc_small_shapes_match_encode(D, H, Hp, gamma, N):
    """Shapes below the array's maximum (the fixed offsets and the D- and
    H-dependent strides), D not a multiple of 4 (scalar Y loads), gamma = 0 and
    Hprime = 1, twice in a row, against prosper_encode."""
    from paper_1908_06843_gb300 import Context, binding
    lib = binding.load()
    dev = torch.device("cuda")
    ctx = Context(0, D, H, Hp, gamma, 0)
    g = synth.rng(D + H + Hp)
    for call in range(2):
        Wt = g.standard_normal((H, D)).astype(np.float32)
        Y = (g.standard_normal((N, D)) * 1.5).astype(np.float32)
        W = torch.tensor(Wt, device=dev)
        theta = torch.tensor([0.15, 1.0, 0.0, 0.0], dtype=torch.float64, device=dev)
        Yg = torch.tensor(Y, device=dev)
        got = _encode_noalloc(lib, D, H, Hp, gamma, W, theta, Yg)
        ref = ctx.encode(ctx.params(W, theta), Yg)
        torch.cuda.synchronize()
        assert torch.equal(got["sel"], ref["sel"]), call
        if gamma > 0:
            assert torch.equal(got["map_idx"], ref["map_idx"]), call
        assert float((got["s_mean"] - ref["s_mean"]).abs().max()) <= 1e-5, call
        assert float((got["map_p"] - ref["map_p"]).abs().max()) <= 1e-5, call
        assert float((got["logZ"] - ref["logZ"]).abs().max()) <= 1e-5 * float(ref["logZ"].abs().max()), call


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1908_06843_gb300 import binding
    lib = binding.load()
    null = ctypes.c_void_p(0)
    rc = lib.prosper_encode_noalloc(256, 256, 10, 5, null, null, null, 4097, null, null, null,
                                    null, null, null)
    assert rc == -1 and b"N=4097" in lib.prosper_last_error()
    rc = lib.prosper_encode_noalloc(512, 256, 10, 5, null, null, null, 10, null, null, null,
                                    null, null, null)
    assert rc == -1
