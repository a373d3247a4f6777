"""ET's data-point cut on the GPU against the oracle (reading of the ET variant
the paper's truncated posteriors, Sec. 2, come from): N_cut =
floor(N P_pi(|s| <= gamma)), statistics over the points whose log Z reaches the
N_cut-th largest value, pi corrected by H pi / E_pi[|s| : |s| <= gamma].

The oracle is given the GPU's candidate sets and the GPU's FP32 log Z values
(from the encode path, which computes them with the same kernels), so that
both sides cut at the same points; the kept points' statistics and the
M-step are then compared with the FP32 tolerances of tests/parity.py.
"""
import numpy as np
import pytest

from paper_1908_06843_gb300 import synth
from parity import REL_AGG, REL_F, relfro, torch_stats_to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(orc, model, Y, Wt, pi, sigma, Hp, gamma, precision=0):
    from paper_1908_06843_gb300 import Context
    H, D = Wt.shape
    Wt32 = np.asarray(Wt, np.float32)
    ctx = Context(model, D, H, Hp, gamma, precision)
    ctx.set_data_cut(True)
    dev = torch.device("cuda")
    W = torch.tensor(Wt32, device=dev)
    theta = torch.tensor([pi, sigma] + [0.0] * 6, dtype=torch.float64, device=dev)
    P = ctx.params(W, theta)
    Yg = torch.tensor(np.asarray(Y, np.float32), device=dev)
    st = ctx.alloc_stats()
    ctx.estep(P, Yg, st)
    enc = ctx.encode(P, Yg)
    torch.cuda.synchronize()
    ctx.status()
    g = torch_stats_to_numpy(st)
    sel = enc["sel"].cpu().numpy().astype(np.int32)
    lz = enc["logZ"].cpu().numpy().astype(np.float64)
    ref, keep, ncut = orc.estep_cut(model, np.asarray(Y, np.float32), Wt32.astype(np.float64), pi,
                                    sigma, Hp, gamma, sel_in=sel, logZ_in=lz)
    assert 1 <= ncut < len(Y)
    assert keep.sum() >= ncut and g["scal"][orc.SC_N] == keep.sum()
    assert lz[keep].min() >= lz[~keep].max()
    assert relfro(g["At"], ref["At"]) <= REL_AGG, relfro(g["At"], ref["At"])
    assert relfro(g["B"], ref["B"]) <= REL_AGG, relfro(g["B"], ref["B"])
    assert abs(g["scal"][orc.SC_F] - ref["scal"][orc.SC_F]) <= REL_F * abs(ref["scal"][orc.SC_F])
    assert abs(g["scal"][orc.SC_S1] - ref["scal"][orc.SC_S1]) <= REL_AGG * ref["scal"][orc.SC_S1]
    return ctx, st, g, (W, theta, P), keep


@pytest.mark.parametrize("precision", [0, 1])
def test_bsc_data_cut(orc, precision):
    """Gabor shape, H' = 10, gamma = 2: P(|s| <= 2) ~ 0.24, so about a quarter
    of the 3,000 points are kept."""
    d = synth.gabor(N=3000, seed=1021)
    Wt = d["Wt"].astype(np.float32).astype(np.float64)
    _run(orc, orc.BSC, d["Y"], Wt, 4 / 256, 0.2, 10, 2, precision)


def test_data_cut_mstep_corrects_pi(orc):
    """The M-step on the kept points' statistics: W as the plain M-step, pi
    times H pi / E_pi[|s| : |s| <= gamma]."""
    d = synth.gabor(N=3000, seed=1022, H=64)
    Wt = d["Wt"].astype(np.float32).astype(np.float64)
    ctx, st, g, (W, theta, P), keep = _run(orc, orc.BSC, d["Y"], Wt, 0.06, 0.2, 8, 3)
    nk = int(keep.sum())
    W2, pi2, s2, _, _ = orc.mstep_cut(orc.BSC, nk, g, Wt, 0.06, 0.2, 3)
    ctx.mstep(st, nk, P)
    torch.cuda.synchronize()
    ctx.status()
    assert relfro(W.cpu().numpy(), W2) <= 1e-6
    th = theta.cpu().numpy()
    assert abs(th[0] - pi2) <= 1e-9 * pi2 and abs(th[1] - s2) <= 1e-7 * s2
    assert orc.pi_correction(64, 3, 0.06) > 1.0


def test_tsc_data_cut(orc):
    d = synth.discrete(N=2000, seed=1023, H=48)
    _run(orc, orc.TSC, d["Y"], d["Wt"], 4 / 48, 0.2, 8, 2)


def test_data_cut_rejected_for_other_models():
    from paper_1908_06843_gb300 import MCA, Context, ProsperError
    ctx = Context(MCA, 100, 20, 8, 4)
    with pytest.raises(ProsperError):
        ctx.set_data_cut(True)
