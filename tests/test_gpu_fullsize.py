"""Oracle parity at the benchmark sizes (Sec. 2: truncated E-step; Eq. 1-2;
Table 1 rows BSC, MCA, GSC): the whole workload of each benchmark line runs
through the C ABI in the launch configuration bench.py times, and the FP64
oracle (all host cores) repeats the E-step on the GPU's candidate sets.

  - BSC Gabor, N = 200,000, D = H = 256, H' = 10, gamma = 5, both forms:
    every candidate set optimal within its form's bound (FP64 scores,
    vectorised), At, B, F, sum<|s|> and the M-step's W, pi, sigma within the
    FP32 tolerances of tests/parity.py;
  - MCA bars, N = 100,000 (H' = 8, gamma = 4): the rho-smoothed statistics,
    F, E||y - f||^2 and the M-step's W;
  - GSC, N = 50,000 (H' = 8, gamma = 3): At, B, the spike-and-slab sums, F.
"""
import numpy as np
import pytest

from paper_1908_06843_gb300 import synth
from parity import REL_AGG, REL_F, relfro, torch_stats_to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bsc_scores(Y, Wt):
    Wd = np.asarray(Wt, np.float64)
    return (np.asarray(Y, np.float64) @ Wd.T) / np.linalg.norm(Wd, axis=1)


def _selection_bad(Y, Wt, sel, Hp, tau_rows, chunk=25_000):
    bad = []
    for a in range(0, len(Y), chunk):
        sc = _bsc_scores(Y[a:a + chunk], Wt)
        kth = -np.partition(-sc, Hp - 1, axis=1)[:, Hp - 1]
        s = np.asarray(sel[a:a + chunk], np.int64)
        inside = np.take_along_axis(sc, s, axis=1).min(1)
        srt = np.sort(s, axis=1)
        distinct = np.all(srt[:, 1:] != srt[:, :-1], axis=1)
        bad.extend((a + np.flatnonzero((inside < kth - tau_rows(Y[a:a + chunk], sc)) | ~distinct)).tolist())
    return bad


@pytest.mark.parametrize("precision", [0, 1])
def test_bsc_full_workload_matches_oracle(orc, precision):
    from paper_1908_06843_gb300 import Context
    d = synth.gabor(N=200_000, seed=1002)
    Wt = d["Wt"].astype(np.float32)
    Wd = Wt.astype(np.float64)
    pi, sigma = 4 / 256, 0.2
    dev = torch.device("cuda")
    ctx = Context(0, 256, 256, 10, 5, precision)
    W = torch.tensor(Wt, device=dev)
    theta = torch.tensor([pi, sigma, 0.0, 0.0], dtype=torch.float64, device=dev)
    P = ctx.params(W, theta)
    Y = torch.tensor(d["Y"], device=dev)
    st = ctx.alloc_stats()
    ctx.estep(P, Y, st)
    sel = ctx.encode(P, Y)["sel"].cpu().numpy().astype(np.int32)
    torch.cuda.synchronize()
    ctx.status()
    g = torch_stats_to_numpy(st)
    if precision:
        A = np.abs(Wd)
        nrm = np.linalg.norm(Wd, axis=1)
        tau = lambda Yc, sc: 2.0 * 2.0 ** -7 * 1.01 * ((np.abs(np.asarray(Yc, np.float64)) @ A.T) / nrm).max(1) + 1e-6
    else:
        tau = lambda Yc, sc: 1e-5 * np.abs(sc).max(1) + 1e-6
    bad = _selection_bad(d["Y"], Wd, sel, 10, tau)
    assert not bad, f"{len(bad)} candidate sets not optimal within the bound, e.g. {bad[:5]}"
    ref = orc.estep(orc.BSC, d["Y"], Wd, pi, sigma, 10, 5, sel_in=sel)
    assert g["scal"][orc.SC_N] == 200_000
    assert relfro(g["At"], ref["At"]) <= REL_AGG, relfro(g["At"], ref["At"])
    assert relfro(g["B"], ref["B"]) <= REL_AGG, relfro(g["B"], ref["B"])
    assert abs(g["scal"][orc.SC_F] - ref["scal"][orc.SC_F]) <= REL_F * abs(ref["scal"][orc.SC_F])
    assert abs(g["scal"][orc.SC_S1] - ref["scal"][orc.SC_S1]) <= REL_AGG * ref["scal"][orc.SC_S1]
    assert abs(g["scal"][orc.SC_YY] - ref["scal"][orc.SC_YY]) <= 1e-6 * ref["scal"][orc.SC_YY]
    # the W update from each side's statistics (spec: W within 1e-5)
    W2, pi2, s2, _, _ = orc.mstep(orc.BSC, 200_000, ref, Wd, pi, sigma)
    ctx.mstep(st, 200_000, P)
    torch.cuda.synchronize()
    assert relfro(W.cpu().numpy(), W2) <= REL_AGG, relfro(W.cpu().numpy(), W2)
    th = theta.cpu().numpy()
    assert abs(th[0] - pi2) <= REL_AGG * pi2 and abs(th[1] - s2) <= REL_AGG * s2


def test_mca_full_workload_matches_oracle(orc):
    from paper_1908_06843_gb300 import MCA, Context
    d = synth.mca_bars(N=100_000, seed=1003)
    Wt = np.asarray(d["Wt"] + 0.05, np.float32)
    Wd = Wt.astype(np.float64)
    pi, sigma, rho = 0.1, 1.0, 20.0
    dev = torch.device("cuda")
    ctx = Context(MCA, 100, 20, 8, 4, max_points=100_000)
    W = torch.tensor(Wt, device=dev)
    theta = torch.tensor([pi, sigma, rho, 0.0], dtype=torch.float64, device=dev)
    P = ctx.params(W, theta)
    Y = torch.tensor(d["Y"], device=dev)
    st = ctx.alloc_stats()
    ctx.estep(P, Y, st)
    sel = ctx.encode(P, Y)["sel"].cpu().numpy().astype(np.int32)
    torch.cuda.synchronize()
    g = torch_stats_to_numpy(st)
    # selection: optimal within the FP32 bound on the MCA score (reading R14)
    sc = (np.asarray(d["Y"], np.float64) @ Wd.T) / Wd.sum(1)
    kth = -np.partition(-sc, 7, axis=1)[:, 7]
    inside = np.take_along_axis(sc, sel.astype(np.int64), axis=1).min(1)
    assert np.all(inside >= kth - (1e-5 * np.abs(sc).max(1) + 1e-6))
    ref = orc.estep(orc.MCA, d["Y"], Wd, pi, sigma, 8, 4, rho=rho, sel_in=sel)
    assert relfro(g["mca"], ref["mca"]) <= REL_AGG, relfro(g["mca"], ref["mca"])
    assert abs(g["scal"][orc.SC_F] - ref["scal"][orc.SC_F]) <= REL_F * abs(ref["scal"][orc.SC_F])
    assert abs(g["scal"][orc.SC_MCA_R2] - ref["scal"][orc.SC_MCA_R2]) <= REL_AGG * ref["scal"][orc.SC_MCA_R2]
    assert abs(g["scal"][orc.SC_S1] - ref["scal"][orc.SC_S1]) <= REL_AGG * ref["scal"][orc.SC_S1]
    W2, pi2, s2, _, _ = orc.mstep(orc.MCA, 100_000, ref, Wd, pi, sigma)
    ctx.mstep(st, 100_000, P)
    torch.cuda.synchronize()
    assert relfro(W.cpu().numpy(), W2) <= REL_AGG


def test_gsc_full_workload_matches_oracle(orc):
    from paper_1908_06843_gb300 import GSC, Context
    d = synth.gsc(N=50_000, seed=1004)
    Wt = np.asarray(d["Wt"], np.float32)
    Wd = Wt.astype(np.float64)
    mu = np.asarray(d["mu"], np.float32)
    psi = np.asarray(d["psi"], np.float32)
    pi, sigma = 3 / 32, 0.3
    dev = torch.device("cuda")
    ctx = Context(GSC, 64, 32, 8, 3, max_points=50_000)
    W = torch.tensor(Wt, device=dev)
    theta = torch.tensor([pi, sigma, 0.0, 0.0], dtype=torch.float64, device=dev)
    P = ctx.params(W, theta, torch.tensor(mu, device=dev), torch.tensor(psi, device=dev))
    Y = torch.tensor(d["Y"], device=dev)
    st = ctx.alloc_stats()
    ctx.estep(P, Y, st)
    sel = ctx.encode(P, Y)["sel"].cpu().numpy().astype(np.int32)
    torch.cuda.synchronize()
    g = torch_stats_to_numpy(st)
    ref = orc.estep(orc.GSC, d["Y"], Wd, pi, sigma, 8, 3, mu=mu.astype(np.float64),
                    psi=psi.astype(np.float64), sel_in=sel)
    assert relfro(g["At"], ref["At"]) <= REL_AGG, relfro(g["At"], ref["At"])
    assert relfro(g["B"], ref["B"]) <= REL_AGG, relfro(g["B"], ref["B"])
    assert relfro(g["gsc"], ref["gsc"]) <= REL_AGG, relfro(g["gsc"], ref["gsc"])
    assert abs(g["scal"][orc.SC_F] - ref["scal"][orc.SC_F]) <= REL_F * abs(ref["scal"][orc.SC_F])
