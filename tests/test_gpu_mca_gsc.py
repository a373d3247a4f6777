"""GPU parity of the MCA and GSC truncated E-steps, encodings and M-steps
against the FP64 oracle on the same seeded inputs.

MCA: Table 1 row MCA (max superposition, binary latents); GSC: Table 1 row
GSC (linear superposition, spike-and-slab prior); truncated posteriors and
EM (Sec. 2); Hprime / gamma, step and inference (Sec. 3).
"""
import numpy as np
import pytest

from paper_1908_06843_gb300 import synth
from parity import (REL_AGG, REL_F, check_points, check_selection, relfro,
                    torch_stats_to_numpy)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tau(n, sc):
    return 1e-5 * np.max(np.abs(sc)) + 1e-5


def run_model(orc, model, Y, Wt, pi, sigma, Hp, gamma, rho=0.0, mu=None, psi=None):
    from paper_1908_06843_gb300 import Context
    H, D = Wt.shape
    Y32 = np.asarray(Y, np.float32)
    Wt32 = np.asarray(Wt, np.float32).astype(np.float64)
    dev = torch.device("cuda")
    ctx = Context(model, D, H, Hp, gamma)
    W = torch.tensor(Wt32.astype(np.float32), device=dev)
    theta = torch.tensor([pi, sigma, rho, 0.0], dtype=torch.float64, device=dev)
    kw = {}
    mu_t = psi_t = None
    if model == orc.GSC:
        mu32 = np.asarray(mu, np.float32).astype(np.float64)
        psi32 = np.asarray(psi, np.float32).astype(np.float64)
        mu_t = torch.tensor(mu32.astype(np.float32), device=dev)
        psi_t = torch.tensor(psi32.astype(np.float32), device=dev)
        kw = dict(mu=mu32, psi=psi32)
    P = ctx.params(W, theta, mu_t, psi_t)
    Yg = torch.tensor(Y32, device=dev)
    st = ctx.alloc_stats()
    ctx.estep(P, Yg, st)
    enc = ctx.encode(P, Yg)
    torch.cuda.synchronize()
    st = torch_stats_to_numpy(st)
    enc = {k: v.cpu().numpy() for k, v in enc.items()}
    sel = enc["sel"].astype(np.int32)
    n_diff, bad = check_selection(orc, model, Y32, Wt32, sel, Hp, lambda n, sc: _tau(n, sc),
                                  pi=pi, sigma=sigma, **kw)
    assert not bad, f"{len(bad)} selections not optimal within tau, e.g. {bad[:5]}"
    ref = orc.estep(model, Y32, Wt32, pi, sigma, Hp, gamma, rho=rho, sel_in=sel, **kw)
    N = len(Y32)
    assert st["scal"][orc.SC_N] == N
    assert abs(st["scal"][orc.SC_F] - ref["scal"][orc.SC_F]) <= REL_F * abs(ref["scal"][orc.SC_F]), \
        (st["scal"][orc.SC_F], ref["scal"][orc.SC_F])
    assert abs(st["scal"][orc.SC_S1] - ref["scal"][orc.SC_S1]) <= REL_AGG * max(1.0, ref["scal"][orc.SC_S1])
    assert abs(st["scal"][orc.SC_YY] - ref["scal"][orc.SC_YY]) <= 1e-6 * ref["scal"][orc.SC_YY]
    if model == orc.MCA:
        assert abs(st["scal"][orc.SC_MCA_R2] - ref["scal"][orc.SC_MCA_R2]) <= REL_AGG * ref["scal"][orc.SC_MCA_R2]
        assert relfro(st["mca"][0], ref["mca"][0]) <= REL_AGG, relfro(st["mca"][0], ref["mca"][0])
        assert relfro(st["mca"][1], ref["mca"][1]) <= REL_AGG, relfro(st["mca"][1], ref["mca"][1])
    else:
        assert relfro(st["At"], ref["At"]) <= REL_AGG, relfro(st["At"], ref["At"])
        assert relfro(st["B"], ref["B"]) <= REL_AGG, relfro(st["B"], ref["B"])
        assert relfro(st["gsc"], ref["gsc"]) <= REL_AGG, relfro(st["gsc"], ref["gsc"])
    a = (model, Y32, Wt32, pi, sigma, Hp, gamma, sel)
    check_points(orc, *a, enc["s_mean"], ref["smean"], "s_mean", **kw)
    check_points(orc, *a, enc["map_p"], ref["map_p"], "map_p", **kw)
    check_points(orc, *a, enc["logZ"], ref["logZ"], "logZ", **kw)
    if gamma > 0:
        for n in np.flatnonzero(np.any(enc["map_idx"] != ref["map_idx"], axis=1)):
            post = orc.posterior(model, Y32[n], Wt32, pi, sigma, Hp, gamma, sel_in=sel[n], **kw)
            qs = np.sort(post["q"])[::-1]
            assert qs[0] - qs[1] <= 1e-5, (n, qs[:2])
    return ctx, st, ref, (W, theta, P, mu_t, psi_t)


# ------------------------------------------------------------------- MCA
def test_mca_bars_small_n(orc):
    """MCA bars (D=10x10, H=20, intensity 8, sigma=1), H'=8, gamma=4 (163 states),
    N=1500 (ragged over the persistent warps), rho = 20."""
    d = synth.mca_bars(N=1500, seed=1003)
    # the generating bars are 0 off the bar; MCA needs W > 0 (the M-step keeps W >= 1e-6)
    run_model(orc, orc.MCA, d["Y"], d["Wt"] + 0.05, 0.1, 1.0, 8, 4, rho=20.0)
    p = synth.init_mca(d["Y"], 20, seed=2003)
    run_model(orc, orc.MCA, d["Y"], p["Wt"], p["pi"], p["sigma"], 8, 4, rho=20.0)


def test_mca_exact_small(orc):
    """Exact EM (H'=H=gamma=10) on 5x5 max-bars: 1024 states per point."""
    d = synth.mca_bars(N=200, seed=9, side=5, value=6.0)
    run_model(orc, orc.MCA, d["Y"], d["Wt"] + 0.05, 0.2, 1.0, 10, 10, rho=20.0)


def test_mca_mstep_matches_oracle(orc):
    d = synth.mca_bars(N=800, seed=1003)
    p = synth.init_mca(d["Y"], 20, seed=2003)
    ctx, st, ref, (W, theta, P, _, _) = run_model(orc, orc.MCA, d["Y"], p["Wt"], p["pi"],
                                                  p["sigma"], 8, 4, rho=20.0)
    Wt0 = W.cpu().numpy().astype(np.float64)
    st_np = dict(st)
    W2, pi2, s2, _, _ = orc.mstep(orc.MCA, 800, st_np, Wt0, p["pi"], p["sigma"])
    stg = {k: (None if v is None else torch.tensor(v, device="cuda")) for k, v in st.items()}
    ctx.mstep(stg, 800, P)
    torch.cuda.synchronize()
    assert relfro(W.cpu().numpy(), W2) <= 1e-6
    th = theta.cpu().numpy()
    assert abs(th[0] - pi2) <= 1e-9 and abs(th[1] - s2) <= 1e-7 * s2


# ------------------------------------------------------------------- GSC
def test_gsc_small_n(orc):
    """GSC (D=64, H=32, psi=0.5, sigma=0.3), H'=8, gamma=3 (93 states), N=1200."""
    d = synth.gsc(N=1200, seed=1004)
    run_model(orc, orc.GSC, d["Y"], d["Wt"], 3 / 32, 0.3, 8, 3, mu=d["mu"], psi=d["psi"])
    p = synth.init_gsc(d["Y"], 32, seed=2004)
    run_model(orc, orc.GSC, d["Y"], p["Wt"], p["pi"], p["sigma"], 8, 3, mu=p["mu"], psi=p["psi"])


@pytest.mark.parametrize("Hp,gamma", [(1, 1), (3, 3), (6, 2), (10, 3)])
def test_gsc_state_sets(orc, Hp, gamma):
    d = synth.gsc(N=300, seed=31, D=32, H=16)
    run_model(orc, orc.GSC, d["Y"], d["Wt"], 0.15, 0.3, Hp, gamma, mu=d["mu"], psi=d["psi"])


def test_gsc_mstep_matches_oracle(orc):
    d = synth.gsc(N=1000, seed=1004)
    p = synth.init_gsc(d["Y"], 32, seed=2004)
    ctx, st, ref, (W, theta, P, mu_t, psi_t) = run_model(orc, orc.GSC, d["Y"], d["Wt"], 3 / 32,
                                                         0.3, 8, 3, mu=d["mu"], psi=d["psi"])
    Wt0 = W.cpu().numpy().astype(np.float64)
    mu0 = mu_t.cpu().numpy().astype(np.float64)
    psi0 = psi_t.cpu().numpy().astype(np.float64)
    W2, pi2, s2, mu2, psi2 = orc.mstep(orc.GSC, 1000, dict(st), Wt0, 3 / 32, 0.3, mu=mu0, psi=psi0)
    stg = {k: (None if v is None else torch.tensor(v, device="cuda")) for k, v in st.items()}
    ctx.mstep(stg, 1000, P)
    torch.cuda.synchronize()
    assert relfro(W.cpu().numpy(), W2) <= 1e-6
    th = theta.cpu().numpy()
    assert abs(th[0] - pi2) <= 1e-9 and abs(th[1] - s2) <= 1e-7 * s2
    np.testing.assert_allclose(mu_t.cpu().numpy(), mu2, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(psi_t.cpu().numpy(), psi2, rtol=1e-6, atol=1e-7)
