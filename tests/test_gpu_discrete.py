"""GPU parity of the table-driven state kernel against the FP64 oracle: TSC and
DSC (Table 1 rows TSC, DSC: linear superposition, discrete latents,
categorical prior), BSC above the register kernel's Hprime range (Sec. 3:
Hprime as a free approximation parameter, here 12 and 16), MCA at Hprime = 12,
and deterministic annealing (Sec. 3, LinearAnnealing: q ~ p(s, y)^(1/T)) in
every E-step kernel.  Each case runs the CUDA path through the C ABI, feeds
the GPU's candidate sets to the oracle and compares statistics and per-point
results with the tolerances of tests/parity.py.
"""
import numpy as np
import pytest

from paper_1908_06843_gb300 import synth
from parity import REL_AGG, REL_F, check_points, check_selection, relfro, torch_stats_to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _theta(pi, sigma, rho=0.0, T=0.0, pvals=()):
    th = np.zeros(8)
    th[:4] = [pi, sigma, rho, T]
    th[4:4 + len(pvals)] = pvals
    return torch.tensor(th, dtype=torch.float64, device="cuda")


def _fp32_tau(n, sc):
    return 1e-5 * np.max(np.abs(sc)) + 1e-6


def _bf16_tau(Y, Wt):
    A = np.abs(np.asarray(Wt, np.float64))
    nrm = np.linalg.norm(np.asarray(Wt, np.float64), axis=1)

    def tau(n, sc):
        b = (A @ np.abs(np.asarray(Y[n], np.float64))) / np.where(nrm > 0, nrm, 1.0)
        return 2.0 * (2.0 ** -7) * 1.01 * np.max(b) + 1e-6
    return tau


def run_case(orc, model, Y, Wt, pi, sigma, Hp, gamma, precision=0, T=0.0, vals=None,
             pvals=None, rho=0.0, mu=None, psi=None, tau=None, check_map=True):
    """E-step + encode on the GPU, oracle E-step on the GPU's candidate sets,
    comparison of aggregates and per-point results.  Returns (ctx, stats, ref)."""
    from paper_1908_06843_gb300 import DSC, GSC, Context
    H, D = Wt.shape
    Y32 = np.asarray(Y, np.float32)
    Wt32 = np.asarray(Wt, np.float32).astype(np.float64)
    ctx = Context(model, D, H, Hp, gamma, precision, values=vals)
    dev = torch.device("cuda")
    W = torch.tensor(Wt32.astype(np.float32), device=dev)
    theta = _theta(pi, sigma, rho, T, pvals if model == DSC else ())
    mu_t = None if mu is None else torch.tensor(np.asarray(mu, np.float32), device=dev)
    psi_t = None if psi is None else torch.tensor(np.asarray(psi, np.float32), device=dev)
    P = ctx.params(W, theta, mu_t, psi_t)
    Yg = torch.tensor(Y32, device=dev)
    st = ctx.alloc_stats()
    ctx.estep(P, Yg, st)
    enc = ctx.encode(P, Yg)
    torch.cuda.synchronize()
    ctx.status()
    st = torch_stats_to_numpy(st)
    enc = {k: v.cpu().numpy() for k, v in enc.items()}
    sel = enc["sel"].astype(np.int32)
    kw = dict(T=T if T > 0 else 1.0)
    okw = {}
    if model == DSC:
        okw = dict(vals=np.asarray(vals, np.float64), pvals=np.asarray(pvals, np.float64))
    if model == GSC:
        okw = dict(mu=np.asarray(mu, np.float32).astype(np.float64),
                   psi=np.asarray(psi, np.float32).astype(np.float64))
    if rho:
        kw["rho"] = rho
    n_diff, bad = check_selection(orc, model, Y32, Wt32, sel, Hp, tau or _fp32_tau, pi=pi,
                                  sigma=sigma, **okw)
    assert not bad, f"{len(bad)} selections not optimal within tau, e.g. {bad[:5]}"
    ref = orc.estep(model, Y32, Wt32, pi, sigma, Hp, gamma, sel_in=sel, **kw, **okw)
    N = len(Y32)
    assert st["scal"][orc.SC_N] == N
    if model in (orc.MCA, orc.MMCA):   # sum <A> y and sum <A> (rho-smoothed (magnitude) max)
        assert relfro(st["mca"], ref["mca"]) <= REL_AGG, relfro(st["mca"], ref["mca"])
        assert abs(st["scal"][orc.SC_MCA_R2] - ref["scal"][orc.SC_MCA_R2]) <= \
            REL_AGG * abs(ref["scal"][orc.SC_MCA_R2])
    else:
        assert relfro(st["At"], ref["At"]) <= REL_AGG, relfro(st["At"], ref["At"])
        assert relfro(st["B"], ref["B"]) <= REL_AGG, relfro(st["B"], ref["B"])
    if model == orc.GSC:
        assert relfro(st["gsc"], ref["gsc"]) <= REL_AGG, relfro(st["gsc"], ref["gsc"])
    assert abs(st["scal"][orc.SC_F] - ref["scal"][orc.SC_F]) <= REL_F * abs(ref["scal"][orc.SC_F])
    for k in (orc.SC_S1, orc.SC_DSC0, orc.SC_DSC0 + 1, orc.SC_DSC0 + 2):
        assert abs(st["scal"][k] - ref["scal"][k]) <= REL_AGG * max(1.0, abs(ref["scal"][k])), k
    scale = float(np.max(np.abs(ctx.values)))
    a = (orc, model, Y32, Wt32, pi, sigma, Hp, gamma, sel)
    check_points(*a, enc["s_mean"], ref["smean"], "s_mean", scale=scale, **kw, **okw)
    check_points(*a, enc["map_p"], ref["map_p"], "map_p", **kw, **okw)
    check_points(*a, enc["logZ"], ref["logZ"], "logZ", **kw, **okw)
    if gamma > 0 and check_map:
        same = np.all(enc["map_idx"] == ref["map_idx"], axis=1)
        if "map_val" in enc:
            same &= np.all(enc["map_val"] == ref["map_val"], axis=1)
        for n in np.flatnonzero(~same):   # MAP may differ only at (near-)ties of the log-joint
            post = orc.posterior(model, Y32[n], Wt32, pi, sigma, Hp, gamma, sel_in=sel[n], **kw, **okw)
            qs = np.sort(post["q"])[::-1]
            assert qs[0] - qs[1] <= 1e-5, (n, qs[:2])
    return ctx, st, ref, (W, theta, P)


# ------------------------------------------------------------------- TSC/DSC
def test_tsc_gabor(orc):
    """TSC on Gabor-dictionary data (D = 256, H = 64, latents -1/0/+1 with
    p = 2/64 each), H' = 8, gamma = 3 (577 states), N = 2,050 (ragged tail)."""
    d = synth.discrete(N=2050, seed=1006)
    run_case(orc, orc.TSC, d["Y"], d["Wt"], 4 / 64, 0.2, 8, 3)


def test_dsc_three_values(orc):
    """DSC with values {0.5, 2, -1.5} (m = 3), H' = 6, gamma = 3 (694 states)."""
    vals, pv = (0.5, 2.0, -1.5), (0.02, 0.01, 0.015)
    d = synth.discrete(N=1500, seed=1007, H=48, vals=vals, pvals=pv, sigma=0.3)
    run_case(orc, orc.DSC, d["Y"], d["Wt"], sum(pv), 0.3, 6, 3, vals=vals, pvals=pv)


def test_dsc_positive_values_signed_selection(orc):
    """DSC with positive values only ({1, 3}): the signed score selects."""
    vals, pv = (1.0, 3.0), (0.03, 0.01)
    d = synth.discrete(N=700, seed=1008, H=40, vals=vals, pvals=pv, sigma=0.25)
    run_case(orc, orc.DSC, d["Y"], d["Wt"], sum(pv), 0.25, 7, 2, vals=vals, pvals=pv)


@pytest.mark.parametrize("Hp,gamma,N", [(1, 0, 65), (1, 1, 129), (5, 5, 300), (16, 2, 257)])
def test_tsc_degenerate_and_wide_state_sets(orc, Hp, gamma, N):
    """gamma = 0 (only s = 0), H' = 1, H' = gamma (all 3^5 patterns), H' = 16."""
    d = synth.discrete(N=N, seed=1009 + Hp, H=32)
    run_case(orc, orc.TSC, d["Y"], d["Wt"], 4 / 32, 0.2, Hp, gamma)


def test_tsc_and_dsc_msteps_match_oracle(orc):
    """FP64 M-steps of TSC and DSC (W = A B^-1, sigma, prior) on the GPU's own
    statistics equal the oracle's M-step on the same statistics."""
    for model, vals, pv in [(orc.TSC, None, None), (orc.DSC, (0.5, 2.0, -1.5), (0.02, 0.01, 0.015))]:
        d = synth.discrete(N=3000, seed=1010, H=48, vals=vals or (-1.0, 1.0),
                           pvals=pv or (1 / 48, 1 / 48), sigma=0.3)
        pi = sum(pv) if pv else 2 / 48
        ctx, st, _, (W, theta, P) = run_case(orc, model, d["Y"], d["Wt"], pi, 0.3, 6, 2,
                                             vals=vals, pvals=pv)
        Wt0 = W.cpu().numpy().astype(np.float64)
        W2, pi2, s2, p2 = orc.mstep_dsc(model, 3000, st, Wt0, pi, 0.3,
                                        vals=None if vals is None else np.array(vals),
                                        pvals=None if pv is None else np.array(pv))
        stg = {k: (None if v is None else torch.tensor(v, device="cuda")) for k, v in st.items()}
        ctx.mstep(stg, 3000, P)
        torch.cuda.synchronize()
        ctx.status()
        assert relfro(W.cpu().numpy(), W2) <= 1e-6
        th = theta.cpu().numpy()
        assert abs(th[0] - pi2) <= 1e-9 and abs(th[1] - s2) <= 1e-7 * s2
        if model == orc.DSC:
            np.testing.assert_allclose(th[4:7], p2, rtol=1e-9)


# ------------------------------------------------------- BSC with Hprime > 10
@pytest.mark.parametrize("Hp,gamma", [(12, 4), (12, 5), (16, 4)])
@pytest.mark.parametrize("precision", [0, 1])
def test_bsc_wide_candidate_sets(orc, Hp, gamma, precision):
    """BSC at H' = 12 (gamma 4, 5: 794 / 1586 states) and H' = 16 (gamma 4:
    2,517 states) on the Gabor shape, both preselection forms, N = 1,100."""
    d = synth.gabor(N=1100, seed=1011)
    Wt = d["Wt"].astype(np.float32).astype(np.float64)
    tau = _bf16_tau(d["Y"], Wt) if precision else None
    run_case(orc, orc.BSC, d["Y"], Wt, 4 / 256, 0.2, Hp, gamma, precision=precision, tau=tau)


def test_bsc_table_kernel_equals_register_kernel(orc):
    """At H' = 10 the table-driven kernel (DSC with the single value 1) and the
    register-resident BSC kernel give the same posterior (FP32 tolerance)."""
    from paper_1908_06843_gb300 import BSC, DSC, Context
    d = synth.gabor(N=1000, seed=1012, H=64)
    dev = torch.device("cuda")
    W = torch.tensor(d["Wt"].astype(np.float32), device=dev)
    Y = torch.tensor(d["Y"], device=dev)
    a = Context(BSC, 256, 64, 10, 5)
    b = Context(DSC, 256, 64, 10, 5, values=[1.0])
    ea = a.encode(a.params(W, _theta(0.05, 0.2)), Y)
    eb = b.encode(b.params(W, _theta(0.05, 0.2, pvals=(0.05,))), Y)
    torch.cuda.synchronize()
    assert torch.equal(ea["sel"], eb["sel"])
    assert float((ea["s_mean"] - eb["s_mean"]).abs().max()) <= 2e-5
    assert float((ea["logZ"] - eb["logZ"]).abs().max()) <= 1e-4 * float(ea["logZ"].abs().max())


# ------------------------------------------------------------- MCA Hprime 12
def test_mca_wide_candidate_set(orc):
    """MCA bars (D = 100, H = 20) at H' = 12, gamma = 3 (299 states)."""
    d = synth.mca_bars(N=600, seed=1013)
    Wt = d["Wt"] + 0.05
    run_case(orc, orc.MCA, d["Y"], Wt, 0.1, 1.0, 12, 3, rho=20.0)


def test_mca_selection_golden_on_gpu(orc):
    """The hand-worked MCA preselection case (tests/golden/mca_selection.txt)
    on the GPU: the same candidate sets, ties to the lower h."""
    from test_oracle_pins import read_mca_selection_golden
    from paper_1908_06843_gb300 import MCA, Context
    Wt, y, _, sel = read_mca_selection_golden()
    for Hp, want in sel.items():
        ctx = Context(MCA, Wt.shape[1], Wt.shape[0], Hp, 1)
        P = ctx.params(torch.tensor(Wt.astype(np.float32), device="cuda"), _theta(0.2, 1.0, 20.0))
        out = ctx.encode(P, torch.tensor(y[None, :].astype(np.float32), device="cuda"))
        torch.cuda.synchronize()
        assert out["sel"].cpu().numpy()[0].tolist() == want, (Hp, want)


# ---------------------------------------------------------------------- MMCA
def test_mmca_signed_bars(orc):
    """MMCA (Table 1 row MMCA: |max| superposition) on signed bars (D = 100,
    H = 20), H' = 8, gamma = 4 (163 states), N = 1,500: statistics, per-point
    results and the M-step (no positivity clamp) against the oracle."""
    d = synth.mmca_bars(N=1500, seed=1019)
    ctx, st, ref, (W, theta, P) = run_case(orc, orc.MMCA, d["Y"], d["Wt"], 0.1, 1.0, 8, 4, rho=20.0)
    Wt0 = W.cpu().numpy().astype(np.float64)
    W2 = orc.mstep(orc.MMCA, 1500, st, Wt0, 0.1, 1.0)[0]
    stg = {k: (None if v is None else torch.tensor(v, device="cuda")) for k, v in st.items()}
    ctx.mstep(stg, 1500, P)
    torch.cuda.synchronize()
    Wg = W.cpu().numpy()
    assert relfro(Wg, W2) <= REL_AGG and np.any(Wg < 0)


def test_mmca_wide_and_annealed(orc):
    d = synth.mmca_bars(N=600, seed=1020)
    run_case(orc, orc.MMCA, d["Y"], d["Wt"], 0.1, 1.0, 12, 3, rho=20.0)
    run_case(orc, orc.MMCA, d["Y"], d["Wt"], 0.1, 1.0, 8, 3, rho=20.0, T=2.0)


# -------------------------------------------------------------- annealing T
@pytest.mark.parametrize("T", [0.6, 3.0])
def test_annealed_estep_bsc(orc, T):
    """BSC E-step at temperature T: register kernel (H' = 10) and table kernel
    (H' = 12) against the oracle's tempered posterior."""
    d = synth.gabor(N=900, seed=1014)
    Wt = d["Wt"].astype(np.float32).astype(np.float64)
    run_case(orc, orc.BSC, d["Y"], Wt, 4 / 256, 0.2, 10, 5, T=T)
    run_case(orc, orc.BSC, d["Y"], Wt, 4 / 256, 0.2, 12, 3, T=T)


def test_annealed_estep_mca_gsc_tsc(orc):
    d = synth.mca_bars(N=500, seed=1015)
    run_case(orc, orc.MCA, d["Y"], d["Wt"] + 0.05, 0.1, 1.0, 8, 4, rho=20.0, T=2.0)
    g = synth.gsc(N=600, seed=1016)
    run_case(orc, orc.GSC, g["Y"], g["Wt"], 3 / 32, 0.3, 8, 3, T=2.0, mu=g["mu"], psi=g["psi"])
    t = synth.discrete(N=600, seed=1017, H=32)
    run_case(orc, orc.TSC, t["Y"], t["Wt"], 4 / 32, 0.2, 8, 3, T=1.7)


def test_annealing_schedule_runs_through_em():
    """EM.run under LinearAnnealing(T0 = 4): the E-steps see the scheduled T
    (the last iterations run at T = 1, so F then equals the plain E-step's)."""
    from paper_1908_06843_gb300 import BSC_ET, EM, LinearAnnealing
    d = synth.bars(N=400, seed=1018)
    model = BSC_ET(25, 10, 6, 3)
    anneal = LinearAnnealing(8, T0=4.0, anneal_steps=4)
    params = model.standard_init({"y": d["Y"]})
    em = EM(model=model, anneal=anneal, data={"y": d["Y"]}, lparams=params)
    em.run()
    assert len(em.history) == 8 and np.all(np.isfinite(em.history))
    assert float(params["theta"][3]) == 1.0
    F_plain = model.free_energy(params, {"y": d["Y"]})
    assert np.isfinite(F_plain)
