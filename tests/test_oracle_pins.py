"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check uses an independent
route (a library Gaussian density over all 2^H states, a closed form, an
invariant, a limit that reduces to another model, stationarity of the
expected log-joint by finite differences, EM monotonicity, recovery of
planted bars), chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.

Models: Eq. 1-2 and Table 1 (rows BSC, GSC, MCA) of the paper; truncated
posteriors and EM (Sec. 2); the Hprime / gamma approximation parameters and
the step / inference API (Sec. 3).
"""
import itertools
import os

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment
from scipy.special import expit, logsumexp
from scipy.stats import multivariate_normal

from paper_1908_06843_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_states(H):
    return np.array(list(itertools.product([0, 1], repeat=H)), dtype=np.float64)


def brute_logjoint_bsc(y, Wt, pi, sigma):
    """log p(s, y) for every s in {0,1}^H, via scipy's Gaussian density."""
    H, D = Wt.shape
    S = all_states(H)
    k = S.sum(1)
    lp = k * np.log(pi) + (H - k) * np.log(1 - pi)
    ll = multivariate_normal(mean=np.zeros(D), cov=sigma ** 2 * np.eye(D)).logpdf(y[None, :] - S @ Wt)
    return S, lp + ll


def brute_logjoint_mca(y, Wt, pi, sigma):
    H, D = Wt.shape
    S = all_states(H)
    k = S.sum(1)
    lp = k * np.log(pi) + (H - k) * np.log(1 - pi)
    F = np.max(S[:, :, None] * Wt[None, :, :], axis=1)       # W >= 0: max_h W_dh s_h
    ll = multivariate_normal(mean=np.zeros(D), cov=sigma ** 2 * np.eye(D)).logpdf(y[None, :] - F)
    return S, lp + ll


def brute_logjoint_gsc(y, Wt, pi, sigma, mu, psi):
    H, D = Wt.shape
    S = all_states(H)
    out = []
    for b in S:
        act = b > 0
        Wb = Wt[act].T
        cov = sigma ** 2 * np.eye(D) + Wb @ np.diag(psi[act]) @ Wb.T
        mean = Wb @ mu[act]
        k = act.sum()
        out.append(k * np.log(pi) + (H - k) * np.log(1 - pi)
                   + multivariate_normal(mean=mean, cov=cov).logpdf(y))
    return S, np.array(out)


def state_vectors(post, H):
    """Global binary vectors of the oracle's states (masks over local units)."""
    sel = post["sel"]
    V = np.zeros((len(post["masks"]), H))
    for i, m in enumerate(post["masks"]):
        for j in range(len(sel)):
            if (int(m) >> j) & 1:
                V[i, sel[j]] = 1
    return V


def match_states(V, S):
    key = {tuple(s.astype(int)): i for i, s in enumerate(S)}
    return np.array([key[tuple(v.astype(int))] for v in V])


# ---------------------------------------------------------------------------
# state set K (Sec. 3: Hprime, gamma)
# ---------------------------------------------------------------------------
def test_state_counts_golden(orc):
    """|K| = sum_{k <= gamma} C(H', k); the golden table lists the counts by hand."""
    path = os.path.join(GOLDEN, "state_counts.txt")
    rows = [l.split("#")[0].split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 5
    for hp, g, n in rows:
        assert orc.num_states(int(hp), int(g)) == int(n)


def test_state_order_is_canonical(orc):
    """By cardinality, then lexicographic (itertools.combinations order)."""
    for hp, g in [(6, 3), (10, 5), (8, 4), (5, 5)]:
        masks = orc.states(hp, g)
        expect = []
        for k in range(g + 1):
            for c in itertools.combinations(range(hp), k):
                expect.append(sum(1 << j for j in c))
        assert list(masks) == expect


# ---------------------------------------------------------------------------
# BSC
# ---------------------------------------------------------------------------
def _small_bsc(seed, H=6, D=9, N=1):
    g = synth.rng(seed)
    Wt = g.standard_normal((H, D))
    Y = g.standard_normal((N, D)) + (g.random((N, H)) < 0.3) @ Wt
    return Y, Wt


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bsc_exact_equals_bruteforce(orc, seed):
    """ET with H' = H = gamma is exact EM: posterior and log p(y) equal the
    brute-force sum over all 2^H states computed with scipy's Gaussian density."""
    Y, Wt = _small_bsc(seed)
    H = Wt.shape[0]
    pi, sigma = 0.3, 0.8
    for y in Y:
        post = orc.posterior(orc.BSC, y, Wt, pi, sigma, H, H)
        S, lj = brute_logjoint_bsc(y, Wt, pi, sigma)
        idx = match_states(state_vectors(post, H), S)
        np.testing.assert_allclose(post["ell"], lj[idx], rtol=1e-12, atol=1e-10)
        q = np.exp(lj - logsumexp(lj))
        np.testing.assert_allclose(post["q"], q[idx], rtol=1e-10, atol=1e-14)
        assert abs(post["q"].sum() - 1.0) < 1e-12
    out = orc.estep(orc.BSC, Y, Wt, pi, sigma, H, H)
    S, lj = brute_logjoint_bsc(Y[0], Wt, pi, sigma)
    assert abs(out["logZ"][0] - logsumexp(lj)) < 1e-10


def test_bsc_single_latent_logistic(orc):
    """H = 1: q(s=1|y) = logistic(log(pi/(1-pi)) + (w.y - |w|^2/2)/sigma^2)."""
    g = synth.rng(5)
    for _ in range(5):
        D = 7
        w = g.standard_normal(D)
        y = g.standard_normal(D) + w
        pi, sigma = g.uniform(0.05, 0.9), g.uniform(0.3, 2.0)
        post = orc.posterior(orc.BSC, y, w[None, :], pi, sigma, 1, 1)
        expect = expit(np.log(pi / (1 - pi)) + (w @ y - 0.5 * w @ w) / sigma ** 2)
        assert abs(post["q"][1] - expect) < 1e-13
        assert abs(post["q"][0] - (1 - expect)) < 1e-13


# ---------------------------------------------------------------------------
# Deterministic annealing (Sec. 3, LinearAnnealing): q_T(s) ~ p(s, y)^(1/T)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T", [0.4, 2.5])
@pytest.mark.parametrize("model", ["BSC", "MCA", "GSC"])
def test_tempered_posterior_equals_bruteforce(orc, model, T):
    """At temperature T and H' = H = gamma the oracle's posterior is the
    softmax of log p(s, y)/T over all 2^H states and its per-point free energy
    is T logsumexp(log p(s, y)/T), with log p(s, y) from scipy's densities."""
    if model == "GSC":
        Y, Wt, mu, psi = _small_gsc(3)
        kw = dict(mu=mu, psi=psi)
        brute = lambda y: brute_logjoint_gsc(y, Wt, 0.3, 0.6, mu, psi)
    elif model == "MCA":
        Y, Wt = _small_mca(3)
        kw = dict(rho=20)
        brute = lambda y: brute_logjoint_mca(y, Wt, 0.3, 0.6)
    else:
        Y, Wt = _small_bsc(3)
        kw = {}
        brute = lambda y: brute_logjoint_bsc(y, Wt, 0.3, 0.6)
    m = getattr(orc, model)
    H = Wt.shape[0]
    for y in Y:
        post = orc.posterior(m, y, Wt, 0.3, 0.6, H, H, T=T, **kw)
        S, lj = brute(y)
        idx = match_states(state_vectors(post, H), S)
        np.testing.assert_allclose(post["q"], np.exp(lj / T - logsumexp(lj / T))[idx],
                                   rtol=1e-10, atol=1e-14)
    out = orc.estep(m, Y, Wt, 0.3, 0.6, H, H, T=T, **kw)
    for n, y in enumerate(Y):
        S, lj = brute(y)
        assert abs(out["logZ"][n] - T * logsumexp(lj / T)) < 1e-9 * max(1.0, abs(out["logZ"][n]))


def test_tempered_free_energy_is_the_variational_optimum(orc):
    """For the truncated set K_n, T log sum_K p(s,y)^(1/T) = sum_K q_T log p(s,y)
    + T H[q_T] (the maximum over q on K_n of E_q log p + T H[q], attained at
    q_T); checked with ET (H' < H) at several T, including T = 1."""
    Y, Wt = _small_bsc(4, H=8, D=9, N=4)
    for T in (0.3, 1.0, 4.0):
        out = orc.estep(orc.BSC, Y, Wt, 0.2, 0.7, 5, 3, T=T)
        for n, y in enumerate(Y):
            post = orc.posterior(orc.BSC, y, Wt, 0.2, 0.7, 5, 3, T=T)
            q = post["q"]
            ent = -np.sum(q[q > 0] * np.log(q[q > 0]))
            assert abs(out["logZ"][n] - (q @ post["ell"] + T * ent)) < 1e-10 * max(1, abs(out["logZ"][n]))


def test_high_temperature_gives_uniform_posterior(orc):
    """T -> infinity: q_T -> uniform over the truncated set K_n."""
    Y, Wt = _small_bsc(5, H=8, D=9, N=2)
    post = orc.posterior(orc.BSC, Y[0], Wt, 0.2, 0.7, 6, 3, T=1e9)
    np.testing.assert_allclose(post["q"], 1.0 / len(post["q"]), rtol=1e-6)


def test_bsc_aggregates_are_scatter_of_point_moments(orc):
    """At = sum_n <s>_n y_n^T and diag(B) = sum_n <s_h>_n (binary s: s_h^2 = s_h),
    B symmetric, sum<|s|> = sum of <s>, F = sum log Z."""
    Y, Wt = _small_bsc(11, H=8, D=10, N=40)
    H, D = Wt.shape
    out = orc.estep(orc.BSC, Y, Wt, 0.25, 0.9, 4, 2)
    At = np.zeros((H, D))
    es = np.zeros(H)
    for n in range(len(Y)):
        for j, h in enumerate(out["sel"][n]):
            At[h] += out["smean"][n, j] * Y[n]
            es[h] += out["smean"][n, j]
    np.testing.assert_allclose(out["At"], At, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.diag(out["B"]), es, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["B"], out["B"].T, atol=1e-12)
    assert abs(out["scal"][orc.SC_S1] - es.sum()) < 1e-9
    assert abs(out["scal"][orc.SC_F] - out["logZ"].sum()) < 1e-9
    assert abs(out["scal"][orc.SC_YY] - (Y.astype(np.float64) ** 2).sum()) < 1e-9


def test_preselection_known_answer(orc):
    """Scores W_h.y/|W_h| with a planted exact tie: the lower index wins, and
    the selection is returned in ascending order."""
    Wt = np.eye(8) * np.array([1.0, 2.0, 0.5, 1.0, 3.0, 1.0, 1.0, 1.0])[:, None]
    y = np.array([5.0, 3.0, 3.0, 1.0, 0.0, -2.0, 4.0, 0.5])
    sc = orc.scores(orc.BSC, y, Wt)
    np.testing.assert_allclose(sc, y, atol=1e-15)          # |W_h| cancels
    post = orc.posterior(orc.BSC, y, Wt, 0.2, 1.0, 3, 1)
    assert list(post["sel"]) == [0, 1, 6]                  # 5, 4, and 3 (tie 1 vs 2 -> 1)
    post = orc.posterior(orc.BSC, y, Wt, 0.2, 1.0, 5, 1)
    assert list(post["sel"]) == [0, 1, 2, 3, 6]


def test_map_is_first_maximum(orc):
    """MAP tie-break: two identical dictionary rows give equal log-joints; the
    state earlier in canonical order (lower local index) wins."""
    w = np.array([1.0, 2.0, -1.0])
    Wt = np.stack([w, w, -w])
    y = 1.0 * w
    out = orc.estep(orc.BSC, y[None, :], Wt, 0.3, 0.5, 3, 1)
    assert list(out["map_idx"][0]) == [0]


def _Q_bsc(posts, Y, Wt, pi, sigma):
    """Expected log-joint sum_n sum_s q_n(s) log p(s, y_n | W, pi, sigma)."""
    H, D = Wt.shape
    Q = 0.0
    for post, y in zip(posts, Y):
        V = state_vectors(post, H)
        k = V.sum(1)
        r2 = ((y[None, :] - V @ Wt) ** 2).sum(1)
        lj = k * np.log(pi) + (H - k) * np.log(1 - pi) - 0.5 * D * np.log(2 * np.pi * sigma ** 2) \
            - r2 / (2 * sigma ** 2)
        Q += post["q"] @ lj
    return Q


def test_bsc_mstep_is_stationary_point_of_Q(orc):
    """The M-step output zeroes the gradient of Q (central differences; Q is
    evaluated from the E-step's truncated posteriors with an independent
    residual formula)."""
    d = synth.bars(N=60, seed=3, side=3, value=3.0)
    Y = d["Y"].astype(np.float64)
    g = synth.rng(9)
    Wt = d["Wt"] + 0.5 * g.standard_normal(d["Wt"].shape)
    pi, sigma, Hp, gam = 0.3, 1.2, 4, 2
    out = orc.estep(orc.BSC, Y, Wt, pi, sigma, Hp, gam)
    posts = [orc.posterior(orc.BSC, y, Wt, pi, sigma, Hp, gam) for y in Y]
    W2, pi2, s2, _, _ = orc.mstep(orc.BSC, len(Y), out, Wt, pi, sigma)
    eps = 1e-5
    base = _Q_bsc(posts, Y, W2, pi2, s2)
    for (h, dd) in [(0, 0), (1, 4), (5, 8), (3, 2)]:
        Wp, Wm = W2.copy(), W2.copy()
        Wp[h, dd] += eps
        Wm[h, dd] -= eps
        grad = (_Q_bsc(posts, Y, Wp, pi2, s2) - _Q_bsc(posts, Y, Wm, pi2, s2)) / (2 * eps)
        assert abs(grad) < 1e-5 * abs(base) / len(Y), (h, dd, grad)
    gpi = (_Q_bsc(posts, Y, W2, pi2 + eps, s2) - _Q_bsc(posts, Y, W2, pi2 - eps, s2)) / (2 * eps)
    gs = (_Q_bsc(posts, Y, W2, pi2, s2 + eps) - _Q_bsc(posts, Y, W2, pi2, s2 - eps)) / (2 * eps)
    assert abs(gpi) < 1e-4 and abs(gs) < 1e-4, (gpi, gs)
    # a perturbed parameter is strictly worse (it is a maximum, not a saddle)
    assert _Q_bsc(posts, Y, W2 * 1.01, pi2, s2) < base
    assert _Q_bsc(posts, Y, W2, pi2, s2 * 1.05) < base


def test_bsc_exact_em_monotone(orc):
    """Exact EM (H' = H = gamma): the log-likelihood never decreases."""
    d = synth.bars(N=200, seed=4, side=3, value=4.0)
    Y = d["Y"]
    p = synth.init_bsc(Y, 6, seed=77, pi=0.5, normalise=False)
    Wt, pi, sigma = p["Wt"], p["pi"], p["sigma"]
    F_prev = -np.inf
    for it in range(15):
        out = orc.estep(orc.BSC, Y, Wt, pi, sigma, 6, 6)
        F = out["scal"][orc.SC_F]
        assert F >= F_prev - 1e-9 * abs(F), (it, F, F_prev)
        F_prev = F
        Wt, pi, sigma, _, _ = orc.mstep(orc.BSC, len(Y), out, Wt, pi, sigma)


def _bars_recovered(Wt_learned, Wt_true, thr=0.95):
    a = Wt_learned - Wt_learned.mean(1, keepdims=True)
    b = Wt_true - Wt_true.mean(1, keepdims=True)
    C = (b / np.linalg.norm(b, axis=1, keepdims=True)) @ (a / (np.linalg.norm(a, axis=1, keepdims=True) + 1e-30)).T
    r, c = linear_sum_assignment(-C)
    return bool(np.all(C[r, c] > thr))


def test_bars_recovery_rate(orc):
    """Bars test (D = 5x5, H = 10, pi = 0.2, sigma = 1, N = 1000; ET H' = 6,
    gamma = 3; 50 iterations from W ~ N(0, 1), pi = 0.5, sigma = std(Y)):
    every true bar matched with correlation > 0.95 in at least 7 of 10 runs."""
    hits = 0
    for r in range(10):
        d = synth.bars(N=1000, seed=1001 + 100 * r)
        p = synth.init_bsc(d["Y"], 10, seed=2001 + 100 * r, pi=0.5, normalise=False)
        Wt, pi, sigma = p["Wt"], p["pi"], p["sigma"]
        for _ in range(50):
            out = orc.estep(orc.BSC, d["Y"], Wt, pi, sigma, 6, 3)
            Wt, pi, sigma, _, _ = orc.mstep(orc.BSC, 1000, out, Wt, pi, sigma)
        hits += _bars_recovered(Wt, d["Wt"])
    assert hits >= 7, hits


# ---------------------------------------------------------------------------
# MCA
# ---------------------------------------------------------------------------
def _small_mca(seed, H=6, D=9, N=3):
    g = synth.rng(seed)
    Wt = np.abs(g.standard_normal((H, D))) * 2 + 0.1
    S = (g.random((N, H)) < 0.3).astype(float)
    Y = np.max(S[:, :, None] * Wt[None], axis=1) + g.standard_normal((N, D))
    return Y, Wt


@pytest.mark.parametrize("seed", [0, 1])
def test_mca_exact_equals_bruteforce(orc, seed):
    Y, Wt = _small_mca(seed)
    H = Wt.shape[0]
    for y in Y:
        post = orc.posterior(orc.MCA, y, Wt, 0.3, 0.9, H, H, rho=20)
        S, lj = brute_logjoint_mca(y, Wt, 0.3, 0.9)
        idx = match_states(state_vectors(post, H), S)
        np.testing.assert_allclose(post["ell"], lj[idx], rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(post["q"], np.exp(lj - logsumexp(lj))[idx], rtol=1e-10, atol=1e-14)


def test_mca_gamma1_equals_bsc_gamma1(orc):
    """With at most one active unit, max superposition equals linear
    superposition: the posteriors of MCA and BSC coincide on the same set."""
    Y, Wt = _small_mca(3, N=10)
    sel = np.tile(np.array([0, 2, 3, 5], np.int32), (len(Y), 1))
    a = orc.estep(orc.MCA, Y, Wt, 0.2, 1.1, 4, 1, rho=20, sel_in=sel)
    b = orc.estep(orc.BSC, Y, Wt, 0.2, 1.1, 4, 1, sel_in=sel)
    np.testing.assert_allclose(a["smean"], b["smean"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(a["logZ"], b["logZ"], rtol=1e-12)


def test_mca_mstep_gamma1_closed_form(orc):
    """gamma = 1: A_dh(s) = s_h exactly, so W_dh = sum<s_h> y_d / sum<s_h>;
    sigma^2 = <||y - f||^2>/(N D) with f = W_h for the single active unit."""
    Y, Wt = _small_mca(4, N=30)
    H, D = Wt.shape
    out = orc.estep(orc.MCA, Y, Wt, 0.2, 1.1, H, 1, rho=20)
    num = np.zeros((H, D))
    den = np.zeros(H)
    r2 = 0.0
    for n, y in enumerate(Y):
        post = orc.posterior(orc.MCA, y, Wt, 0.2, 1.1, H, 1, rho=20)
        V = state_vectors(post, H)
        for q, v in zip(post["q"], V):
            f = v @ Wt
            r2 += q * ((y - f) ** 2).sum()
            num += q * v[:, None] * y[None, :]
            den += q * v
    W2, pi2, s2, _, _ = orc.mstep(orc.MCA, len(Y), out, Wt, 0.2, 1.1)
    np.testing.assert_allclose(W2, np.maximum(num / den[:, None], 1e-6), rtol=1e-10)
    assert abs(s2 ** 2 - r2 / (len(Y) * D)) < 1e-10
    assert abs(pi2 - den.sum() / (len(Y) * H)) < 1e-12


def test_mca_mstep_large_rho_is_hard_argmax(orc):
    """rho -> infinity: A_dh(s) -> 1 for the unit that attains the max at pixel
    d and 0 for the others, so the update tends to the hard-argmax average."""
    Y, Wt = _small_mca(6, H=5, D=6, N=25)
    H, D = Wt.shape
    rho = 3000.0
    out = orc.estep(orc.MCA, Y, Wt, 0.3, 1.0, H, 3, rho=rho)
    num = np.zeros((H, D))
    den = np.zeros((H, D))
    for y in Y:
        post = orc.posterior(orc.MCA, y, Wt, 0.3, 1.0, H, 3, rho=rho)
        for q, v in zip(post["q"], state_vectors(post, H)):
            if v.sum() == 0:
                continue
            act = np.flatnonzero(v)
            win = act[np.argmax(Wt[act], axis=0)]            # per pixel
            for d in range(D):
                num[win[d], d] += q * y[d]
                den[win[d], d] += q
    W2, _, _, _, _ = orc.mstep(orc.MCA, len(Y), out, Wt, 0.3, 1.0)
    m = den > 1e-3
    np.testing.assert_allclose(W2[m], np.maximum(num[m] / den[m], 1e-6), rtol=2e-3)


def read_mca_selection_golden():
    """The hand-worked MCA preselection case of tests/golden/mca_selection.txt."""
    W, y, score, sel = [], None, None, {}
    with open(os.path.join(GOLDEN, "mca_selection.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "W":
                W.append([float(v) for v in t[1:]])
            elif t[0] == "y":
                y = np.array([float(v) for v in t[1:]])
            elif t[0] == "score":
                score = np.array([float(v) for v in t[1:]])
            elif t[0] == "sel":
                sel[int(t[1])] = [int(v) for v in t[2:]]
    return np.array(W), y, score, sel


def test_mca_selection_known_answer(orc):
    """MCA preselection (Table 1 MCA row; score S_h = sum_d W_dh y_d / sum_d W_dh,
    ties to the lower h) against scores and candidate sets worked by hand, with
    three exactly tied scores.  A wrong normaliser (L2 norm, none) or the
    reversed tie rule selects a different set at Hprime = 2."""
    Wt, y, score, sel = read_mca_selection_golden()
    H = Wt.shape[0]
    got = orc.scores(orc.MCA, y, Wt)
    np.testing.assert_array_equal(got, score)      # exact: every value is a dyadic fraction
    for Hp, want in sel.items():
        post = orc.posterior(orc.MCA, y, Wt, 0.2, 1.0, Hp, 1, rho=20)
        assert post["sel"].tolist() == want, (Hp, post["sel"], want)
    # the sets the wrong readings would give differ from the golden one
    l2 = (Wt @ y) / np.linalg.norm(Wt, axis=1)
    assert sorted(np.lexsort((np.arange(H), -l2))[:2].tolist()) != sel[2]
    raw = Wt @ y
    assert sorted(np.lexsort((np.arange(H), -raw))[:2].tolist()) != sel[2]


# ---------------------------------------------------------------------------
# ET data-point cut (N_cut and the pi correction; reading, see the oracle)
# ---------------------------------------------------------------------------
def test_cut_size_is_binomial_cdf(orc):
    from scipy.stats import binom
    for H, gamma, pi in [(10, 3, 0.2), (256, 5, 4 / 256), (20, 0, 0.1), (8, 8, 0.4)]:
        P = orc.trunc_prob(H, gamma, pi)
        assert abs(P - binom.cdf(gamma, H, pi)) < 1e-12
        assert orc.cut_size(100_000, H, gamma, pi) == int(np.floor(100_000 * P))


def test_pi_correction_bruteforce(orc):
    """E_pi[|s| : |s| <= gamma] by enumerating all 2^H binary states."""
    H, pi = 9, 0.27
    S = all_states(H)
    k = S.sum(1)
    p = pi ** k * (1 - pi) ** (H - k)
    for gamma in (0, 2, 4, 9):
        if gamma == 0:
            continue            # E[|s| : |s| = 0] = 0: no correction defined
        m = (k[k <= gamma] * p[k <= gamma]).sum() / p[k <= gamma].sum()
        assert abs(orc.pi_correction(H, gamma, pi) - (H * pi / m if gamma < H else 1.0)) < 1e-12
    # fixed point: a kept set with exactly the truncated prior's mean restores pi
    m = (k[k <= 3] * p[k <= 3]).sum() / p[k <= 3].sum()
    assert abs(m / H * orc.pi_correction(H, 3, pi) - pi) < 1e-14


def test_cut_keeps_the_best_explained_points(orc):
    g = synth.rng(61)
    lz = g.standard_normal(500)
    keep = orc.cut_keep(lz, 123)
    assert keep.sum() == 123 and lz[keep].min() >= lz[~keep].max()
    lz[[3, 7, 11]] = np.sort(lz)[::-1][122]      # a three-way tie at the boundary: all kept
    keep = orc.cut_keep(lz, 123)
    assert keep[[3, 7, 11]].all() and lz[keep].min() >= lz[~keep].max()


def test_cut_without_truncation_is_the_plain_estep(orc):
    """gamma = H' = H: K_n holds every pattern, N_cut = N, nothing is cut."""
    Y, Wt = _small_bsc(12, H=6, D=9, N=20)
    sub, keep, ncut = orc.estep_cut(orc.BSC, Y, Wt, 0.3, 0.8, 6, 6)
    full = orc.estep(orc.BSC, Y, Wt, 0.3, 0.8, 6, 6)
    assert ncut == 20 and keep.all()
    np.testing.assert_allclose(sub["At"], full["At"], rtol=1e-13)
    np.testing.assert_allclose(sub["scal"], full["scal"], rtol=1e-13)
    assert orc.pi_correction(6, 6, 0.3) == 1.0


# ---------------------------------------------------------------------------
# MMCA (Table 1: |max| superposition, signed dictionary, binary latents)
# ---------------------------------------------------------------------------
def brute_logjoint_mmca(y, Wt, pi, sigma):
    """log p(s, y) over {0,1}^H: per pixel the active W_dh of largest |W_dh|
    (first in unit order on a tie), scipy's Gaussian density."""
    H, D = Wt.shape
    S = all_states(H)
    k = S.sum(1)
    lp = k * np.log(pi) + (H - k) * np.log(1 - pi)
    F = np.zeros((len(S), D))
    for i, s_ in enumerate(S):
        act = np.flatnonzero(s_)
        if len(act):
            win = act[np.argmax(np.abs(Wt[act]), axis=0)]      # argmax takes the first on ties
            F[i] = Wt[win, np.arange(D)]
    ll = multivariate_normal(mean=np.zeros(D), cov=sigma ** 2 * np.eye(D)).logpdf(y[None, :] - F)
    return S, lp + ll


def _small_mmca(seed, H=6, D=7, N=3):
    g = synth.rng(seed)
    Wt = g.standard_normal((H, D)) * 2.0
    S = (g.random((N, H)) < 0.3).astype(float)
    Y = np.zeros((N, D))
    for n in range(N):
        act = np.flatnonzero(S[n])
        if len(act):
            win = act[np.argmax(np.abs(Wt[act]), axis=0)]
            Y[n] = Wt[win, np.arange(D)]
    return Y + g.standard_normal((N, D)), Wt


@pytest.mark.parametrize("seed", [0, 1])
def test_mmca_exact_equals_bruteforce(orc, seed):
    Y, Wt = _small_mmca(seed)
    H = Wt.shape[0]
    for y in Y:
        post = orc.posterior(orc.MMCA, y, Wt, 0.3, 0.9, H, H, rho=20)
        S, lj = brute_logjoint_mmca(y, Wt, 0.3, 0.9)
        idx = match_states(state_vectors(post, H), S)
        np.testing.assert_allclose(post["ell"], lj[idx], rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(post["q"], np.exp(lj - logsumexp(lj))[idx], rtol=1e-10, atol=1e-14)


def test_mmca_nonnegative_dictionary_is_mca(orc):
    """With W > 0 the largest magnitude is the largest value: MMCA = MCA in the
    E-step and its rho-smoothed statistics; the M-steps agree wherever MCA's
    positivity clamp (W >= 1e-6) is not active, and where it is, MMCA keeps
    the unclamped (signed) update."""
    Y, Wt = _small_mca(7, N=12)
    Wt = Wt + 0.5
    a = orc.estep(orc.MMCA, Y, Wt, 0.2, 1.1, 4, 2, rho=20)
    b = orc.estep(orc.MCA, Y, Wt, 0.2, 1.1, 4, 2, rho=20)
    for k in ("sel", "smean", "logZ", "mca", "scal"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-13)
    Wa = orc.mstep(orc.MMCA, 12, a, Wt, 0.2, 1.1)[0]
    Wb = orc.mstep(orc.MCA, 12, b, Wt, 0.2, 1.1)[0]
    free = Wb > 1e-6
    np.testing.assert_allclose(Wa[free], Wb[free], rtol=1e-12)
    assert np.all(Wa[~free] <= 1e-6)


def test_mmca_gamma1_equals_bsc_gamma1(orc):
    """At most one active unit: f = W_h s_h, the linear superposition."""
    Y, Wt = _small_mmca(3, N=10)
    sel = np.tile(np.array([0, 2, 3, 5], np.int32), (len(Y), 1))
    a = orc.estep(orc.MMCA, Y, Wt, 0.2, 1.1, 4, 1, rho=20, sel_in=sel)
    b = orc.estep(orc.BSC, Y, Wt, 0.2, 1.1, 4, 1, sel_in=sel)
    np.testing.assert_allclose(a["smean"], b["smean"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(a["logZ"], b["logZ"], rtol=1e-12)


def test_mmca_mstep_limits(orc):
    """gamma = 1: A_dh = s_h, W_dh = sum<s_h> y_d / sum<s_h> (signs kept, no
    clamp); rho -> infinity: the unit of largest |W_dh| takes pixel d."""
    Y, Wt = _small_mmca(4, N=30)
    H, D = Wt.shape
    out = orc.estep(orc.MMCA, Y, Wt, 0.2, 1.1, H, 1, rho=20)
    num = np.zeros((H, D))
    den = np.zeros(H)
    for y in Y:
        post = orc.posterior(orc.MMCA, y, Wt, 0.2, 1.1, H, 1, rho=20)
        for q, v in zip(post["q"], state_vectors(post, H)):
            num += q * v[:, None] * y[None, :]
            den += q * v
    W2 = orc.mstep(orc.MMCA, len(Y), out, Wt, 0.2, 1.1)[0]
    np.testing.assert_allclose(W2, num / den[:, None], rtol=1e-10)
    assert np.any(W2 < 0)
    rho = 3000.0
    out = orc.estep(orc.MMCA, Y, Wt, 0.3, 1.0, H, 3, rho=rho)
    num = np.zeros((H, D))
    den = np.zeros((H, D))
    for y in Y:
        post = orc.posterior(orc.MMCA, y, Wt, 0.3, 1.0, H, 3, rho=rho)
        for q, v in zip(post["q"], state_vectors(post, H)):
            act = np.flatnonzero(v)
            if not len(act):
                continue
            win = act[np.argmax(np.abs(Wt[act]), axis=0)]
            for d in range(D):
                num[win[d], d] += q * y[d]
                den[win[d], d] += q
    W2 = orc.mstep(orc.MMCA, len(Y), out, Wt, 0.3, 1.0)[0]
    m = den > 1e-3
    np.testing.assert_allclose(W2[m], num[m] / den[m], rtol=2e-3, atol=1e-3)


def test_mmca_selection_uses_magnitude_normaliser(orc):
    """MMCA score (reading): sum_d W_dh y_d / sum_d |W_dh|, worked by hand."""
    Wt = np.array([[1.0, -1.0, 0.0], [2.0, 0.0, 2.0], [0.0, -3.0, 1.0]])
    y = np.array([2.0, -1.0, 4.0])
    # h0: (2 + 1) / 2 = 1.5; h1: (4 + 8) / 4 = 3; h2: (3 + 4) / 4 = 1.75
    np.testing.assert_array_equal(orc.scores(orc.MMCA, y, Wt), [1.5, 3.0, 1.75])
    assert orc.posterior(orc.MMCA, y, Wt, 0.2, 1.0, 2, 1, rho=20)["sel"].tolist() == [1, 2]


# ---------------------------------------------------------------------------
# TSC / DSC (Table 1: linear superposition, discrete latents, categorical prior)
# ---------------------------------------------------------------------------
DSC_VALS = np.array([0.5, 2.0, -1.5])
DSC_P = np.array([0.15, 0.1, 0.05])


def brute_logjoint_dsc(y, Wt, vals, pvals, sigma):
    """log p(s, y) for every s in {0, vals}^H: categorical prior, scipy Gaussian."""
    H, D = Wt.shape
    levels = np.concatenate([[0.0], vals])
    lp = np.log(np.concatenate([[1.0 - np.sum(pvals)], pvals]))
    idx = np.array(list(itertools.product(range(len(levels)), repeat=H)))
    S = levels[idx]
    prior = lp[idx].sum(1)
    ll = multivariate_normal(mean=np.zeros(D), cov=sigma ** 2 * np.eye(D)).logpdf(y[None, :] - S @ Wt)
    return S, prior + ll


def dsc_state_vectors(post, H, vals):
    sel = post["sel"]
    V = np.zeros((len(post["masks"]), H))
    for i, (m, c) in enumerate(zip(post["masks"], post["vcodes"])):
        a = 0
        for j in range(len(sel)):
            if (int(m) >> j) & 1:
                V[i, sel[j]] = vals[(int(c) >> (2 * a)) & 3]
                a += 1
    return V


def match_value_states(V, S):
    key = {tuple(np.round(s, 12)): i for i, s in enumerate(S)}
    return np.array([key[tuple(np.round(v, 12))] for v in V])


def test_dsc_state_counts_golden(orc):
    path = os.path.join(GOLDEN, "dsc_state_counts.txt")
    rows = [l.split("#")[0].split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 5
    for hp, g, m, n in rows:
        assert orc.num_states_m(int(hp), int(g), int(m)) == int(n)
        assert len(orc.states_dsc(int(hp), int(g), int(m))[0]) == int(n)


def test_dsc_state_order_is_canonical(orc):
    """By number of nonzero units, then the units' combination order, then the
    value indices (itertools.product order, first unit most significant)."""
    for hp, g, m in [(5, 3, 2), (4, 4, 3), (6, 2, 1)]:
        masks, codes = orc.states_dsc(hp, g, m)
        expect = []
        for k in range(g + 1):
            for c in itertools.combinations(range(hp), k):
                for v in itertools.product(range(m), repeat=k):
                    expect.append((sum(1 << j for j in c), sum(vi << (2 * a) for a, vi in enumerate(v))))
        assert list(zip(masks.tolist(), codes.tolist())) == expect


@pytest.mark.parametrize("model", ["TSC", "DSC"])
def test_discrete_exact_equals_bruteforce(orc, model):
    """ET with H' = H = gamma is exact: log-joints, posterior and log p(y) equal
    the sum over all |Phi|^H states with scipy's Gaussian density and the
    categorical prior (TSC: Phi = {-1, 0, 1}, p(+-1) = pi/2)."""
    g = synth.rng(21)
    if model == "TSC":
        H, D, pi = 5, 7, 0.3
        vals, pvals, kw = np.array([-1.0, 1.0]), np.array([pi / 2, pi / 2]), {}
    else:
        H, D, pi = 4, 6, float(DSC_P.sum())
        vals, pvals = DSC_VALS, DSC_P
        kw = dict(vals=vals, pvals=pvals)
    Wt = g.standard_normal((H, D))
    m = getattr(orc, model)
    sigma = 0.9
    for _ in range(3):
        s_true = g.choice(np.concatenate([[0.0], vals]), H)
        y = s_true @ Wt + sigma * g.standard_normal(D)
        post = orc.posterior(m, y, Wt, pi, sigma, H, H, **kw)
        S, lj = brute_logjoint_dsc(y, Wt, vals, pvals, sigma)
        assert len(post["q"]) == len(S)
        idx = match_value_states(dsc_state_vectors(post, H, vals), S)
        assert len(set(idx.tolist())) == len(S)
        np.testing.assert_allclose(post["ell"], lj[idx], rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(post["q"], np.exp(lj - logsumexp(lj))[idx], rtol=1e-10, atol=1e-14)
        out = orc.estep(m, y[None, :], Wt, pi, sigma, H, H, **kw)
        assert abs(out["logZ"][0] - logsumexp(lj)) < 1e-10
        # moments from the brute-force posterior
        q = np.exp(lj - logsumexp(lj))
        np.testing.assert_allclose(out["At"], np.outer(q @ S, y), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(out["B"], (S * q[:, None]).T @ S, rtol=1e-10, atol=1e-12)


def test_dsc_binary_values_reduce_to_bsc(orc):
    """DSC with the single nonzero value 1 (probability pi) is BSC."""
    Y, Wt = _small_bsc(8, H=8, D=9, N=5)
    a = orc.estep(orc.DSC, Y, Wt, 0.2, 0.8, 5, 3, vals=[1.0], pvals=[0.2])
    b = orc.estep(orc.BSC, Y, Wt, 0.2, 0.8, 5, 3)
    for k in ("sel", "smean", "logZ", "At", "B", "map_idx"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a["scal"][:4], b["scal"][:4], rtol=1e-12)


def test_tsc_is_dsc_with_symmetric_values(orc):
    Y, Wt = _small_bsc(9, H=8, D=9, N=5)
    a = orc.estep(orc.TSC, Y, Wt, 0.2, 0.8, 5, 3)
    b = orc.estep(orc.DSC, Y, Wt, 0.2, 0.8, 5, 3, vals=[-1.0, 1.0], pvals=[0.1, 0.1])
    for k in ("sel", "smean", "logZ", "At", "B", "map_idx", "map_val", "scal"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-13)


def test_tsc_selection_takes_magnitude(orc):
    """TSC preselection (reading): |W_h^T y| / ||W_h||, so a latent that explains
    y with the value -1 is a candidate; BSC's signed score would skip it."""
    D = 6
    Wt = np.eye(D)[:5] * np.array([[1.0], [2.0], [1.0], [1.0], [3.0]])
    y = np.array([0.5, -4.0, 0.1, 1.0, 0.0, 0.0])       # scores: .5, -4, .1, 1, 0
    tsc = orc.scores(orc.TSC, y, Wt)
    bsc = orc.scores(orc.BSC, y, Wt)
    np.testing.assert_array_equal(tsc, [0.5, 4.0, 0.1, 1.0, 0.0])
    np.testing.assert_array_equal(bsc, [0.5, -4.0, 0.1, 1.0, 0.0])
    assert orc.posterior(orc.TSC, y, Wt, 0.2, 1.0, 2, 1)["sel"].tolist() == [1, 3]
    assert orc.posterior(orc.BSC, y, Wt, 0.2, 1.0, 2, 1)["sel"].tolist() == [0, 3]
    # DSC with only negative values negates the score
    neg = orc.scores(orc.DSC, y, Wt, vals=[-1.0, -2.0], pvals=[0.1, 0.1])
    np.testing.assert_array_equal(neg, -bsc)


def _Q_dsc(orc, model, posts, Y, Wt, sigma, vals, pvals):
    """sum_n E_q[log p(s) + log p(y|s)] with the categorical prior and an
    independent residual formula (q and the states from the E-step)."""
    H, D = Wt.shape
    lp = np.log(np.concatenate([[1 - np.sum(pvals)], pvals]))
    Q = 0.0
    for post, y in zip(posts, Y):
        V = dsc_state_vectors(post, H, vals)
        vi = np.zeros(V.shape, int)
        for k, v in enumerate(vals):
            vi[V == v] = k + 1
        prior = lp[vi].sum(1)
        r2 = ((y[None, :] - V @ Wt) ** 2).sum(1)
        Q += post["q"] @ (prior - 0.5 * D * np.log(2 * np.pi * sigma ** 2) - r2 / (2 * sigma ** 2))
    return Q


def test_dsc_mstep_is_stationary_point_of_Q(orc):
    """The DSC M-step (W = A B^-1, sigma^2, each value's probability = its
    expected frequency) zeroes the gradient of Q, including along the simplex
    directions of the categorical prior."""
    g = synth.rng(31)
    H, D, N = 6, 8, 40
    Wt0 = g.standard_normal((H, D))
    S = g.choice(np.concatenate([[0.0], DSC_VALS]), (N, H), p=[0.7, 0.15, 0.1, 0.05])
    Y = S @ Wt0 + 0.7 * g.standard_normal((N, D))
    Wt = Wt0 + 0.3 * g.standard_normal((H, D))
    kw = dict(vals=DSC_VALS, pvals=DSC_P)
    Hp, gam = 4, 2
    out = orc.estep(orc.DSC, Y, Wt, DSC_P.sum(), 0.8, Hp, gam, **kw)
    posts = [orc.posterior(orc.DSC, y, Wt, DSC_P.sum(), 0.8, Hp, gam, **kw) for y in Y]
    W2, pi2, s2, p2 = orc.mstep_dsc(orc.DSC, N, out, Wt, DSC_P.sum(), 0.8, **kw)
    assert abs(pi2 - p2.sum()) < 1e-12
    Q = lambda W, s, p: _Q_dsc(orc, orc.DSC, posts, Y, W, s, DSC_VALS, p)
    base = Q(W2, s2, p2)
    eps = 1e-5
    for (h, dd) in [(0, 0), (2, 5), (5, 7)]:
        Wp, Wm = W2.copy(), W2.copy()
        Wp[h, dd] += eps
        Wm[h, dd] -= eps
        assert abs((Q(Wp, s2, p2) - Q(Wm, s2, p2)) / (2 * eps)) < 1e-6 * abs(base)
    assert abs((Q(W2, s2 + eps, p2) - Q(W2, s2 - eps, p2)) / (2 * eps)) < 1e-6 * abs(base)
    for v in range(3):          # moving mass between value v and 0 (pi_0 absorbs it)
        e = np.zeros(3)
        e[v] = eps
        assert abs((Q(W2, s2, p2 + e) - Q(W2, s2, p2 - e)) / (2 * eps)) < 1e-6 * abs(base), v
    assert Q(W2, s2, p2 * 1.1) < base and Q(W2 * 1.01, s2, p2) < base


def test_tsc_exact_em_monotone(orc):
    """Exact TSC EM (H' = H = gamma): the log-likelihood never decreases."""
    g = synth.rng(41)
    H, D, N = 5, 6, 80
    Wt0 = g.standard_normal((H, D))
    S = g.choice([-1.0, 0.0, 1.0], (N, H), p=[0.15, 0.7, 0.15])
    Y = S @ Wt0 + 0.5 * g.standard_normal((N, D))
    Wt, pi, sigma = g.standard_normal((H, D)), 0.5, float(Y.std())
    F_prev = -np.inf
    for it in range(12):
        out = orc.estep(orc.TSC, Y, Wt, pi, sigma, H, H)
        F = out["scal"][orc.SC_F]
        assert F >= F_prev - 1e-9 * abs(F), (it, F, F_prev)
        F_prev = F
        Wt, pi, sigma, _ = orc.mstep_dsc(orc.TSC, N, out, Wt, pi, sigma)


# ---------------------------------------------------------------------------
# GSC
# ---------------------------------------------------------------------------
def _small_gsc(seed, H=5, D=7, N=3):
    g = synth.rng(seed)
    Wt = g.standard_normal((H, D)) / np.sqrt(D)
    mu = g.uniform(-1, 1, H)
    psi = g.uniform(0.2, 0.8, H)
    S = (g.random((N, H)) < 0.3) * (mu + np.sqrt(psi) * g.standard_normal((N, H)))
    Y = S @ Wt + 0.3 * g.standard_normal((N, D))
    return Y, Wt, mu, psi


@pytest.mark.parametrize("seed", [0, 1])
def test_gsc_exact_equals_bruteforce(orc, seed):
    Y, Wt, mu, psi = _small_gsc(seed)
    H = Wt.shape[0]
    for y in Y:
        post = orc.posterior(orc.GSC, y, Wt, 0.3, 0.35, H, H, mu=mu, psi=psi)
        S, lj = brute_logjoint_gsc(y, Wt, 0.3, 0.35, mu, psi)
        idx = match_states(state_vectors(post, H), S)
        np.testing.assert_allclose(post["ell"], lj[idx], rtol=1e-11, atol=1e-9)
        np.testing.assert_allclose(post["q"], np.exp(lj - logsumexp(lj))[idx], rtol=1e-9, atol=1e-14)


def test_gsc_single_unit_closed_form(orc):
    """|b| = 1: y ~ N(mu w, sigma^2 I + psi w w^T) has the closed form
    log|C| = D log sigma^2 + log(1 + psi|w|^2/sigma^2) (determinant lemma) and
    C^-1 = (I - psi w w^T/(sigma^2 + psi|w|^2))/sigma^2 (Sherman-Morrison);
    the slab posterior is kappa = mu + psi w.(y - mu w)/(sigma^2 + psi|w|^2),
    Lambda = psi sigma^2/(sigma^2 + psi|w|^2)."""
    g = synth.rng(12)
    D, H = 6, 4
    Wt = g.standard_normal((H, D))
    mu = g.uniform(-1, 1, H)
    psi = g.uniform(0.1, 2.0, H)
    y = g.standard_normal(D)
    pi, sigma = 0.2, 0.6
    post = orc.posterior(orc.GSC, y, Wt, pi, sigma, H, 1, mu=mu, psi=psi)
    s2 = sigma ** 2
    for i, m in enumerate(post["masks"]):
        if m == 0:
            continue
        j = int(m).bit_length() - 1
        h = post["sel"][j]
        w = Wt[h]
        a = s2 + psi[h] * w @ w
        r = y - mu[h] * w
        logdet = D * np.log(s2) + np.log(a / s2)
        quad = (r @ r - psi[h] * (w @ r) ** 2 / a) / s2
        lj = np.log(pi) + (H - 1) * np.log(1 - pi) - 0.5 * D * np.log(2 * np.pi) - 0.5 * logdet - 0.5 * quad
        assert abs(post["ell"][i] - lj) < 1e-11
        assert abs(post["kappa"][i, 0] - (mu[h] + psi[h] * (w @ r) / a)) < 1e-12
        assert abs(post["lam"][i, 0, 0] - psi[h] * s2 / a) < 1e-12
        # the GSC preselection score is this singleton log-joint
        assert abs(post["scores"][h] - lj) < 1e-11


def test_gsc_vanishing_slab_reduces_to_bsc(orc):
    """psi -> 0: s_h = b_h mu_h, so GSC is BSC with dictionary W diag(mu)."""
    Y, Wt, mu, psi = _small_gsc(2, N=6)
    H = Wt.shape[0]
    tiny = np.full(H, 1e-13)
    sel = np.tile(np.arange(H, dtype=np.int32), (len(Y), 1))
    a = orc.estep(orc.GSC, Y, Wt, 0.3, 0.4, H, 3, mu=mu, psi=tiny, sel_in=sel)
    b = orc.estep(orc.BSC, Y, Wt * mu[:, None], 0.3, 0.4, H, 3, sel_in=sel)
    np.testing.assert_allclose(a["logZ"], b["logZ"], rtol=1e-9)
    np.testing.assert_allclose(a["gsc"][:H], np.diag(b["B"]), rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(a["smean"], b["smean"] * mu[None, :], rtol=1e-7, atol=1e-12)


def _Q_gsc(posts, Y, Wt, pi, sigma, mu, psi):
    H, D = Wt.shape
    Q = 0.0
    for post, y in zip(posts, Y):
        sel = post["sel"]
        for i, m in enumerate(post["masks"]):
            loc = [j for j in range(len(sel)) if (int(m) >> j) & 1]
            act = sel[loc]
            k = len(act)
            q = post["q"][i]
            kap = post["kappa"][i, :k]
            lam = post["lam"][i, :k, :k]
            Wb = Wt[act].T
            r = y - Wb @ kap
            e_ll = -0.5 * D * np.log(2 * np.pi * sigma ** 2) - (r @ r + np.trace(Wb.T @ Wb @ lam)) / (2 * sigma ** 2)
            e_lp = np.sum(-0.5 * np.log(2 * np.pi * psi[act]) - ((kap - mu[act]) ** 2 + np.diag(lam)) / (2 * psi[act]))
            Q += q * (k * np.log(pi) + (H - k) * np.log(1 - pi) + e_ll + e_lp)
    return Q


def test_gsc_mstep_is_stationary_point_of_Q(orc):
    d = synth.gsc(N=40, seed=7, D=8, H=5)
    Y = d["Y"].astype(np.float64)
    Wt, mu, psi = d["Wt"], d["mu"] + 0.1, d["psi"] * 1.3
    pi, sigma, Hp, gam = 0.25, 0.4, 4, 2
    out = orc.estep(orc.GSC, Y, Wt, pi, sigma, Hp, gam, mu=mu, psi=psi)
    posts = [orc.posterior(orc.GSC, y, Wt, pi, sigma, Hp, gam, mu=mu, psi=psi) for y in Y]
    W2, pi2, s2, mu2, psi2 = orc.mstep(orc.GSC, len(Y), out, Wt, pi, sigma, mu=mu, psi=psi)
    eps = 1e-6
    Q = lambda W=W2, p=pi2, s=s2, m=mu2, v=psi2: _Q_gsc(posts, Y, W, p, s, m, v)
    base = Q()
    for (h, dd) in [(0, 0), (2, 5), (4, 7)]:
        Wp, Wm = W2.copy(), W2.copy()
        Wp[h, dd] += eps
        Wm[h, dd] -= eps
        assert abs((Q(W=Wp) - Q(W=Wm)) / (2 * eps)) < 1e-5 * abs(base)
    assert abs((Q(p=pi2 + eps) - Q(p=pi2 - eps)) / (2 * eps)) < 1e-4
    assert abs((Q(s=s2 + eps) - Q(s=s2 - eps)) / (2 * eps)) < 1e-4
    for h in range(5):
        if out["gsc"][h] <= 1e-9 * len(Y):
            continue
        mp, mm = mu2.copy(), mu2.copy()
        mp[h] += eps
        mm[h] -= eps
        assert abs((Q(m=mp) - Q(m=mm)) / (2 * eps)) < 1e-4
        vp, vm = psi2.copy(), psi2.copy()
        vp[h] += eps
        vm[h] -= eps
        assert abs((Q(v=vp) - Q(v=vm)) / (2 * eps)) < 1e-4


def test_gsc_exact_em_monotone(orc):
    d = synth.gsc(N=80, seed=8, D=8, H=4)
    Y = d["Y"]
    p = synth.init_gsc(Y, 4, seed=3)
    Wt, pi, sigma, mu, psi = p["Wt"], p["pi"], p["sigma"], p["mu"], p["psi"]
    F_prev = -np.inf
    for it in range(12):
        out = orc.estep(orc.GSC, Y, Wt, pi, sigma, 4, 4, mu=mu, psi=psi)
        F = out["scal"][orc.SC_F]
        assert F >= F_prev - 1e-9 * abs(F), (it, F, F_prev)
        F_prev = F
        Wt, pi, sigma, mu, psi = orc.mstep(orc.GSC, len(Y), out, Wt, pi, sigma, mu=mu, psi=psi)
