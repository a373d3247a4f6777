"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI,
run the oracle on the same inputs, and compare with the stated tolerances.

Tolerances (written here, used by every parity test):
  - aggregated statistics At, B and the M-step's W: relative Frobenius error
    <= 1e-5 (FP32 form);
  - per-point posterior means <s> and q(MAP): abs error <= 1e-5 + 8 u Lambda_n,
    where u = 2^-24 and Lambda_n = max |log p(s,y_n) - log p(0,y_n)| over the
    states with q_n(s) > 1e-8: the FP32 rounding of log-joints of that size
    (FP32 cannot hold a log-joint of 1000 nats to better than 6e-5);
  - per-point log Z: abs error <= 1e-5 + 1e-6 T_n, with T_n = y^T y/(2 sigma^2)
    + (D/2)|log 2 pi sigma^2| + H |log(1-pi)| + Lambda_n the sizes of the terms
    that log Z sums (relative FP32 precision of the largest term);
  - F / N (truncated log-likelihood per point): relative error <= 1e-6;
  - selections: identical except at score near-ties, where the GPU's set must
    be optimal within tau = 1e-5 max|score| (FP32 form) or within the BF16
    rounding bound (BF16 form); the oracle then re-runs with the GPU's set.
"""
import numpy as np

REL_AGG = 1e-5
ABS_POINT = 1e-5
REL_F = 1e-6


def relfro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def check_selection(orc, model, Y, Wt, sel_gpu, Hp, tau_fn, mu=None, psi=None, pi=0.5, sigma=1.0,
                    **kw):
    """Return (n_differ, bad): every GPU set must be within tau of optimal
    (kw: DSC values / probabilities for the oracle's score)."""
    Yd = np.asarray(Y, np.float64)
    orc_sel = None
    n_diff = 0
    bad = []
    for n in range(len(Yd)):
        sg = np.sort(np.asarray(sel_gpu[n][:Hp], np.int64))
        sc = orc.scores(model, Yd[n], Wt, pi, sigma, mu=mu, psi=psi, **kw)
        order = np.lexsort((np.arange(len(sc)), -sc))
        so = np.sort(order[:Hp])
        if np.array_equal(sg, so):
            continue
        n_diff += 1
        kth = sc[order[Hp - 1]]
        tau = tau_fn(n, sc)
        if np.any(sc[sg] < kth - tau) or len(set(sg.tolist())) != Hp:
            bad.append(n)
    return n_diff, bad


def torch_stats_to_numpy(st):
    out = {}
    for k, v in st.items():
        out[k] = None if v is None else v.detach().cpu().numpy()
    return out


U32 = 2.0 ** -24


def loglik_scale(orc, model, y, Wt, pi, sigma, Hp, gamma, sel, **kw):
    """Lambda_n of one point (see the tolerance list above); at temperature T
    the kernels round log-joints divided by T."""
    post = orc.posterior(model, y, Wt, pi, sigma, Hp, gamma, sel_in=sel, **kw)
    rel = (post["ell"] - post["ell"][0]) / kw.get("T", 1.0)
    return float(np.max(np.abs(rel[post["q"] > 1e-8])))


def check_points(orc, model, Y, Wt, pi, sigma, Hp, gamma, sel, got, ref, key, scale=1.0, **kw):
    """Per-point check with the FP32 tolerances above; returns the max raw error.
    key "logZ" uses the log Z bound, every other key the posterior bound
    (times ``scale``, the largest |latent value|, for posterior means of
    discrete latents).  kw goes to the oracle (mu, psi, rho, T, vals, pvals)."""
    err = np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))
    if err.ndim > 1:
        err = err.max(axis=1)
    for n in np.flatnonzero(err > ABS_POINT):
        y = np.asarray(Y[n], np.float64)
        lam = loglik_scale(orc, model, y, Wt, pi, sigma, Hp, gamma, sel[n], **kw)
        if key == "logZ":
            H, D = np.asarray(Wt).shape
            T = (y @ y / (2 * sigma ** 2) + 0.5 * D * abs(np.log(2 * np.pi * sigma ** 2))
                 + H * abs(np.log(1 - pi)) + lam)
            tol = ABS_POINT + 1e-6 * T
        else:
            tol = (ABS_POINT + 8 * U32 * lam) * scale
        assert err[n] <= tol, (key, n, err[n], tol, lam)
    return float(err.max()) if len(err) else 0.0
