"""FP64 CPU oracle for the ProSper truncated-EM E-step and M-steps (BSC, MCA, GSC).

TEST INFRASTRUCTURE ONLY.  This package is the correctness reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product package
``paper_1908_06843_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``prosper_oracle.c`` (plain C, double precision,
OpenMP over data points).  This module only compiles it with gcc and marshals
numpy arrays through ctypes.  See the C file's header for what each function
computes and which part of the paper (Eq. 1-2, Table 1, Sec. 2-3) it follows.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
except the MCA rho-smoothed M-step away from its two limits (gamma = 1 and
rho -> infinity), whose general form the paper does not state: parity
unpinned for that update.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prosper_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libprosper_oracle.so")
_lock = threading.Lock()
_lib = None

BSC, MCA, GSC, TSC, DSC, MMCA = 0, 1, 2, 3, 4, 5
SC_F, SC_S1, SC_YY, SC_N, SC_MCA_R2, SC_DSC0, SC_LEN = 0, 1, 2, 3, 4, 5, 8
TH_LEN = 12
TSC_VALUES = (-1.0, 1.0)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP). Returns its path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            _lib.orc_num_states.argtypes = [i32, i32]
            _lib.orc_states.argtypes = [i32, i32, P, i32]
            _lib.orc_num_states_m.argtypes = [i32, i32, i32]
            _lib.orc_states_dsc.argtypes = [i32, i32, i32, P, P, i32]
            _lib.orc_estep.argtypes = [i32, i64, i32, i32, i32, i32] + [P] * 17 + [i32]
            _lib.orc_posterior.argtypes = [i32, i32, i32, i32, i32] + [P] * 14
            _lib.orc_scores.argtypes = [i32, i32, i32] + [P] * 6
            _lib.orc_mstep.argtypes = [i32, i32, i32, dbl] + [P] * 9
            _lib.orc_trunc_prob.argtypes = [i32, i32, dbl]
            _lib.orc_trunc_prob.restype = dbl
            _lib.orc_cut_size.argtypes = [i64, i32, i32, dbl]
            _lib.orc_cut_size.restype = i64
            _lib.orc_pi_correction.argtypes = [i32, i32, dbl]
            _lib.orc_pi_correction.restype = dbl
            _lib.orc_cut_keep.argtypes = [i64, P, i64, P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def num_states(Hp: int, gamma: int) -> int:
    return _load().orc_num_states(Hp, gamma)


def states(Hp: int, gamma: int) -> np.ndarray:
    """Canonical state masks over local units (by size, then lexicographic)."""
    n = num_states(Hp, gamma)
    out = np.zeros(n, dtype=np.uint32)
    _load().orc_states(Hp, gamma, _p(out), n)
    return out


def theta_vec(pi, sigma, rho=0.0, T=1.0, vals=None, pvals=None):
    """The oracle's theta: {pi, sigma, rho, T, p_1..p_3, m, phi_1..phi_3, 0}.
    T is the posterior temperature of deterministic annealing (q ~ p(s, y)^(1/T);
    1 = the plain truncated posterior).  DSC: vals = the m <= 3 nonzero values
    phi_v, pvals = their prior probabilities."""
    th = np.zeros(TH_LEN)
    th[:4] = [pi, sigma, rho, T]
    if vals is not None:
        m = len(vals)
        assert 1 <= m <= 3 and len(pvals) == m
        th[4:4 + m] = pvals
        th[7] = m
        th[8:8 + m] = vals
    return th


def num_states_m(Hp: int, gamma: int, m: int) -> int:
    """sum_{k <= gamma} C(Hp, k) m^k: discrete states with m nonzero values."""
    return _load().orc_num_states_m(Hp, gamma, m)


def states_dsc(Hp: int, gamma: int, m: int):
    """Canonical discrete states: (unit masks, value codes: 2 bits per nonzero unit)."""
    n = num_states_m(Hp, gamma, m)
    masks = np.zeros(n, dtype=np.uint32)
    codes = np.zeros(n, dtype=np.uint32)
    _load().orc_states_dsc(Hp, gamma, m, _p(masks), _p(codes), n)
    return masks, codes


def _values(model, vals):
    if model == TSC:
        return np.array(TSC_VALUES)
    if model == DSC:
        return np.asarray(vals, np.float64)
    return np.array([1.0])


def estep(model, Y, Wt, pi, sigma, Hp, gamma, rho=0.0, mu=None, psi=None,
          sel_in=None, nthreads=0, T=1.0, vals=None, pvals=None):
    """Truncated E-step over all rows of Y (at posterior temperature T).
    Returns a dict of numpy arrays: sel, smean, map_idx, map_val, map_p, logZ
    (per point; logZ = T log sum_{K_n} p(s, y_n)^(1/T)) and At, B, scal, gsc,
    mca.  DSC: vals / pvals are the nonzero values and their probabilities."""
    lib = _load()
    Y = _f64(Y)
    Wt = _f64(Wt)
    N, D = Y.shape
    H = Wt.shape[0]
    th = theta_vec(pi, sigma, rho, T, vals, pvals)
    mu, psi = _f64(mu), _f64(psi)
    if model == GSC:
        assert mu is not None and psi is not None
    si = None if sel_in is None else np.ascontiguousarray(sel_in, dtype=np.int32)
    out = dict(
        sel=np.zeros((N, Hp), np.int32), smean=np.zeros((N, Hp)),
        map_idx=np.zeros((N, max(gamma, 1)), np.int32), map_val=np.zeros((N, max(gamma, 1))),
        map_p=np.zeros(N),
        logZ=np.zeros(N), At=np.zeros((H, D)), B=np.zeros((H, H)),
        scal=np.zeros(SC_LEN),
        gsc=np.zeros(3 * H) if model == GSC else None,
        mca=np.zeros(2 * H * D) if model in (MCA, MMCA) else None,
    )
    rc = lib.orc_estep(model, N, D, H, Hp, gamma, _p(Y), _p(Wt), _p(th), _p(mu), _p(psi),
                       _p(si), _p(out["sel"]), _p(out["smean"]),
                       _p(out["map_idx"]) if gamma > 0 else None,
                       _p(out["map_val"]) if gamma > 0 else None, _p(out["map_p"]),
                       _p(out["logZ"]), _p(out["At"]), _p(out["B"]), _p(out["scal"]),
                       _p(out["gsc"]), _p(out["mca"]), int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_estep failed ({rc})")
    if gamma == 0:
        out["map_idx"] = np.zeros((N, 0), np.int32)
        out["map_val"] = np.zeros((N, 0))
    if out["mca"] is not None:
        out["mca"] = out["mca"].reshape(2, H, D)
    return out


def posterior(model, y, Wt, pi, sigma, Hp, gamma, rho=0.0, mu=None, psi=None, sel_in=None,
              T=1.0, vals=None, pvals=None):
    """Full truncated posterior of one point at temperature T:
    dict(sel, masks, vcodes, ell (log p(s, y)), q, kappa, lambda, scores)."""
    lib = _load()
    y = _f64(y)
    Wt = _f64(Wt)
    H, D = Wt.shape
    nK = num_states_m(Hp, gamma, len(_values(model, vals)))
    th = theta_vec(pi, sigma, rho, T, vals, pvals)
    mu, psi = _f64(mu), _f64(psi)
    si = None if sel_in is None else np.ascontiguousarray(sel_in, dtype=np.int32)
    sel = np.zeros(Hp, np.int32)
    masks = np.zeros(nK, np.uint32)
    vcodes = np.zeros(nK, np.uint32)
    ell = np.zeros(nK)
    q = np.zeros(nK)
    kappa = np.zeros((nK, Hp)) if model == GSC else None
    lam = np.zeros((nK, Hp, Hp)) if model == GSC else None
    scores = np.zeros(H)
    rc = lib.orc_posterior(model, D, H, Hp, gamma, _p(y), _p(Wt), _p(th), _p(mu), _p(psi),
                           _p(si), _p(sel), _p(masks), _p(vcodes), _p(ell), _p(q), _p(kappa),
                           _p(lam), _p(scores))
    if rc < 0:
        raise ValueError("orc_posterior failed")
    return dict(sel=sel, masks=masks, vcodes=vcodes, ell=ell, q=q, kappa=kappa, lam=lam,
                scores=scores)


def scores(model, y, Wt, pi=0.5, sigma=1.0, mu=None, psi=None, vals=None, pvals=None):
    lib = _load()
    y = _f64(y)
    Wt = _f64(Wt)
    H, D = Wt.shape
    th = theta_vec(pi, sigma, vals=vals, pvals=pvals)
    out = np.zeros(H)
    lib.orc_scores(model, D, H, _p(y), _p(Wt), _p(th), _p(_f64(mu)), _p(_f64(psi)), _p(out))
    return out


def mstep(model, N, stats, Wt, pi, sigma, mu=None, psi=None):
    """Closed-form M-step.  Returns (Wt_new, pi_new, sigma_new, mu_new, psi_new)."""
    lib = _load()
    Wt = np.array(Wt, dtype=np.float64, copy=True)
    H, D = Wt.shape
    th = theta_vec(pi, sigma)
    mu = None if mu is None else np.array(mu, dtype=np.float64, copy=True)
    psi = None if psi is None else np.array(psi, dtype=np.float64, copy=True)
    mca = None if stats.get("mca") is None else _f64(stats["mca"]).reshape(-1)
    rc = lib.orc_mstep(model, D, H, float(N), _p(_f64(stats["At"])), _p(_f64(stats["B"])),
                       _p(_f64(stats["scal"])), _p(_f64(stats.get("gsc"))), _p(mca),
                       _p(Wt), _p(th), _p(mu), _p(psi))
    if rc != 0:
        raise ValueError(f"orc_mstep failed ({rc})")
    return Wt, th[0], th[1], mu, psi


def mstep_dsc(model, N, stats, Wt, pi, sigma, vals=None, pvals=None):
    """Closed-form M-step of TSC / DSC.  Returns (Wt_new, pi_new, sigma_new,
    pvals_new): TSC pi = the fraction of nonzero units (p(+-1) = pi/2); DSC
    the new probability of each nonzero value (pi_new = their sum)."""
    lib = _load()
    Wt = np.array(Wt, dtype=np.float64, copy=True)
    H, D = Wt.shape
    th = theta_vec(pi, sigma, vals=vals, pvals=pvals)
    rc = lib.orc_mstep(model, D, H, float(N), _p(_f64(stats["At"])), _p(_f64(stats["B"])),
                       _p(_f64(stats["scal"])), None, None, _p(Wt), _p(th), None, None)
    if rc != 0:
        raise ValueError(f"orc_mstep failed ({rc})")
    m = len(vals) if vals is not None else 0
    return Wt, th[0], th[1], th[4:4 + m].copy()


def trunc_prob(H, gamma, pi):
    """P_pi(|s| <= gamma) under the Bernoulli prior."""
    return _load().orc_trunc_prob(H, gamma, float(pi))


def cut_size(N, H, gamma, pi):
    """N_cut = floor(N P_pi(|s| <= gamma)), at least 1 (ET data-point cut)."""
    return _load().orc_cut_size(int(N), H, gamma, float(pi))


def pi_correction(H, gamma, pi):
    """H pi / E_pi[|s| : |s| <= gamma]."""
    return _load().orc_pi_correction(H, gamma, float(pi))


def cut_keep(logZ, ncut):
    """Boolean mask of the points whose log Z reaches the ncut-th largest value."""
    lz = np.ascontiguousarray(logZ, dtype=np.float64)
    keep = np.zeros(len(lz), np.uint8)
    _load().orc_cut_keep(len(lz), _p(lz), int(ncut), _p(keep))
    return keep.astype(bool)


def mstep_cut(model, ncut_kept, stats, Wt, pi, sigma, gamma, mu=None, psi=None):
    """M-step on the kept points' statistics with ET's pi correction:
    pi_new = (sum<|s|> / (N_kept H)) * H pi / E_pi[|s| : |s| <= gamma]."""
    H = np.asarray(Wt).shape[0]
    W2, pi2, s2, mu2, psi2 = mstep(model, ncut_kept, stats, Wt, pi, sigma, mu, psi)
    return W2, pi2 * pi_correction(H, gamma, pi), s2, mu2, psi2


def estep_cut(model, Y, Wt, pi, sigma, Hp, gamma, sel_in=None, logZ_in=None, **kw):
    """E-step with ET's data-point cut: the plain E-step gives every point's
    log Z (or logZ_in, e.g. the values a GPU compared against), the cut keeps
    the points reaching the N_cut-th largest, and the statistics are the
    E-step's over the kept points (with their candidate sets).  Returns
    (statistics of the kept points, keep mask, N_cut)."""
    full = estep(model, Y, Wt, pi, sigma, Hp, gamma, sel_in=sel_in, **kw)
    H = np.asarray(Wt).shape[0]
    ncut = cut_size(len(Y), H, gamma, pi)
    keep = cut_keep(full["logZ"] if logZ_in is None else logZ_in, ncut)
    sub = estep(model, np.asarray(Y)[keep], Wt, pi, sigma, Hp, gamma,
                sel_in=full["sel"][keep], **kw)
    return sub, keep, ncut


def exact_em_free_energy(model, Y, Wt, pi, sigma, rho=0.0, mu=None, psi=None):
    """Exact log-likelihood sum_n log p(y_n) (ET with H' = H = gamma)."""
    H = np.asarray(Wt).shape[0]
    return estep(model, Y, Wt, pi, sigma, H, H, rho=rho, mu=mu, psi=psi)["scal"][SC_F]
