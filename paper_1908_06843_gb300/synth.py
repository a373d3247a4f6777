"""Seeded synthetic inputs shaped like the ProSper workloads.

This module draws data and initial parameters only; it holds none of the
E-step or M-step arithmetic.  Both the CUDA path and the CPU oracle are fed
from it.  Every generator uses ``numpy.random.Generator(PCG64(seed))``.

Workloads (the paper names no dataset; its scale statement in the abstract --
hundreds of dictionary elements, tens of millions of floats -- and its Table 1
model list fix the shapes):

- ``bars``:     BSC bars test. D = 5x5, H = 10 bars (5 horizontal, 5 vertical,
                pixel value 10 on the bar), s_h ~ Bernoulli(0.2),
                y = W s + N(0, 1).
- ``gabor``:    image-patch-shaped BSC data. D = 16x16, H = 256 random unit-norm
                Gabor filters (orientation U(0, pi), frequency U(0.1, 0.3)
                cycles/pixel, centre U[4, 12]^2, envelope std U(2, 4) px,
                phase U(0, 2 pi)), s_h ~ Bernoulli(4/256), y = W s + N(0, 0.2^2).
- ``mca_bars``: D = 10x10, H = 20 non-negative bars of intensity 8,
                s_h ~ Bernoulli(0.1), y_d = max_h W_dh s_h + N(0, 1).
- ``gsc``:      D = 64, H = 32, W ~ N(0, 1)/sqrt(D), b_h ~ Bernoulli(3/32),
                z_h ~ N(mu_h, psi_h = 0.5) with mu_h ~ U(-1, 1), s = b * z,
                y = W s + N(0, 0.3^2).
- ``mmca_bars``: the MCA bars with random signs, |max| superposition.
- ``discrete``: TSC / DSC data on the Gabor dictionary: s_h takes the value
                phi_v with probability p_v (else 0), y = W s + N(0, sigma^2)
                (TSC: values -1, +1 with pi/2 each).

Dictionaries are returned as ``Wt`` (H x D, row h = dictionary element W_h).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# dictionaries
# --------------------------------------------------------------------------
def bars_dictionary(side: int, value: float) -> np.ndarray:
    """2*side bars on a side x side grid: side horizontal then side vertical."""
    H, D = 2 * side, side * side
    Wt = np.zeros((H, D), dtype=np.float64)
    for i in range(side):
        img = np.zeros((side, side))
        img[i, :] = value
        Wt[i] = img.reshape(-1)
        img = np.zeros((side, side))
        img[:, i] = value
        Wt[side + i] = img.reshape(-1)
    return Wt


def gabor_dictionary(H: int, side: int, g: np.random.Generator) -> np.ndarray:
    yy, xx = np.meshgrid(np.arange(side, dtype=np.float64),
                         np.arange(side, dtype=np.float64), indexing="ij")
    Wt = np.zeros((H, side * side))
    for h in range(H):
        theta = g.uniform(0.0, np.pi)
        freq = g.uniform(0.1, 0.3)
        cy, cx = g.uniform(4.0, 12.0, size=2)
        env = g.uniform(2.0, 4.0)
        phase = g.uniform(0.0, 2.0 * np.pi)
        u = (xx - cx) * np.cos(theta) + (yy - cy) * np.sin(theta)
        r2 = (xx - cx) ** 2 + (yy - cy) ** 2
        img = np.exp(-r2 / (2.0 * env * env)) * np.cos(2.0 * np.pi * freq * u + phase)
        v = img.reshape(-1)
        Wt[h] = v / np.linalg.norm(v)
    return Wt


# --------------------------------------------------------------------------
# datasets: each returns dict(Y float32 N x D, Wt_true, S_true, params_true)
# --------------------------------------------------------------------------
def bars(N: int = 1000, seed: int = 1001, pi: float = 0.2, sigma: float = 1.0,
         side: int = 5, value: float = 10.0):
    g = rng(seed)
    Wt = bars_dictionary(side, value)
    H, D = Wt.shape
    S = (g.random((N, H)) < pi).astype(np.float64)
    Y = S @ Wt + sigma * g.standard_normal((N, D))
    return dict(Y=Y.astype(np.float32), Wt=Wt, S=S, pi=pi, sigma=sigma)


def gabor(N: int = 200_000, seed: int = 1002, H: int = 256, side: int = 16,
          pi: float = 4.0 / 256.0, sigma: float = 0.2, chunk: int = 50_000):
    g = rng(seed)
    Wt = gabor_dictionary(H, side, g)
    D = side * side
    Y = np.empty((N, D), dtype=np.float32)
    nnz = 0
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        S = (g.random((b - a, H)) < pi).astype(np.float64)
        nnz += int(S.sum())
        Y[a:b] = (S @ Wt + sigma * g.standard_normal((b - a, D))).astype(np.float32)
    return dict(Y=Y, Wt=Wt, S=None, pi=pi, sigma=sigma, nnz=nnz)


def mca_bars(N: int = 100_000, seed: int = 1003, pi: float = 0.1, sigma: float = 1.0,
             side: int = 10, value: float = 8.0):
    g = rng(seed)
    Wt = bars_dictionary(side, value)
    H, D = Wt.shape
    S = (g.random((N, H)) < pi).astype(np.float64)
    F = np.max(S[:, :, None] * Wt[None, :, :], axis=1)
    Y = F + sigma * g.standard_normal((N, D))
    return dict(Y=Y.astype(np.float32), Wt=Wt, S=S, pi=pi, sigma=sigma)


def mmca_bars(N: int = 20_000, seed: int = 1005, pi: float = 0.1, sigma: float = 1.0,
              side: int = 10, value: float = 8.0):
    """MMCA data: the bars of ``mca_bars`` with a random sign per bar; per pixel
    the active bar of largest magnitude (the lower index on a tie) plus noise."""
    g = rng(seed)
    Wt = bars_dictionary(side, value) * np.where(g.random(2 * side) < 0.5, -1.0, 1.0)[:, None]
    H, D = Wt.shape
    S = (g.random((N, H)) < pi).astype(np.float64)
    A = np.abs(S[:, :, None] * Wt[None, :, :])                  # N x H x D magnitudes
    win = np.argmax(A, axis=1)                                   # first maximum: the lower h
    F = np.where(A.max(axis=1) > 0, Wt[win, np.arange(D)[None, :]], 0.0)
    Y = F + sigma * g.standard_normal((N, D))
    return dict(Y=Y.astype(np.float32), Wt=Wt, S=S, pi=pi, sigma=sigma)


def gsc(N: int = 50_000, seed: int = 1004, D: int = 64, H: int = 32,
        pi: float = 3.0 / 32.0, psi: float = 0.5, sigma: float = 0.3):
    g = rng(seed)
    Wt = g.standard_normal((H, D)) / np.sqrt(D)
    mu = g.uniform(-1.0, 1.0, size=H)
    psi_v = np.full(H, psi)
    B = (g.random((N, H)) < pi).astype(np.float64)
    Z = mu[None, :] + np.sqrt(psi_v)[None, :] * g.standard_normal((N, H))
    S = B * Z
    Y = S @ Wt + sigma * g.standard_normal((N, D))
    return dict(Y=Y.astype(np.float32), Wt=Wt, S=S, pi=pi, sigma=sigma, mu=mu, psi=psi_v)


def discrete(N: int = 50_000, seed: int = 1006, H: int = 64, side: int = 16,
             vals=(-1.0, 1.0), pvals=(2.0 / 64, 2.0 / 64), sigma: float = 0.2):
    """Linear superposition of a Gabor dictionary with discrete latents."""
    g = rng(seed)
    Wt = gabor_dictionary(H, side, g)
    D = side * side
    levels = np.concatenate([[0.0], np.asarray(vals, np.float64)])
    probs = np.concatenate([[1.0 - float(np.sum(pvals))], np.asarray(pvals, np.float64)])
    S = levels[g.choice(len(levels), size=(N, H), p=probs)]
    Y = S @ Wt + sigma * g.standard_normal((N, D))
    return dict(Y=Y.astype(np.float32), Wt=Wt, S=S, vals=np.asarray(vals, np.float64),
                pvals=np.asarray(pvals, np.float64), sigma=sigma)


# --------------------------------------------------------------------------
# initial parameters
# --------------------------------------------------------------------------
def init_bsc(Y: np.ndarray, H: int, seed: int, pi: float, normalise: bool):
    """W ~ N(0, 1) (columns scaled to unit norm if ``normalise``), sigma = std(Y)."""
    g = rng(seed)
    D = Y.shape[1]
    Wt = g.standard_normal((H, D))
    if normalise:
        Wt /= np.linalg.norm(Wt, axis=1, keepdims=True)
    return dict(Wt=Wt, pi=pi, sigma=float(np.std(Y, dtype=np.float64)))


def init_mca(Y: np.ndarray, H: int, seed: int, pi: float = 0.1):
    """W = |N(0, 1)| + mean(Y) (non-negative), sigma = std(Y)."""
    g = rng(seed)
    D = Y.shape[1]
    Wt = np.abs(g.standard_normal((H, D))) + float(np.mean(Y, dtype=np.float64))
    Wt = np.maximum(Wt, 1e-3)
    return dict(Wt=Wt, pi=pi, sigma=float(np.std(Y, dtype=np.float64)))


def init_gsc(Y: np.ndarray, H: int, seed: int, pi: float = 0.1):
    g = rng(seed)
    D = Y.shape[1]
    Wt = g.standard_normal((H, D))
    Wt /= np.linalg.norm(Wt, axis=1, keepdims=True)
    return dict(Wt=Wt, pi=pi, sigma=float(np.std(Y, dtype=np.float64)),
                mu=np.zeros(H), psi=np.ones(H))


# --------------------------------------------------------------------------
# serving workload: request sizes and Poisson arrival times
# --------------------------------------------------------------------------
def request_sizes(n: int, seed: int, max_size: int = 4096) -> np.ndarray:
    """floor(exp(U(0, ln max_size))) clamped to [1, max_size] (log-uniform)."""
    g = rng(seed)
    s = np.floor(np.exp(g.uniform(0.0, np.log(max_size), size=n))).astype(np.int64)
    return np.clip(s, 1, max_size)


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times in seconds of a Poisson process of the given rate."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate, size=n))
