"""The paper's user interface (Sec. 3) on top of the C ABI.

    model = BSC_ET(D, H, Hprime, gamma)          # or MCA_ET, GSC_ET
    anneal = LinearAnnealing(150)
    params = model.standard_init({"y": data})
    em = EM(model=model, anneal=anneal, data={"y": data}, lparams=params)
    em.run()
    res = model.inference(anneal, em.lparams, data)   # res["s"], res["p"]

Every E-step, M-step and encoding runs in the CUDA kernels behind
include/prosper.h; this module only keeps the parameters as device tensors
and calls the library in order.  LinearAnnealing controls the number of
iterations and the posterior temperature of deterministic annealing (the
E-step uses q ~ p(s, y)^(1/T)); parameter noise is not built.
"""
from __future__ import annotations

import numpy as np

from . import binding, distributed, synth


class LinearAnnealing:
    """Schedule object of Sec. 3: ``next()`` advances one EM iteration and
    returns False after ``steps`` iterations; ``reset()`` starts over.

    Deterministic annealing: the posterior temperature ``T`` falls linearly
    from ``T0`` at the first iteration to 1 at iteration ``anneal_steps``
    (default: half of the iterations) and stays 1 afterwards; every E-step
    then uses q(s) ~ p(s, y)^(1/T).  ``T0 = 1`` (the default) is plain EM."""

    def __init__(self, steps: int, T0: float = 1.0, anneal_steps=None):
        self.steps = int(steps)
        self.T0 = float(T0)
        self.anneal_steps = max(1, int(anneal_steps if anneal_steps is not None else steps // 2))
        self.cur = 0
        self.T = self.T0

    def temperature(self, it: int) -> float:
        """T at (0-based) iteration it."""
        f = min(1.0, it / self.anneal_steps)
        return self.T0 + (1.0 - self.T0) * f

    def reset(self):
        self.cur = 0
        self.T = self.T0

    def next(self) -> bool:
        if self.cur >= self.steps:
            return False
        self.T = self.temperature(self.cur)
        self.cur += 1
        return True


class _Model:
    kind = binding.BSC

    def __init__(self, D, H, Hprime, gamma, precision=binding.FP32, device="cuda",
                 max_points=1 << 20, data_cut=False):
        import torch
        self.D, self.H, self.Hprime, self.gamma = D, H, Hprime, gamma
        self.device = torch.device(device)
        self.ctx = binding.Context(self.kind, D, H, Hprime, gamma, precision, max_points)
        if data_cut:     # ET's data-point cut (BSC, TSC)
            self.ctx.set_data_cut(True)
        self._st = None

    # -------------------------------------------------------------- helpers
    def _y(self, data):
        import torch
        y = data["y"] if isinstance(data, dict) else data
        if isinstance(y, torch.Tensor):
            return y.to(self.device, torch.float32).contiguous()
        return torch.tensor(np.ascontiguousarray(y, np.float32), device=self.device)

    def _P(self, params):
        return self.ctx.params(params["W"], params["theta"], params.get("mu"), params.get("psi"))

    def _pack(self, Wt, pi, sigma, rho=0.0, mu=None, psi=None, pvals=None):
        import torch
        th = np.zeros(binding.THETA_LEN)
        th[:4] = [pi, sigma, rho, 1.0]
        if pvals is not None:
            th[binding.TH_DSC_P:binding.TH_DSC_P + len(pvals)] = pvals
        p = {"W": torch.tensor(np.asarray(Wt, np.float32), device=self.device),
             "theta": torch.tensor(th, dtype=torch.float64, device=self.device)}
        if mu is not None:
            p["mu"] = torch.tensor(np.asarray(mu, np.float32), device=self.device)
            p["psi"] = torch.tensor(np.asarray(psi, np.float32), device=self.device)
        return p

    # ------------------------------------------------------------ interface
    def step(self, anneal, params, data, group=None):
        """One EM iteration (truncated E-step, then M-step) in place on params;
        returns the truncated log-likelihood F of the E-step (host float).
        With a process group (``group``, or the default group when
        torch.distributed is initialised) ``data`` is this rank's shard: the
        statistics are summed over the ranks and every rank runs the same
        M-step on the sums, so the parameters stay identical across ranks."""
        Y = self._y(data)
        if self._st is None:
            self._st = self.ctx.alloc_stats(self.device)
        P = self._P(params)
        params["theta"][binding.TH_T] = float(getattr(anneal, "T", 1.0))
        self.ctx.estep(P, Y, self._st)
        _, world = distributed.process_group_info(group)
        if world > 1:
            distributed.allreduce_stats(self._st, group)
        F = float(self._st["scal"][binding.SC_F].item())
        N = int(round(float(self._st["scal"][binding.SC_N].item())))
        self.ctx.mstep(self._st, N, P)
        return F

    def free_energy(self, params, data):
        Y = self._y(data)
        st = self.ctx.alloc_stats(self.device)
        self.ctx.estep(self._P(params), Y, st)
        return float(st["scal"][binding.SC_F].item())

    def inference(self, anneal, params, data):
        """Per point: res["s"] the most likely state (N x H, 0/1), res["p"] its
        approximate posterior probability, plus the candidates, posterior
        means over them and log p(y) restricted to the truncated set."""
        import torch
        Y = self._y(data)
        out = self.ctx.encode(self._P(params), Y)
        N = Y.shape[0]
        s = torch.zeros(N, self.H, dtype=torch.int8, device=self.device)
        if self.gamma > 0:
            idx = out["map_idx"].long()
            rows = torch.arange(N, device=self.device)[:, None].expand_as(idx)
            ok = idx >= 0
            s[rows[ok], idx[ok]] = 1
        return {"s": s, "p": out["map_p"], "sel": out["sel"], "s_mean": out["s_mean"],
                "logZ": out["logZ"], "map_idx": out["map_idx"]}


class BSC_ET(_Model):
    """Binary sparse coding with truncated posteriors (Table 1, row BSC)."""
    kind = binding.BSC

    def standard_init(self, data, seed=0):
        y = np.asarray(data["y"] if isinstance(data, dict) else data, np.float32)
        p = synth.init_bsc(y, self.H, seed=seed, pi=min(0.5, self.Hprime / (2.0 * self.H) + 0.01),
                           normalise=self.H >= self.D)
        return self._pack(p["Wt"], p["pi"], p["sigma"])


class TSC_ET(_Model):
    """Ternary sparse coding with truncated posteriors (Table 1, row TSC):
    latents in {-1, 0, 1}, p(s_h = +-1) = pi/2."""
    kind = binding.TSC

    def standard_init(self, data, seed=0):
        y = np.asarray(data["y"] if isinstance(data, dict) else data, np.float32)
        p = synth.init_bsc(y, self.H, seed=seed, pi=min(0.5, self.Hprime / (2.0 * self.H) + 0.01),
                           normalise=self.H >= self.D)
        return self._pack(p["Wt"], p["pi"], p["sigma"])


class DSC_ET(_Model):
    """Discrete sparse coding with truncated posteriors (Table 1, row DSC):
    latents in {0, values[0], .., values[m-1]} under a categorical prior."""
    kind = binding.DSC

    def __init__(self, D, H, Hprime, gamma, values, **kw):
        import torch
        self.D, self.H, self.Hprime, self.gamma = D, H, Hprime, gamma
        self.device = torch.device(kw.get("device", "cuda"))
        self.values = np.asarray(values, np.float32)
        self.ctx = binding.Context(binding.DSC, D, H, Hprime, gamma,
                                   max_points=kw.get("max_points", 1 << 20), values=self.values)
        self._st = None

    def standard_init(self, data, seed=0):
        y = np.asarray(data["y"] if isinstance(data, dict) else data, np.float32)
        p = synth.init_bsc(y, self.H, seed=seed, pi=0.1, normalise=self.H >= self.D)
        m = len(self.values)
        pv = np.full(m, min(0.5, self.Hprime / (2.0 * self.H) + 0.01) / m)
        return self._pack(p["Wt"], float(pv.sum()), p["sigma"], pvals=pv)


class MCA_ET(_Model):
    """Maximal causes analysis (Table 1, row MCA); rho is the exponent of the
    smoothed max used by the M-step."""
    kind = binding.MCA

    def __init__(self, D, H, Hprime, gamma, rho=20.0, **kw):
        super().__init__(D, H, Hprime, gamma, **kw)
        self.rho = rho

    def standard_init(self, data, seed=0):
        y = np.asarray(data["y"] if isinstance(data, dict) else data, np.float32)
        p = synth.init_mca(y, self.H, seed=seed)
        return self._pack(p["Wt"], p["pi"], p["sigma"], rho=self.rho)


class MMCA_ET(MCA_ET):
    """Max-magnitude causes analysis (Table 1, row MMCA): per pixel the active
    component of largest |W_dh|; signed dictionary."""
    kind = binding.MMCA

    def standard_init(self, data, seed=0):
        y = np.asarray(data["y"] if isinstance(data, dict) else data, np.float32)
        p = synth.init_bsc(y, self.H, seed=seed, pi=0.1, normalise=False)
        return self._pack(p["Wt"], p["pi"], p["sigma"], rho=self.rho)


class GSC_ET(_Model):
    """Gaussian sparse coding, spike-and-slab prior (Table 1, row GSC)."""
    kind = binding.GSC

    def standard_init(self, data, seed=0):
        y = np.asarray(data["y"] if isinstance(data, dict) else data, np.float32)
        p = synth.init_gsc(y, self.H, seed=seed)
        return self._pack(p["Wt"], p["pi"], p["sigma"], mu=p["mu"], psi=p["psi"])


class EM:
    """Runs ``model.step`` under the annealing schedule (Sec. 3).

    Data parallel (the paper's MPI design, Sec. 1): when torch.distributed is
    initialised (or ``group`` is given) and ``shard`` is True, every rank keeps
    the contiguous block of the data that ``distributed.shard_range`` assigns
    to it, E-steps that block on its own GPU, and the ranks sum their
    statistics before the replicated M-step.  ``shard=False`` means ``data`` is
    already this rank's block.  The initial parameters must be the same on
    every rank (pass ``lparams`` or use the same seed)."""

    def __init__(self, model, anneal, data=None, lparams=None, group=None, shard=True):
        self.model, self.anneal = model, anneal
        self.data, self.lparams = data, lparams
        self.group, self.shard = group, shard
        self.history = []

    def _local(self, data):
        rank, world = distributed.process_group_info(self.group)
        if world == 1 or not self.shard:
            return data
        y = data["y"] if isinstance(data, dict) else data
        a, b = distributed.shard_range(len(y), rank, world)
        return {"y": y[a:b]}

    def run(self, data=None, verbose=False):
        data = data if data is not None else self.data
        if self.lparams is None:
            self.lparams = self.model.standard_init(data)
        local = self._local(data)
        while self.anneal.next():
            F = self.model.step(self.anneal, self.lparams, local, group=self.group)
            self.history.append(F)
            if verbose:
                print(f"iteration {self.anneal.cur}: F = {F:.6f}")
        return self.lparams


def save_params(path, params):
    """Checkpoint: parameters (device tensors) to an .npz file."""
    np.savez(path, **{k: v.detach().cpu().numpy() for k, v in params.items()})


def load_params(path, device="cuda"):
    """Resume: parameters saved by save_params back to device tensors."""
    import torch
    z = np.load(path)
    return {k: torch.tensor(z[k], device=device) for k in z.files}
