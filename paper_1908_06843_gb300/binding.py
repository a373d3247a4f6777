"""Thin ctypes binding of libprosper (include/prosper.h).

Argument marshalling only: every computation runs in the CUDA kernels of the
shared library.  Tensors are torch CUDA tensors (device memory and streams are
the only things torch provides); host-side arrays for the ``*_host`` calls are
numpy arrays or pinned torch CPU tensors.  There is no CPU fallback: if the
library or a GPU is missing, these functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

BSC, MCA, GSC, TSC, DSC, MMCA = 0, 1, 2, 3, 4, 5
FP32, BF16_RESCORE = 0, 1
TH_PI, TH_SIGMA, TH_RHO, TH_T, TH_DSC_P, THETA_LEN = 0, 1, 2, 3, 4, 8
SC_F, SC_S1, SC_YY, SC_N, SC_MCA_R2, SC_DSC0, SC_LEN = 0, 1, 2, 3, 4, 5, 8
MAX_HPRIME, MAX_STATES = 16, 4096

# function name -> (restype, argtypes); the list is the exported C ABI
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
ABI = {
    "prosper_init": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _I, _I64]),
    "prosper_init_dsc": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _P, _I64]),
    "prosper_set_data_cut": (_I, [_P, _I]),
    "prosper_encode_values": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "prosper_destroy": (_I, [_P]),
    "prosper_estep": (_I, [_P, _P, _P, _I64, _P, _P]),
    "prosper_mstep": (_I, [_P, _P, _I64, _P, _P]),
    "prosper_encode": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "prosper_estep_host": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "prosper_last_error": (ctypes.c_char_p, []),
    "prosper_serve_start": (_I, [_P, _P, _I, _I]),
    "prosper_serve_submit": (_I, [_P, _P, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "prosper_serve_wait": (_I, [_P, ctypes.c_uint64, _I, _P, _P, _P, _P, _P,
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "prosper_serve_stop": (_I, [_P]),
    "prosper_serve_loadgen": (_I, [_P, _P, _I64, _I, _P, _P, _P, _P, _P, _P]),
    "prosper_encode_noalloc": (_I, [_I, _I, _I, _I, _P, _P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "prosper_status": (_I, [_P, _P]),
    "prosper_trace_enable": (_I, [_P, _I]),
    "prosper_trace_read": (_I, [_P, _I, _P, _P, _P]),
}


class Params(ctypes.Structure):
    _fields_ = [("W", _P), ("theta", _P), ("mu", _P), ("psi", _P)]


class Stats(ctypes.Structure):
    _fields_ = [("At", _P), ("B", _P), ("scal", _P), ("gsc", _P), ("mca", _P)]


_lib = None
_lock = threading.Lock()


class ProsperError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libprosper.so (building it first if needed) and declare the ABI."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise ProsperError(f"libprosper not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in ABI.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().prosper_last_error().decode(errors="replace")
        raise ProsperError(f"{what} failed ({rc}): {msg}")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(_P)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ProsperError("expected a CUDA tensor")
        if t is not None and not t.is_contiguous():
            raise ProsperError("expected a contiguous tensor")


class Context:
    """Owns a prosper_ctx (one model and approximation, paper Sec. 3:
    BSC_ET(D, H, Hprime, gamma)).  DSC contexts take ``values``: the m <= 3
    nonzero latent values (prosper_init_dsc)."""

    def __init__(self, model, D, H, Hprime, gamma, precision=FP32, max_points=1 << 20,
                 values=None):
        self.lib = load()
        self.model, self.D, self.H, self.Hp, self.gamma = model, D, H, Hprime, gamma
        self.precision = precision
        h = _P()
        if model == DSC:
            vals = np.ascontiguousarray(values, np.float32)
            self.values = vals
            _check(self.lib.prosper_init_dsc(ctypes.byref(h), D, H, Hprime, gamma, len(vals),
                                             _ptr(vals), int(max_points)), "prosper_init_dsc")
        else:
            self.values = np.array([-1.0, 1.0] if model == TSC else [1.0], np.float32)
            _check(self.lib.prosper_init(ctypes.byref(h), model, D, H, Hprime, gamma, precision,
                                         int(max_points)), "prosper_init")
        self.h = h

    def set_data_cut(self, on=True):
        """ET's data-point cut on the following E-steps (prosper_set_data_cut)."""
        _check(self.lib.prosper_set_data_cut(self.h, 1 if on else 0), "prosper_set_data_cut")

    def close(self):
        if getattr(self, "h", None):
            self.lib.prosper_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- helpers
    def params(self, W, theta, mu=None, psi=None) -> Params:
        """prosper_params pointing at these device tensors.  The struct keeps
        references to them, so they stay allocated while it is in use."""
        _require_cuda(W, theta, mu, psi)
        P = Params(_ptr(W), _ptr(theta), _ptr(mu), _ptr(psi))
        P._tensors = (W, theta, mu, psi)
        return P

    def alloc_stats(self, device="cuda"):
        import torch
        H, D = self.H, self.D
        f64 = dict(dtype=torch.float64, device=device)
        st = dict(At=torch.zeros(H, D, **f64), B=torch.zeros(H, H, **f64),
                  scal=torch.zeros(SC_LEN, **f64),
                  gsc=torch.zeros(3 * H, **f64) if self.model == GSC else None,
                  mca=torch.zeros(2, H, D, **f64) if self.model in (MCA, MMCA) else None)
        return st

    @staticmethod
    def _stats_struct(st) -> Stats:
        return Stats(_ptr(st["At"]), _ptr(st["B"]), _ptr(st["scal"]), _ptr(st.get("gsc")),
                     _ptr(st.get("mca")))

    # -------------------------------------------------------------- C ABI
    def estep(self, P: Params, Y, st, stream=None):
        _require_cuda(Y)
        S = self._stats_struct(st)
        _check(self.lib.prosper_estep(self.h, ctypes.byref(P), _ptr(Y), int(Y.shape[0]),
                                      ctypes.byref(S), _stream(stream)), "prosper_estep")
        return st

    def mstep(self, st, N, P: Params, stream=None):
        S = self._stats_struct(st)
        _check(self.lib.prosper_mstep(self.h, ctypes.byref(S), int(N), ctypes.byref(P),
                                      _stream(stream)), "prosper_mstep")

    def encode(self, P: Params, Y, out=None, stream=None):
        """Per-point encoding (prosper_encode; TSC/DSC: prosper_encode_values,
        which adds map_val, the values of the MAP state's units)."""
        import torch
        _require_cuda(Y)
        N = int(Y.shape[0])
        discrete = self.model in (TSC, DSC)
        if out is None:
            dev = Y.device
            out = dict(sel=torch.empty(N, self.Hp, dtype=torch.int16, device=dev),
                       s_mean=torch.empty(N, self.Hp, dtype=torch.float32, device=dev),
                       map_idx=torch.empty(N, self.gamma, dtype=torch.int16, device=dev),
                       map_p=torch.empty(N, dtype=torch.float32, device=dev),
                       logZ=torch.empty(N, dtype=torch.float32, device=dev))
            if discrete:
                out["map_val"] = torch.empty(N, self.gamma, dtype=torch.float32, device=dev)
        g = self.gamma > 0
        if discrete:
            _check(self.lib.prosper_encode_values(
                self.h, ctypes.byref(P), _ptr(Y), N, _ptr(out["sel"]), _ptr(out["s_mean"]),
                _ptr(out["map_idx"]) if g else None, _ptr(out["map_val"]) if g else None,
                _ptr(out["map_p"]), _ptr(out["logZ"]), _stream(stream)), "prosper_encode_values")
            return out
        _check(self.lib.prosper_encode(self.h, ctypes.byref(P), _ptr(Y), N, _ptr(out["sel"]),
                                       _ptr(out["s_mean"]),
                                       _ptr(out["map_idx"]) if g else None,
                                       _ptr(out["map_p"]), _ptr(out["logZ"]), _stream(stream)),
               "prosper_encode")
        return out

    def estep_host(self, P: Params, Y_host, At_host=None, B_host=None, scal_host=None,
                   stream=None):
        """E-step from host data; statistics returned in host arrays (synchronous)."""
        N = int(Y_host.shape[0])
        if At_host is None:
            At_host = np.zeros((self.H, self.D))
            B_host = np.zeros((self.H, self.H))
            scal_host = np.zeros(SC_LEN)
        _check(self.lib.prosper_estep_host(self.h, ctypes.byref(P), _ptr(Y_host), N,
                                           _ptr(At_host), _ptr(B_host), _ptr(scal_host),
                                           _stream(stream)), "prosper_estep_host")
        return dict(At=At_host, B=B_host, scal=scal_host)

    def status(self, stream=None):
        """Synchronise and report kernel-flagged failures (raises ProsperError)."""
        _check(self.lib.prosper_status(self.h, _stream(stream)), "prosper_status")

    # ------------------------------------------------------------- tracing
    def trace_enable(self, on=True):
        _check(self.lib.prosper_trace_enable(self.h, 1 if on else 0), "prosper_trace_enable")

    def trace_read(self, max_kernels=32):
        """{kernel name: (total ms, launches)} since the last read (synchronises)."""
        names = ctypes.create_string_buffer(48 * max_kernels)
        ms = np.zeros(max_kernels)
        cnt = np.zeros(max_kernels, np.int32)
        k = self.lib.prosper_trace_read(self.h, max_kernels, names, _ptr(ms), _ptr(cnt))
        if k < 0:
            _check(k, "prosper_trace_read")
        raw = names.raw
        return {raw[48 * i:48 * i + 48].split(b"\0")[0].decode(): (float(ms[i]), int(cnt[i]))
                for i in range(k)}

    # ------------------------------------------------------------- serving
    def serve_start(self, P: Params, n_slots=4, slot_points=8192):
        self._serve_params = P
        _check(self.lib.prosper_serve_start(self.h, ctypes.byref(P), n_slots, slot_points),
               "prosper_serve_start")

    def serve_submit(self, Y_host: np.ndarray) -> int:
        Y_host = np.ascontiguousarray(Y_host, dtype=np.float32)
        t = ctypes.c_uint64()
        _check(self.lib.prosper_serve_submit(self.h, _ptr(Y_host), int(Y_host.shape[0]),
                                             ctypes.byref(t)), "prosper_serve_submit")
        return t.value

    def serve_wait(self, ticket: int, n: int, timeout_ms: int = -1):
        out = dict(sel=np.empty((n, self.Hp), np.int16), s_mean=np.empty((n, self.Hp), np.float32),
                   map_idx=np.empty((n, self.gamma), np.int16), map_p=np.empty(n, np.float32),
                   logZ=np.empty(n, np.float32))
        ts, td = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.prosper_serve_wait(self.h, ticket, timeout_ms, _ptr(out["sel"]),
                                           _ptr(out["s_mean"]),
                                           _ptr(out["map_idx"]) if self.gamma > 0 else None,
                                           _ptr(out["map_p"]), _ptr(out["logZ"]),
                                           ctypes.byref(ts), ctypes.byref(td)),
               "prosper_serve_wait")
        out["t_submit_ns"], out["t_done_ns"] = ts.value, td.value
        return out

    def serve_loadgen(self, Y_pool: np.ndarray, sizes, offsets, arrival_s):
        """Native open-loop load (prosper_serve_loadgen): request i of sizes[i]
        rows of Y_pool from offsets[i], submitted arrival_s[i] seconds after the
        start.  Returns per-request (t_submit, t_observed, t_done) in ns."""
        Y_pool = np.ascontiguousarray(Y_pool, dtype=np.float32)
        sizes = np.ascontiguousarray(sizes, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        arr = np.ascontiguousarray(np.round(np.asarray(arrival_s) * 1e9), dtype=np.int64)
        n = len(sizes)
        ts, to, td = (np.zeros(n, np.int64) for _ in range(3))
        _check(self.lib.prosper_serve_loadgen(self.h, _ptr(Y_pool), int(Y_pool.shape[0]), n,
                                              _ptr(sizes), _ptr(offsets), _ptr(arr), _ptr(ts),
                                              _ptr(to), _ptr(td)), "prosper_serve_loadgen")
        return ts, to, td

    def serve_stop(self):
        _check(self.lib.prosper_serve_stop(self.h), "prosper_serve_stop")
