"""Thin Python binding of the FS-1 C ABI (include/fs1.h), via ctypes.

Argument marshalling only: every step of the solve runs in the CUDA library
``_build/libfs1.so``.  The names mirror the C functions (fs1_create, fs1_w1,
fs1_solve_batch, fs1_kernel_apply_log, fs1_destroy); ``Solver`` wraps a handle
for torch tensors.  There is no CPU fallback: if the library is missing this
module raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, byref, c_char_p, c_double, c_float, c_int, c_int64,
                    c_longlong, c_size_t, c_void_p)
from typing import List, Optional, Sequence

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libfs1.so")

FS1_OK, FS1_EINVAL, FS1_ENOMEM, FS1_ENUMERIC, FS1_ETIMEOUT, FS1_ENOTCONV, FS1_ECUDA, \
    FS1_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "FS1_OK", 1: "FS1_EINVAL", 2: "FS1_ENOMEM", 3: "FS1_ENUMERIC",
                4: "FS1_ETIMEOUT", 5: "FS1_ENOTCONV", 6: "FS1_ECUDA", 7: "FS1_EUNSUPPORTED"}
FS1_VARIANT_PLAIN, FS1_VARIANT_LOG, FS1_VARIANT_PAPER = 0, 1, 2
FS1_FP64, FS1_FP32 = 0, 1
FS1_MEM_DEVICE, FS1_MEM_HOST = 0, 1


class fs1_config(Structure):
    _fields_ = [("variant", c_int), ("precision", c_int), ("check_every", c_int),
                ("team_size", c_int), ("spin_cap", c_longlong), ("hbm_budget", c_size_t),
                ("stream", c_void_p), ("autotune", c_int), ("trial_iters", c_int),
                ("use_graph", c_int), ("tau", c_double), ("grid2d", c_int), ("units", c_int)]


class fs1_problem(Structure):
    _fields_ = [("ndim", c_int), ("dtype", c_int), ("location", c_int), ("reserved", c_int),
                ("n", c_int64 * 3), ("h", c_double * 3), ("eps", c_double), ("tol", c_double),
                ("itr_max", c_int64), ("a", c_void_p), ("b", c_void_p), ("f_out", c_void_p),
                ("g_out", c_void_p), ("f_init", c_void_p), ("g_init", c_void_p)]


class fs1_info(Structure):
    _fields_ = [("status", c_int), ("variant", c_int), ("precision", c_int),
                ("team_size", c_int), ("iters", c_int64), ("marginal_err", c_double),
                ("w1", c_double), ("ms", c_float), ("reserved", c_float)]


EXPORTED = ["fs1_config_default", "fs1_create", "fs1_w1", "fs1_solve_batch",
            "fs1_kernel_apply_log", "fs1_destroy", "fs1_status_string", "fs1_version",
            "fs1_launch_count", "fs1_w1_noalloc", "fs1_handle_stats",
            "fs1_handle_launch_stats", "fs1_test_missing_partner"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"FS-1 CUDA library not built ({path}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    L.fs1_config_default.argtypes = [POINTER(fs1_config)]
    L.fs1_config_default.restype = c_int
    L.fs1_create.argtypes = [POINTER(fs1_config), POINTER(c_void_p)]
    L.fs1_create.restype = c_int
    L.fs1_w1.argtypes = [c_void_p, POINTER(fs1_problem), POINTER(c_double), POINTER(fs1_info)]
    L.fs1_w1.restype = c_int
    L.fs1_solve_batch.argtypes = [c_void_p, POINTER(fs1_problem), c_int64, POINTER(c_double),
                                  POINTER(fs1_info)]
    L.fs1_solve_batch.restype = c_int
    L.fs1_kernel_apply_log.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_double, c_double]
    L.fs1_kernel_apply_log.restype = c_int
    L.fs1_test_missing_partner.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_double, c_double, c_longlong,
                                           POINTER(c_int)]
    L.fs1_test_missing_partner.restype = c_int
    L.fs1_destroy.argtypes = [c_void_p]
    L.fs1_destroy.restype = None
    L.fs1_status_string.argtypes = [c_int]
    L.fs1_status_string.restype = c_char_p
    L.fs1_version.argtypes = []
    L.fs1_version.restype = c_char_p
    L.fs1_launch_count.argtypes = []
    L.fs1_launch_count.restype = c_int64
    L.fs1_w1_noalloc.argtypes = [POINTER(fs1_config), POINTER(fs1_problem), POINTER(c_double),
                                 POINTER(fs1_info)]
    L.fs1_w1_noalloc.restype = c_int
    L.fs1_handle_stats.argtypes = [c_void_p, POINTER(c_int64)]
    L.fs1_handle_stats.restype = c_int
    L.fs1_handle_launch_stats.argtypes = [c_void_p, POINTER(c_int64)]
    L.fs1_handle_launch_stats.restype = c_int
    _lib = L
    return L


# ---- C-named wrappers -------------------------------------------------------

def fs1_config_default() -> fs1_config:
    cfg = fs1_config()
    _check(load().fs1_config_default(ctypes.byref(cfg)))
    return cfg


def fs1_create(cfg: Optional[fs1_config] = None) -> c_void_p:
    h = c_void_p()
    st = load().fs1_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h))
    _check(st)
    return h


def fs1_destroy(h: c_void_p) -> None:
    load().fs1_destroy(h)


def fs1_w1(h, prob: fs1_problem):
    w = c_double()
    info = fs1_info()
    st = load().fs1_w1(h, ctypes.byref(prob), ctypes.byref(w), ctypes.byref(info))
    return st, w.value, info


def fs1_solve_batch(h, probs: Sequence[fs1_problem]):
    n = len(probs)
    arr = (fs1_problem * n)(*probs)
    w = (c_double * n)()
    infos = (fs1_info * n)()
    st = load().fs1_solve_batch(h, arr, n, w, infos)
    return st, np.frombuffer(w, dtype=np.float64).copy(), list(infos)


def fs1_kernel_apply_log(h, in_ptr: int, out_ptr: int, n: int, hx: float, eps: float) -> int:
    return load().fs1_kernel_apply_log(h, c_void_p(in_ptr), c_void_p(out_ptr), int(n),
                                       float(hx), float(eps))


def fs1_test_missing_partner(h, a_ptr: int, b_ptr: int, n: int, hx: float, eps: float, spin_cap: int):
    """(status of the call, status of the pair): a pair on a team of two CTAs
    of which only one runs gives up its bounded waits (FS1_ETIMEOUT)."""
    ps = c_int(-1)
    st = load().fs1_test_missing_partner(h, c_void_p(a_ptr), c_void_p(b_ptr), int(n), float(hx), float(eps),
                                         int(spin_cap), byref(ps))
    return st, ps.value


def fs1_status_string(s: int) -> str:
    return load().fs1_status_string(int(s)).decode()


def fs1_version() -> str:
    return load().fs1_version().decode()


def fs1_launch_count() -> int:
    return int(load().fs1_launch_count())


def fs1_handle_stats(h) -> dict:
    out = (c_int64 * 4)()
    _check(load().fs1_handle_stats(h, out))
    out2 = (c_int64 * 2)()
    _check(load().fs1_handle_launch_stats(h, out2))
    return {"graph_replays": out[0], "graphs_captured": out[1], "tuned_classes": out[2],
            "trial_launches": out[3], "exact_launches": out2[0], "last_exact_E": out2[1]}


def fs1_w1_noalloc(cfg: Optional[fs1_config], prob: fs1_problem):
    """One device-located 1D problem through the allocation-free entry point."""
    w = c_double()
    info = fs1_info()
    st = load().fs1_w1_noalloc(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(prob),
                               ctypes.byref(w), ctypes.byref(info))
    return st, w.value, info


def _check(st: int) -> None:
    if st != FS1_OK:
        raise RuntimeError(f"fs1 call failed: {STATUS_NAMES.get(st, st)}")


# ---- convenience wrapper for torch tensors ------------------------------------

class Solver:
    """One library handle.  `variant` is "log" (stabilised, FP32), "plain"
    (FP32 or FP64) or "paper" (the Remarks' tau-triggered absorption as
    written, FP64, 1D); `precision` "fp32" or "fp64"."""

    def __init__(self, variant: str = "log", precision: str = "fp32", team_size: int = 0,
                 stream=None, spin_cap: int = 0, hbm_budget: int = 0, autotune: bool = True,
                 use_graph: bool = True, trial_iters: int = 0, tau: float = 0.0, grid2d: bool = False,
                 units: bool = True):
        cfg = fs1_config_default()
        cfg.variant = {"log": FS1_VARIANT_LOG, "plain": FS1_VARIANT_PLAIN, "paper": FS1_VARIANT_PAPER}[variant]
        cfg.precision = FS1_FP32 if precision == "fp32" else FS1_FP64
        cfg.team_size = int(team_size)
        if spin_cap:
            cfg.spin_cap = int(spin_cap)
        cfg.hbm_budget = int(hbm_budget)
        cfg.autotune = 1 if autotune else 0
        cfg.use_graph = 1 if use_graph else 0
        if tau:
            cfg.tau = float(tau)
        cfg.grid2d = 1 if grid2d else 0
        cfg.units = 1 if units else 0
        if trial_iters:
            cfg.trial_iters = int(trial_iters)
        if stream is not None:
            cfg.stream = c_void_p(int(stream))
        self.cfg = cfg
        self.h = fs1_create(cfg)

    def close(self):
        if self.h is not None:
            fs1_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def problem(a, b, h, eps: float, tol: float, itr_max: int, f_out=None, g_out=None,
                f_init=None, g_init=None, shape=None) -> fs1_problem:
        """Build an fs1_problem from torch tensors (CUDA: device location; CPU:
        host location).  1D: a, b of shape (n,), h a float.  2D: a, b of shape
        (n_slow, n_fast), h = (h_fast, h_slow).  3D: shape (n_slow, n_mid,
        n_fast), h = (h_fast, h_mid, h_slow)."""
        import torch
        p = fs1_problem()
        p.ndim = a.dim()
        assert 1 <= p.ndim <= 3
        hs = tuple(h) if isinstance(h, (tuple, list)) else (h,)
        for ax in range(3):
            p.n[ax] = a.shape[p.ndim - 1 - ax] if ax < p.ndim else 1
            p.h[ax] = float(hs[ax]) if ax < p.ndim else 0.0
        assert a.dtype == b.dtype and a.is_contiguous() and b.is_contiguous()
        p.dtype = FS1_FP32 if a.dtype == torch.float32 else FS1_FP64
        p.location = FS1_MEM_DEVICE if a.is_cuda else FS1_MEM_HOST
        p.eps = float(eps)
        p.tol = float(tol)
        p.itr_max = int(itr_max)
        p.a = a.data_ptr()
        p.b = b.data_ptr()
        for name, t in (("f_out", f_out), ("g_out", g_out), ("f_init", f_init), ("g_init", g_init)):
            if t is not None:
                assert t.dtype == torch.float64 and t.is_contiguous()
                setattr(p, name, t.data_ptr())
        return p

    def solve(self, probs: Sequence[fs1_problem]):
        st, w, infos = fs1_solve_batch(self.h, probs)
        return st, w, infos

    def stats(self) -> dict:
        return fs1_handle_stats(self.h)
