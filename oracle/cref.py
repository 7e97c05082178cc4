"""ctypes wrapper of fs1_ref.c, the sequential FP64 FS-1 in plain C.

Test infrastructure only (see ``oracle/__init__.py``).  ``build()`` compiles the
C file with the host compiler into ``oracle/_build/``; nothing here touches a
GPU.  Calls release the GIL (ctypes), so a thread pool runs pairs on several
host cores at once.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fs1_ref.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfs1_oracle.so")

OK, EINVAL, ENOMEM, ENUMERIC = 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> str:
    """Compile fs1_ref.c (no FMA contraction, so x86 and Arm hosts round alike)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        cc = os.environ.get("CC", "cc")
        subprocess.check_call([cc, "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.fs1ref_solve.restype = ctypes.c_int
        L.fs1ref_solve.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_long, ctypes.c_double,
                                   dp, ctypes.POINTER(ctypes.c_long), dp, dp, dp]
        L.fs1ref_matvec.restype = ctypes.c_int
        L.fs1ref_matvec.argtypes = [dp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int]
        _lib = L
    return _lib


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclasses.dataclass
class RefResult:
    status: int
    w: float
    iters: int
    err: float
    f: Optional[np.ndarray] = None
    g: Optional[np.ndarray] = None


def _axes(shape, h):
    """(n1, n2, n3) fast to slow and (h1, h2, h3) of a 1D, 2D or 3D array."""
    if len(shape) == 1:
        return (shape[0], 1, 1), (float(h[0] if isinstance(h, (tuple, list)) else h), 0.0, 0.0)
    if len(shape) == 2:
        return (shape[1], shape[0], 1), (float(h[0]), float(h[1]), 0.0)
    return (shape[2], shape[1], shape[0]), (float(h[0]), float(h[1]), float(h[2]))


def solve(a, b, h, eps: float, tol: float, itr_max: int, tau: float = 1e10,
          potentials: bool = False) -> RefResult:
    """Run FS-1 on one pair.  1D: a, b of shape (n,), h a float or (h,).
    2D: a, b of shape (n_slow, n_fast), h = (h_fast, h_slow).  3D: shape
    (n_slow, n_mid, n_fast), h = (h_fast, h_mid, h_slow).  tau = inf selects
    the plain form of Algorithm 1 / 2; a finite tau the stabilised form
    (requires a, b > 0)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    (n1, n2, n3), (h1, h2, h3) = _axes(a.shape, h)
    w = ctypes.c_double()
    it = ctypes.c_long()
    e = ctypes.c_double()
    f = np.empty(a.size) if potentials else None
    g = np.empty(a.size) if potentials else None
    st = lib().fs1ref_solve(_p(a), _p(b), n1, n2, n3, h1, h2, h3, float(eps), float(tol), int(itr_max),
                            float(tau), ctypes.byref(w), ctypes.byref(it), ctypes.byref(e),
                            _p(f) if f is not None else None, _p(g) if g is not None else None)
    if f is not None and a.ndim > 1:
        f = f.reshape(a.shape)
        g = g.reshape(a.shape)
    return RefResult(st, w.value, it.value, e.value, f, g)


def solve_many(pairs: Sequence, workers: int = 0, **kw):
    """Run solve() over (a, b, h, eps, tol, itr_max) tuples on a thread pool."""
    workers = workers or max(1, len(os.sched_getaffinity(0)))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(solve, *p, **kw) for p in pairs]
        return [fu.result() for fu in futs]


def matvec(x, h, eps: float, weighted_fast: bool = False, weighted_slow: bool = False,
           weighted_axes: int = -1):
    """K x with the plain recurrences (1D: x of shape (n,); 2D: (n_slow,
    n_fast); 3D: (n_slow, n_mid, n_fast)).  Distance-weighted along the fast /
    slow axis of a 2D array by the flags, or along the axes in the bit mask
    weighted_axes (bit 0 fast, 1 middle, 2 slow) when it is given."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    (n1, n2, n3), (h1, h2, h3) = _axes(x.shape, h)
    if weighted_axes < 0:
        weighted_axes = int(weighted_fast) | (int(weighted_slow) << (1 if x.ndim <= 2 else 2))
    y = np.empty_like(x)
    st = lib().fs1ref_matvec(_p(x), _p(y), n1, n2, n3, h1, h2, h3, float(eps), int(weighted_axes))
    assert st == OK
    return y
