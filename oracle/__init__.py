"""FP64 CPU oracle for the temporally parallel Kalman filter / RTS smoother.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  The product path (``paper_1905_13002_gb300``) never does, and this
package imports nothing from it.

Contents
--------
* ``kf``, ``rts``, ``kf_rts`` -- the sequential Kalman filter and RTS smoother
  (Section II-A; the k = 1 equations of Lemma 3 applied at every step, and the
  RTS gain of Lemma 5), written in plain C (``kf_rts.c``) and called through
  ctypes.  By Theorems 1 and 2 these are exactly the filtering and smoothing
  posteriors the parallel scans must reach.
* ``oracle.lemmas`` -- Lemmas 3-6 (elements and combine operators of Section
  IV), the all-prefix-sums definition (Section II-B) and the suffix scan of
  Theorem 2, in numpy FP64, used to check the GPU's element builders and
  operators one by one.

Inputs are promoted to FP64 from the FP32 values the GPU reads, so measured
differences are arithmetic error, not input quantisation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_rts.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libks_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2, no fast-math) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    D = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_kf.argtypes = [ctypes.c_int, ctypes.c_int, i64,
                              D, i64, D, i64, D, i64, D, i64, D, i64, D, i64,
                              D, D, D, D, D, D]
    lib.oracle_kf.restype = ctypes.c_int
    lib.oracle_rts.argtypes = [ctypes.c_int, i64, D, i64, D, i64, D, i64, D, D, D, D]
    lib.oracle_rts.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _param(a, T, shape):
    """Return (contiguous float64 array, per-step stride) for a model parameter
    given either time-invariant ``shape`` or time-varying ``(T,) + shape``."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    size = int(np.prod(shape)) if shape else 1
    if a.shape == tuple(shape):
        return a, 0
    if a.shape == (T,) + tuple(shape):
        return a, size
    raise ValueError(f"parameter shape {a.shape} is neither {shape} nor {(T,) + tuple(shape)}")


def kf(model, y, loglik: bool = False):
    """Sequential Kalman filter in FP64.

    ``model`` has attributes F, u, Q, H, d, R (time-invariant or with a leading
    T axis), m0, P0.  ``y`` is [T, ny].  Returns (fmean[T,nx], fcov[T,nx,nx])
    and, with ``loglik``, the per-step log p(y_k | y_{1:k-1}).
    """
    lib = _load()
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    T, ny = y.shape
    nx = np.asarray(model.m0).shape[0]
    F, sF = _param(model.F, T, (nx, nx))
    u, su = _param(model.u, T, (nx,))
    Q, sQ = _param(model.Q, T, (nx, nx))
    H, sH = _param(model.H, T, (ny, nx))
    d, sd = _param(model.d, T, (ny,))
    R, sR = _param(model.R, T, (ny, ny))
    m0 = np.ascontiguousarray(model.m0, dtype=np.float64)
    P0 = np.ascontiguousarray(model.P0, dtype=np.float64)
    fm = np.empty((T, nx))
    fP = np.empty((T, nx, nx))
    ll = np.empty(T) if loglik else None
    rc = lib.oracle_kf(nx, ny, T, _ptr(F), sF, _ptr(u), su, _ptr(Q), sQ, _ptr(H), sH,
                       _ptr(d), sd, _ptr(R), sR, _ptr(m0), _ptr(P0), _ptr(y),
                       _ptr(fm), _ptr(fP), _ptr(ll))
    if rc:
        raise FloatingPointError(f"oracle_kf failed with code {rc}")
    return (fm, fP, ll) if loglik else (fm, fP)


def rts(model, fmean, fcov):
    """RTS smoother in FP64 from filtered means [T,nx] and covariances [T,nx,nx]."""
    lib = _load()
    fm = np.ascontiguousarray(np.asarray(fmean, dtype=np.float64))
    fP = np.ascontiguousarray(np.asarray(fcov, dtype=np.float64))
    T, nx = fm.shape
    F, sF = _param(model.F, T, (nx, nx))
    u, su = _param(model.u, T, (nx,))
    Q, sQ = _param(model.Q, T, (nx, nx))
    sm = np.empty_like(fm)
    sP = np.empty_like(fP)
    rc = lib.oracle_rts(nx, T, _ptr(F), sF, _ptr(u), su, _ptr(Q), sQ,
                        _ptr(fm), _ptr(fP), _ptr(sm), _ptr(sP))
    if rc:
        raise FloatingPointError(f"oracle_rts failed with code {rc}")
    return sm, sP


def kf_rts(model, y):
    """Filter then smoother: returns (fmean, fcov, smean, scov), all FP64."""
    fm, fP = kf(model, y)
    sm, sP = rts(model, fm, fP)
    return fm, fP, sm, sP
