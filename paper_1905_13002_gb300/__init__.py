"""GB300 temporally parallel Kalman filter / RTS smoother.

Python binding of ``libks`` (C ABI in ``include/ks.h``), the CUDA
implementation of the parallel linear/Gaussian filter and smoother of
Särkkä & García-Fernández, "Temporal Parallelization of Bayesian Smoothers"
(Section IV): Lemma 3 / Lemma 4 elements and operator scanned forward
(Theorem 1), Lemma 5 / Lemma 6 elements and operator scanned in reverse
(Theorem 2).

This module only marshals arguments: it passes torch CUDA tensors (device
memory) and the current torch stream to the library, whose kernels do every
step.  There is no CPU fallback; if the library is not built, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

__all__ = [
    "KsError", "Model", "ModelBatch", "smooth_batch", "workspace_bytes_batch", "smooth_batched",
    "workspace_bytes_batched", "lib", "workspace_bytes", "alloc_workspace", "smooth", "build_elements",
    "elements", "filter_scan", "smooth_scan", "status", "refinements", "filter_combine_batch",
    "smoother_combine_batch", "supported", "KS_WS_SMOOTH", "KS_WS_ELEMENTS",
    "HmmModel", "hmm_supported", "hmm_workspace_bytes", "hmm_smooth",
]

KS_OK, KS_EINVAL, KS_ECUDA, KS_ENUMERIC, KS_ETIMEOUT, KS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
KS_WS_SMOOTH, KS_WS_ELEMENTS = 0, 1

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libks.so")


class KsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().ks_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


class _KsModel(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("time_varying", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("F", ctypes.c_void_p), ("u", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("d", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("m0", ctypes.c_void_p), ("P0", ctypes.c_void_p)]


class _KsModelBatch(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("B", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("F", ctypes.c_void_p), ("u", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("d", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("m0", ctypes.c_void_p), ("P0", ctypes.c_void_p), ("offsets", ctypes.c_void_p)]


class _KsBatchGroup(ctypes.Structure):
    _fields_ = [("models", _KsModelBatch), ("total_T", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("fmean", ctypes.c_void_p), ("fcov", ctypes.c_void_p), ("smean", ctypes.c_void_p),
                ("scov", ctypes.c_void_p)]


class _KsChunkRule(ctypes.Structure):
    _fields_ = [("T_below", ctypes.c_int64), ("steps", ctypes.c_int32), ("fold", ctypes.c_int32)]


class _KsHmm(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("reserved", ctypes.c_int32), ("pi", ctypes.c_void_p),
                ("Pi", ctypes.c_void_p)]


class _KsLayout(ctypes.Structure):
    _fields_ = [("ld", ctypes.c_int64), ("offset_A", ctypes.c_int64), ("offset_b", ctypes.c_int64),
                ("offset_C", ctypes.c_int64), ("offset_eta", ctypes.c_int64),
                ("offset_J", ctypes.c_int64)]


_lib = None


def lib():
    """Load libks.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libks is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int
        M = ctypes.POINTER(_KsModel)
        sig = {
            "ks_version": ([], i32),
            "ks_supported": ([i32, i32], i32),
            "ks_strerror": ([i32], ctypes.c_char_p),
            "ks_workspace_bytes": ([M, i64, i32], sz),
            "ks_workspace_init": ([vp, sz, vp], i32),
            "ks_elements_layout_get": ([M, i64, ctypes.POINTER(_KsLayout)], i32),
            "ks_build_elements": ([M, vp, i64, vp, sz, vp], i32),
            "ks_filter_scan": ([M, i64, vp, sz, vp, vp, vp], i32),
            "ks_smooth_scan": ([M, i64, vp, vp, vp, sz, vp, vp, vp], i32),
            "ks_smooth": ([M, vp, i64, vp, sz, vp, vp, vp, vp, vp], i32),
            "ks_smooth_traced": ([M, vp, i64, vp, sz, vp, vp, vp, vp, vp, ctypes.POINTER(vp)], i32),
            "ks_status": ([vp, vp], i32),
            "ks_refinements": ([vp, vp, ctypes.POINTER(ctypes.c_uint32)], i32),
            "ks_workspace_set_waits": ([vp, sz, ctypes.c_uint32, ctypes.c_uint32, vp], i32),
            "ks_workspace_bytes_batch": ([i32, i32, i32, i64], sz),
            "ks_smooth_batch": ([ctypes.POINTER(_KsModelBatch), vp, i64, vp, sz, vp, vp, vp, vp, vp], i32),
            "ks_workspace_bytes_batched": ([i32, ctypes.POINTER(_KsBatchGroup)], sz),
            "ks_set_chunk_rules": ([i32, i32, ctypes.POINTER(_KsChunkRule)], i32),
            "ks_chunk_steps": ([i32, i64], i32),
            "ks_chunk_fold": ([i32, i64], i32),
            "ks_smooth_batched": ([i32, ctypes.POINTER(_KsBatchGroup), vp, sz, vp], i32),
            "ks_filter_combine_batch": ([i32, i64, vp, vp, vp, vp, sz, vp], i32),
            "ks_smoother_combine_batch": ([i32, i64, vp, vp, vp, vp, sz, vp], i32),
            "ks_workspace_bytes_aggregate": ([M, i64], sz),
            "ks_loglik": ([M, vp, i64, vp, vp, vp, vp, vp, vp], i32),
            "ks_filter_aggregate": ([M, vp, i64, i32, vp, sz, vp, vp], i32),
            "ks_smoother_aggregate": ([M, i64, vp, vp, i32, vp, sz, vp, vp], i32),
            "ks_hmm_supported": ([i32], i32),
            "ks_hmm_workspace_bytes": ([i32, i64], sz),
            "ks_hmm_smooth": ([ctypes.POINTER(_KsHmm), vp, i64, vp, sz, vp, vp, vp, vp], i32),
            "ks_hmm_smooth_traced": ([ctypes.POINTER(_KsHmm), vp, i64, vp, sz, vp, vp, vp, vp,
                                      ctypes.POINTER(vp)], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        from . import tune
        tune.load_default()
    return _lib


def set_chunk_rules(nx: int, rules) -> None:
    """Block-length table of one state size (``ks_set_chunk_rules``): rules
    are (T_below, steps, fold) triples (fold 1: the linear block fold); an
    empty list restores the built-in table."""
    arr = (_KsChunkRule * max(len(rules), 1))()
    for i, (tb, steps, fold) in enumerate(rules):
        arr[i].T_below, arr[i].steps, arr[i].fold = int(tb), int(steps), int(fold)
    _check(lib().ks_set_chunk_rules(nx, len(rules), arr), "ks_set_chunk_rules")


def chunk_steps(nx: int, T: int) -> int:
    """Steps per thread a call of T steps of state size nx uses (0: mixed batches)."""
    return int(lib().ks_chunk_steps(nx, T))


def chunk_fold(nx: int, T: int) -> int:
    """1 if a call of T steps of state size nx folds full blocks with the
    linear block fold, else 0."""
    return int(lib().ks_chunk_fold(nx, T))


def _check(rc: int, what: str):
    if rc != KS_OK:
        raise KsError(rc, what)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(x, dtype, device):
    t = torch.as_tensor(x, dtype=dtype, device=device)
    return t.contiguous()


@dataclass
class Model:
    """Device-resident linear/Gaussian model (Sections II and IV).

    Time-invariant: F [nx,nx], u [nx], Q [nx,nx], H [ny,nx], d [ny], R [ny,ny]
    FP32.  Time-varying: the same with a leading step axis, F [T,nx,nx] ...
    (F[k], u[k], Q[k] predict step k from step k-1, F[0] from the prior;
    H[k], d[k], R[k] observe step k).  m0 [nx], P0 [nx,nx] are FP64 (the
    k = 1 element is built in FP64).
    """

    F: torch.Tensor
    Q: torch.Tensor
    H: torch.Tensor
    R: torch.Tensor
    m0: torch.Tensor
    P0: torch.Tensor
    u: torch.Tensor | None = None
    d: torch.Tensor | None = None

    @classmethod
    def create(cls, F, Q, H, R, m0, P0, u=None, d=None, device="cuda") -> "Model":
        f32, f64 = torch.float32, torch.float64
        return cls(F=_dev(F, f32, device), Q=_dev(Q, f32, device), H=_dev(H, f32, device),
                   R=_dev(R, f32, device), m0=_dev(m0, f64, device), P0=_dev(P0, f64, device),
                   u=None if u is None else _dev(u, f32, device),
                   d=None if d is None else _dev(d, f32, device))

    @property
    def time_varying(self) -> bool:
        return self.F.dim() == 3

    @property
    def nx(self) -> int:
        return int(self.F.shape[-1])

    @property
    def ny(self) -> int:
        return int(self.H.shape[-2])

    def check_steps(self, T: int) -> None:
        """A time-varying model must carry (at least) T contiguous per-step
        entries of every parameter: the device reads entry k for step k."""
        if not self.time_varying:
            return
        nx, ny = self.nx, self.ny
        want = {"F": (nx, nx), "Q": (nx, nx), "H": (ny, nx), "R": (ny, ny), "u": (nx,), "d": (ny,)}
        for name, tail in want.items():
            t = getattr(self, name)
            if t is None:
                continue
            if t.dim() != len(tail) + 1 or tuple(t.shape[1:]) != tail or t.shape[0] < T or not t.is_contiguous():
                raise ValueError(f"time-varying {name} must be a contiguous [T >= {T}, {tail}] tensor, "
                                 f"got {tuple(t.shape)}")

    def struct(self) -> _KsModel:
        return _KsModel(self.nx, self.ny, int(self.time_varying), 0, self.F.data_ptr(),
                        0 if self.u is None else self.u.data_ptr(), self.Q.data_ptr(),
                        self.H.data_ptr(), 0 if self.d is None else self.d.data_ptr(),
                        self.R.data_ptr(), self.m0.data_ptr(), self.P0.data_ptr())


def supported(nx: int, ny: int) -> bool:
    return bool(lib().ks_supported(nx, ny))


def workspace_bytes(model: Model, T: int, purpose: int = KS_WS_SMOOTH) -> int:
    m = model.struct()
    n = lib().ks_workspace_bytes(ctypes.byref(m), T, purpose)
    if n == 0:
        raise KsError(KS_EUNSUPPORTED if not supported(model.nx, model.ny) else KS_EINVAL,
                      "ks_workspace_bytes")
    return int(n)


def alloc_workspace(model: Model, T: int, purpose: int = KS_WS_SMOOTH, stream=None) -> torch.Tensor:
    """A zero-initialised workspace tensor (uint8, on the model's device)."""
    nbytes = workspace_bytes(model, T, purpose)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=model.F.device)
    _check(lib().ks_workspace_init(_p(ws), nbytes, _stream(stream)), "ks_workspace_init")
    return ws


def _out(shape, like, out):
    if out is not None:
        return out
    return torch.empty(shape, dtype=torch.float32, device=like.device)


def smooth(model: Model, y: torch.Tensor, ws: torch.Tensor | None = None, *, fmean=None, fcov=None,
           smean=None, scov=None, keep_filtered: bool = True, filter_only: bool = False, stream=None,
           events=None):
    """End to end (``ks_smooth``): returns (fmean, fcov, smean, scov).

    With ``keep_filtered=False`` the filtered moments stay in the workspace
    (which must then be a KS_WS_ELEMENTS workspace) and None is returned for
    them.  With ``filter_only=True`` only the forward scan runs and None is
    returned for the smoothed moments.  ``events``: 4 recorded-or-fresh
    torch.cuda.Event objects to time the kernels (``ks_smooth_traced``).
    """
    T = int(y.shape[0])
    model.check_steps(T)
    if filter_only and not keep_filtered:
        raise ValueError("filter_only needs keep_filtered")
    purpose = KS_WS_SMOOTH if keep_filtered else KS_WS_ELEMENTS
    ws = alloc_workspace(model, T, purpose, stream) if ws is None else ws
    if keep_filtered:
        fmean = _out((T, model.nx), y, fmean)
        fcov = _out((T, model.nx, model.nx), y, fcov)
    else:
        fmean = fcov = None
    if filter_only:
        smean = scov = None
    else:
        smean = _out((T, model.nx), y, smean)
        scov = _out((T, model.nx, model.nx), y, scov)
    m = model.struct()
    args = (ctypes.byref(m), _p(y), T, _p(ws), ws.numel(), _p(fmean), _p(fcov), _p(smean), _p(scov),
            _stream(stream))
    if events is None:
        _check(lib().ks_smooth(*args), "ks_smooth")
    else:
        for e in events:
            if e is not None and not e.cuda_event:   # torch creates events lazily
                e.record(torch.cuda.current_stream() if stream is None else stream)
        handles = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) if e is not None else None
                                          for e in events])
        _check(lib().ks_smooth_traced(*args, handles), "ks_smooth_traced")
    return fmean, fcov, smean, scov


def loglik(model: Model, y: torch.Tensor, fmean: torch.Tensor | None, fcov: torch.Tensor | None, stream=None):
    """Marginal log-likelihood (``ks_loglik``) from the filtered moments:
    returns (per-step log p(y_k | y_1:k-1) [T] FP32, total FP64 [1], status
    word [1]), all on the device."""
    T = int(y.shape[0])
    ll = torch.empty(T, dtype=torch.float32, device=y.device)
    total = torch.empty(1, dtype=torch.float64, device=y.device)
    st = torch.empty(1, dtype=torch.int32, device=y.device)
    _check(lib().ks_loglik(ctypes.byref(model.struct()), _p(y), T, _p(fmean), _p(fcov), _p(ll), _p(total), _p(st),
                           _stream(stream)), "ks_loglik")
    return ll, total, st


def workspace_bytes_aggregate(model: Model, T: int) -> int:
    n = lib().ks_workspace_bytes_aggregate(ctypes.byref(model.struct()), T)
    if n == 0:
        raise KsError(KS_EUNSUPPORTED if not supported(model.nx, model.ny) else KS_EINVAL,
                      "ks_workspace_bytes_aggregate")
    return int(n)


def _agg_ws(model: Model, T: int, ws, stream):
    if ws is not None:
        return ws
    nbytes = workspace_bytes_aggregate(model, T)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=model.F.device)
    _check(lib().ks_workspace_init(_p(ws), nbytes, _stream(stream)), "ks_workspace_init")
    return ws


def filter_aggregate(model: Model, y: torch.Tensor, first: bool, ws=None, stream=None):
    """One shard's filtering aggregate (``ks_filter_aggregate``): the packed
    Lemma 4 fold of its Lemma 3 elements, [3nx^2 + 2nx]; returns (out, ws)."""
    T = int(y.shape[0])
    ws = _agg_ws(model, T, ws, stream)
    out = torch.empty(3 * model.nx * model.nx + 2 * model.nx, dtype=torch.float32, device=y.device)
    _check(lib().ks_filter_aggregate(ctypes.byref(model.struct()), _p(y), T, int(bool(first)), _p(ws), ws.numel(),
                                     _p(out), _stream(stream)), "ks_filter_aggregate")
    return out, ws


def smoother_aggregate(model: Model, fmean: torch.Tensor, fcov: torch.Tensor, last: bool, ws=None, stream=None):
    """One shard's smoothing aggregate (``ks_smoother_aggregate``): the packed
    Lemma 6 fold of its Lemma 5 elements, [2nx^2 + nx]; returns (out, ws)."""
    T = int(fmean.shape[0])
    ws = _agg_ws(model, T, ws, stream)
    out = torch.empty(2 * model.nx * model.nx + model.nx, dtype=torch.float32, device=fmean.device)
    _check(lib().ks_smoother_aggregate(ctypes.byref(model.struct()), T, _p(fmean), _p(fcov), int(bool(last)),
                                       _p(ws), ws.numel(), _p(out), _stream(stream)), "ks_smoother_aggregate")
    return out, ws


def build_elements(model: Model, y: torch.Tensor, ws: torch.Tensor, stream=None):
    """Lemma 3 elements into the workspace (``ks_build_elements``)."""
    m = model.struct()
    _check(lib().ks_build_elements(ctypes.byref(m), _p(y), int(y.shape[0]), _p(ws), ws.numel(),
                                   _stream(stream)), "ks_build_elements")


def elements(model: Model, T: int, ws: torch.Tensor) -> dict:
    """Views of the materialised elements: A, C, J [T,nx,nx]; b, eta [T,nx]."""
    m = model.struct()
    lay = _KsLayout()
    _check(lib().ks_elements_layout_get(ctypes.byref(m), T, ctypes.byref(lay)), "ks_elements_layout_get")
    n = model.nx
    f = ws.view(torch.float32) if ws.numel() % 4 == 0 else None

    def comp(off, k):
        return f[off // 4: off // 4 + k * lay.ld].view(k, lay.ld)[:, :T]

    return {"A": comp(lay.offset_A, n * n).T.reshape(T, n, n),
            "b": comp(lay.offset_b, n).T.reshape(T, n),
            "C": comp(lay.offset_C, n * n).T.reshape(T, n, n),
            "eta": comp(lay.offset_eta, n).T.reshape(T, n),
            "J": comp(lay.offset_J, n * n).T.reshape(T, n, n)}


def filter_scan(model: Model, T: int, ws: torch.Tensor, *, fmean=None, fcov=None, stream=None):
    """Forward scan over materialised elements (``ks_filter_scan``)."""
    fmean = _out((T, model.nx), ws, fmean)
    fcov = _out((T, model.nx, model.nx), ws, fcov)
    m = model.struct()
    _check(lib().ks_filter_scan(ctypes.byref(m), T, _p(ws), ws.numel(), _p(fmean), _p(fcov),
                                _stream(stream)), "ks_filter_scan")
    return fmean, fcov


def smooth_scan(model: Model, fmean: torch.Tensor, fcov: torch.Tensor, ws: torch.Tensor | None = None, *,
                smean=None, scov=None, stream=None):
    """Reverse scan from filtered moments (``ks_smooth_scan``)."""
    T = int(fmean.shape[0])
    ws = alloc_workspace(model, T, KS_WS_SMOOTH, stream) if ws is None else ws
    smean = _out((T, model.nx), fmean, smean)
    scov = _out((T, model.nx, model.nx), fmean, scov)
    m = model.struct()
    _check(lib().ks_smooth_scan(ctypes.byref(m), T, _p(fmean), _p(fcov), _p(ws), ws.numel(), _p(smean),
                                _p(scov), _stream(stream)), "ks_smooth_scan")
    return smean, scov


def status(ws: torch.Tensor, stream=None) -> int:
    """Synchronise, read and clear the device status word (``ks_status``)."""
    return int(lib().ks_status(_p(ws), _stream(stream)))


def set_waits(ws: torch.Tensor, wait_polls: int = 0, first_tile: int = 0, stream=None) -> None:
    """Testing aid (``ks_workspace_set_waits``): the look-back wait limit in
    polls (0: default) and the forward scan's first tile number (1 leaves
    tile 0 unpublished, so a wait must run out)."""
    _check(lib().ks_workspace_set_waits(_p(ws), ws.numel(), wait_polls, first_tile, _stream(stream)),
           "ks_workspace_set_waits")


def refinements(ws: torch.Tensor, stream=None) -> int:
    """Synchronise, read and clear the workspace's count of warps (or lane
    groups) that refined an ill-conditioned inverse (``ks_refinements``)."""
    n = ctypes.c_uint32(0)
    _check(lib().ks_refinements(_p(ws), _stream(stream), ctypes.byref(n)), "ks_refinements")
    return int(n.value)


def _combine(fn, name, nx, left, right, ws, stream):
    count = int(left.shape[0])
    out = torch.empty_like(left)
    if ws is None:
        ws = torch.zeros(256, dtype=torch.uint8, device=left.device)
    _check(fn(nx, count, _p(left), _p(right), _p(out), _p(ws), ws.numel(), _stream(stream)), name)
    return out, ws


def filter_combine_batch(nx: int, left: torch.Tensor, right: torch.Tensor, ws=None, stream=None):
    """Lemma 4 on packed element pairs [count, 3nx^2+2nx]; returns (out, ws)."""
    return _combine(lib().ks_filter_combine_batch, "ks_filter_combine_batch", nx, left, right, ws, stream)


def smoother_combine_batch(nx: int, left: torch.Tensor, right: torch.Tensor, ws=None, stream=None):
    """Lemma 6 on packed element pairs [count, 2nx^2+nx]; returns (out, ws)."""
    return _combine(lib().ks_smoother_combine_batch, "ks_smoother_combine_batch", nx, left, right, ws,
                    stream)


@dataclass
class ModelBatch:
    """B time-invariant models for sequences laid end to end (``ks_smooth_batch``).

    Per-sequence arrays stacked on a leading axis of length B (FP32; m0, P0
    FP64) and the int64 ``offsets`` [B+1] of each sequence's first step.
    """

    F: torch.Tensor
    Q: torch.Tensor
    H: torch.Tensor
    R: torch.Tensor
    m0: torch.Tensor
    P0: torch.Tensor
    offsets: torch.Tensor
    u: torch.Tensor | None = None
    d: torch.Tensor | None = None

    @classmethod
    def create(cls, models, lengths, device="cuda") -> "ModelBatch":
        """``models``: objects with F, Q, H, R, m0, P0 (and optionally u, d) of
        one common (nx, ny); ``lengths``: steps of each sequence (>= 1)."""
        import numpy as np
        f32, f64 = torch.float32, torch.float64

        def stack(name, dtype):
            return _dev(np.stack([np.asarray(getattr(m, name)) for m in models]), dtype, device)

        has_u = any(getattr(m, "u", None) is not None and np.any(np.asarray(m.u) != 0) for m in models)
        has_d = any(getattr(m, "d", None) is not None and np.any(np.asarray(m.d) != 0) for m in models)
        off = np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])
        return cls(F=stack("F", f32), Q=stack("Q", f32), H=stack("H", f32), R=stack("R", f32),
                   m0=stack("m0", f64), P0=stack("P0", f64),
                   offsets=torch.as_tensor(off, dtype=torch.int64, device=device),
                   u=stack("u", f32) if has_u else None, d=stack("d", f32) if has_d else None)

    @property
    def nx(self) -> int:
        return int(self.F.shape[1])

    @property
    def ny(self) -> int:
        return int(self.H.shape[1])

    @property
    def B(self) -> int:
        return int(self.F.shape[0])

    def struct(self) -> _KsModelBatch:
        return _KsModelBatch(self.nx, self.ny, self.B, 0, self.F.data_ptr(),
                             0 if self.u is None else self.u.data_ptr(), self.Q.data_ptr(),
                             self.H.data_ptr(), 0 if self.d is None else self.d.data_ptr(),
                             self.R.data_ptr(), self.m0.data_ptr(), self.P0.data_ptr(),
                             self.offsets.data_ptr())


def workspace_bytes_batch(nx: int, ny: int, B: int, total_T: int) -> int:
    n = lib().ks_workspace_bytes_batch(nx, ny, B, total_T)
    if n == 0:
        raise KsError(KS_EUNSUPPORTED if not supported(nx, ny) else KS_EINVAL, "ks_workspace_bytes_batch")
    return int(n)


def smooth_batch(batch: ModelBatch, y: torch.Tensor, ws: torch.Tensor | None = None, *, fmean=None,
                 fcov=None, smean=None, scov=None, stream=None):
    """Batched end to end (``ks_smooth_batch``) over ``y`` [total_T, ny]
    (sequences concatenated); returns concatenated (fmean, fcov, smean, scov)."""
    T = int(y.shape[0])
    n = batch.nx
    if ws is None:
        nbytes = workspace_bytes_batch(n, batch.ny, batch.B, T)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=y.device)
        _check(lib().ks_workspace_init(_p(ws), nbytes, _stream(stream)), "ks_workspace_init")
    fmean = _out((T, n), y, fmean)
    fcov = _out((T, n, n), y, fcov)
    smean = _out((T, n), y, smean)
    scov = _out((T, n, n), y, scov)
    mb = batch.struct()
    _check(lib().ks_smooth_batch(ctypes.byref(mb), _p(y), T, _p(ws), ws.numel(), _p(fmean), _p(fcov),
                                 _p(smean), _p(scov), _stream(stream)), "ks_smooth_batch")
    return fmean, fcov, smean, scov


def _groups_struct(groups):
    arr = (_KsBatchGroup * len(groups))()
    for i, (batch, y, outs) in enumerate(groups):
        arr[i].models = batch.struct()
        arr[i].total_T = int(y.shape[0])
        arr[i].y = y.data_ptr()
        arr[i].fmean, arr[i].fcov, arr[i].smean, arr[i].scov = (o.data_ptr() for o in outs)
    return arr


def workspace_bytes_batched(sizes) -> int:
    """Workspace of ``ks_smooth_batched`` for groups given as (nx, ny, B,
    total_T) tuples."""
    arr = (_KsBatchGroup * len(sizes))()
    for i, (nx, ny, B, T) in enumerate(sizes):
        arr[i].models.nx, arr[i].models.ny, arr[i].models.B = nx, ny, B
        arr[i].total_T = T
    n = lib().ks_workspace_bytes_batched(len(sizes), arr)
    if n == 0:
        raise KsError(KS_EINVAL, "ks_workspace_bytes_batched")
    return int(n)


def smooth_batched(groups, ws: torch.Tensor | None = None, *, outs=None, stream=None):
    """Mixed-size batch (``ks_smooth_batched``): ``groups`` is a list of
    (ModelBatch, y) pairs, one per state size (nx in {2, 4, 6}, distinct), each
    y [total_T_g, ny_g] the group's sequences concatenated.  One preparation,
    one forward and one reverse launch for all groups.  Returns, per group,
    (fmean, fcov, smean, scov); ``outs`` may give them preallocated."""
    if outs is None:
        outs = []
        for batch, y in groups:
            T, n = int(y.shape[0]), batch.nx
            outs.append((_out((T, n), y, None), _out((T, n, n), y, None), _out((T, n), y, None),
                         _out((T, n, n), y, None)))
    if ws is None:
        nbytes = workspace_bytes_batched([(b.nx, b.ny, b.B, int(y.shape[0])) for b, y in groups])
        ws = torch.empty(nbytes, dtype=torch.uint8, device=groups[0][1].device)
        _check(lib().ks_workspace_init(_p(ws), nbytes, _stream(stream)), "ks_workspace_init")
    arr = _groups_struct([(b, y, o) for (b, y), o in zip(groups, outs)])
    _check(lib().ks_smooth_batched(len(groups), arr, _p(ws), ws.numel(), _stream(stream)), "ks_smooth_batched")
    return outs


# ---------------------------------------------------------------- discrete-state models
@dataclass
class HmmModel:
    """Device-resident hidden Markov model (``ks_hmm``): prior pi [K] of x_0
    and row-stochastic transitions Pi [K, K], FP32."""

    pi: torch.Tensor
    Pi: torch.Tensor

    @classmethod
    def create(cls, pi, Pi, device="cuda") -> "HmmModel":
        return cls(pi=_dev(pi, torch.float32, device), Pi=_dev(Pi, torch.float32, device))

    @property
    def K(self) -> int:
        return int(self.pi.shape[0])

    def struct(self) -> _KsHmm:
        return _KsHmm(self.K, 0, self.pi.data_ptr(), self.Pi.data_ptr())


def hmm_supported(K: int) -> bool:
    return bool(lib().ks_hmm_supported(K))


def hmm_workspace_bytes(K: int, T: int) -> int:
    n = lib().ks_hmm_workspace_bytes(K, T)
    if n == 0:
        raise KsError(KS_EUNSUPPORTED if not hmm_supported(K) else KS_EINVAL, "ks_hmm_workspace_bytes")
    return int(n)


def hmm_smooth(model: HmmModel, lik: torch.Tensor, ws: torch.Tensor | None = None, *, filt=None, smooth=None,
               loglik=None, filter_only: bool = False, want_loglik: bool = True, stream=None, events=None):
    """Discrete-state filter and smoother (``ks_hmm_smooth``) over the
    likelihoods ``lik`` [T, K]: returns (filt [T, K], smooth [T, K] or None,
    loglik [T] or None)."""
    T, K = int(lik.shape[0]), int(lik.shape[1])
    if K != model.K or not lik.is_contiguous():
        raise ValueError("lik must be a contiguous [T, K] tensor with the model's K")
    if ws is None:
        nbytes = hmm_workspace_bytes(K, T)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=lik.device)
        _check(lib().ks_workspace_init(_p(ws), nbytes, _stream(stream)), "ks_workspace_init")
    filt = _out((T, K), lik, filt)
    smooth = None if filter_only else _out((T, K), lik, smooth)
    if want_loglik:
        loglik = _out((T,), lik, loglik)
    else:
        loglik = None
    h = model.struct()
    args = (ctypes.byref(h), _p(lik), T, _p(ws), ws.numel(), _p(filt), _p(smooth), _p(loglik), _stream(stream))
    if events is None:
        _check(lib().ks_hmm_smooth(*args), "ks_hmm_smooth")
    else:
        for e in events:
            if e is not None and not e.cuda_event:
                e.record(torch.cuda.current_stream() if stream is None else stream)
        handles = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) if e is not None else None
                                          for e in events])
        _check(lib().ks_hmm_smooth_traced(*args, handles), "ks_hmm_smooth_traced")
    return filt, smooth, loglik, ws
