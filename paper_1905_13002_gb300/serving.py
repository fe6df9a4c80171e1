"""Continuous batching of smoothing requests (the serving workload).

A request is one sequence: a time-invariant model of state size nx and its
measurements y [T, ny] in (pinned) host memory.  The loop

- admits a request once the device memory it needs (its measurements, the
  filtered and smoothed moments, its share of the scan workspace) fits in the
  budget that the requests already admitted leave free, in arrival order;
- groups admitted requests of one (nx, ny) into a single segmented launch
  (``ks_smooth_batch``: the sequences end to end, one forward and one reverse
  scan over all of them, no combine crossing a sequence start), so a long
  request is scanned in parallel with the short ones beside it instead of
  holding them up;
- keeps up to ``streams`` launches in flight on separate CUDA streams: a
  request that arrives while launches run joins the next launch on the first
  stream that frees up, and its work overlaps theirs on the device;
- takes a request's completion time from the CUDA event recorded after its
  launch (the results are then on the device) and releases its memory.

The scheduling (admission, grouping, stream slots, timing) is independent of
the device: ``Server`` drives a launcher object, ``GpuLauncher`` for the
CUDA path.  Latency is measured from a request's scheduled arrival time
(open loop), so a slow loop cannot hide queueing delay.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import torch

from . import KS_OK, ModelBatch, lib, smooth_batch, workspace_bytes_batch, _check, _p, _stream


@dataclass
class Request:
    rid: int
    nx: int
    ny: int
    T: int
    model: int                 # index into the launcher's model set for (nx, ny)
    y: torch.Tensor            # [T, ny] FP32 host (pinned) or device tensor
    arrival: float             # scheduled arrival (s, on the server's clock)
    admitted: float = -1.0
    launched: float = -1.0
    done: float = -1.0
    batch: int = -1
    result: tuple | None = None   # (smean, scov) device views when results are kept

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def request_bytes(nx: int, ny: int, T: int) -> int:
    """Device bytes a request holds while admitted: measurements, filtered and
    smoothed moments (FP32), its share of the segmented workspace, and its
    model in the launch's gathered batch (F, Q, H, R in FP32, m0 and P0 in
    FP64, one int64 offset and one int64 index).

    The budget this counts against is logical: torch's caching allocator may
    keep freed blocks reserved beyond it, and a launch's handful of small
    tensors are rounded up to the allocator's block size."""
    model = 4 * (2 * nx * nx + nx * ny + ny * ny) + 8 * (nx + nx * nx) + 16
    return 4 * T * ny + 2 * 4 * T * (nx + nx * nx) + workspace_bytes_batch(nx, ny, 1, T) + model


@dataclass
class _Launch:
    key: tuple
    reqs: list
    stream: int
    handle: object
    launched: float


@dataclass
class ServerStats:
    requests: int = 0
    steps: int = 0
    launches: int = 0
    max_reserved: int = 0
    max_in_flight: int = 0
    batch_sizes: list = field(default_factory=list)


class Server:
    """Open-loop request loop over a launcher.

    ``launcher`` provides ``launch(key, reqs, stream) -> handle``,
    ``poll(handle) -> completion time or None`` (non-blocking) and
    ``finish(handle, reqs, keep)`` (status check, results).  Times are in
    seconds on ``clock`` relative to the start of ``run``.
    """

    def __init__(self, launcher, budget_bytes: int, streams: int = 3, max_batch_steps: int = 1 << 24,
                 max_batch_requests: int = 1024, bytes_fn=request_bytes, clock=time.perf_counter):
        if streams < 1:
            raise ValueError("streams must be >= 1")
        self.launcher = launcher
        self.budget = int(budget_bytes)
        self.streams = streams
        self.max_batch_steps = max_batch_steps
        self.max_batch_requests = max_batch_requests
        self.bytes_fn = bytes_fn
        self.clock = clock
        self.stats = ServerStats()

    def run(self, requests: list, keep_results: bool = False, idle_sleep: float = 20e-6) -> list:
        """Serve ``requests`` (any order; ``arrival`` = scheduled time) to
        completion; returns them with admitted/launched/done times set."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting = collections.deque()                 # arrived, not admitted (FIFO)
        admitted = collections.OrderedDict()          # key -> deque of admitted, not launched
        need = {}
        reserved = 0
        free_streams = list(range(self.streams))
        in_flight: list[_Launch] = []
        done = []
        st = self.stats
        t0 = self.clock()
        self.launcher.start(t0)
        while pending or waiting or any(admitted.values()) or in_flight:
            now = self.clock() - t0
            progressed = False
            while pending and pending[0].arrival <= now:          # arrivals
                waiting.append(pending.popleft())
            while waiting:                                        # admission, in arrival order
                r = waiting[0]
                if r.rid not in need:
                    need[r.rid] = int(self.bytes_fn(r.nx, r.ny, r.T))
                b = need[r.rid]
                if b > self.budget:
                    raise ValueError(f"request {r.rid} needs {b} bytes, more than the whole budget")
                if reserved + b > self.budget:
                    break
                waiting.popleft()
                reserved += b
                st.max_reserved = max(st.max_reserved, reserved)
                r.admitted = now
                admitted.setdefault((r.nx, r.ny), collections.deque()).append(r)
                progressed = True
            for L in list(in_flight):                             # completions
                t_done = self.launcher.poll(L.handle)
                if t_done is None:
                    continue
                self.launcher.finish(L.handle, L.reqs, keep_results)
                in_flight.remove(L)
                free_streams.append(L.stream)
                for r in L.reqs:
                    r.done = t_done
                    if not keep_results:
                        reserved -= need.pop(r.rid)
                    done.append(r)
                progressed = True
            while free_streams:                                   # launches
                key = self._oldest_group(admitted)
                if key is None:
                    break
                q = admitted[key]
                batch, steps = [], 0
                while q and len(batch) < self.max_batch_requests and (
                        not batch or steps + q[0].T <= self.max_batch_steps):
                    r = q.popleft()
                    batch.append(r)
                    steps += r.T
                s = free_streams.pop(0)
                now = self.clock() - t0
                for r in batch:
                    r.launched = now
                    r.batch = st.launches
                handle = self.launcher.launch(key, batch, s)
                in_flight.append(_Launch(key, batch, s, handle, now))
                st.launches += 1
                st.batch_sizes.append(len(batch))
                st.max_in_flight = max(st.max_in_flight, len(in_flight))
                progressed = True
            if not progressed and waiting and not in_flight and not any(admitted.values()):
                raise RuntimeError("the budget is held by kept results: request "
                                   f"{waiting[0].rid} can never be admitted")
            if not progressed:
                nxt = pending[0].arrival - (self.clock() - t0) if pending else idle_sleep
                if not in_flight and nxt > 0:
                    time.sleep(min(nxt, 1e-3))
                elif idle_sleep > 0:
                    time.sleep(idle_sleep)
        st.requests += len(done)
        st.steps += sum(r.T for r in done)
        return done

    @staticmethod
    def _oldest_group(admitted):
        best, bt = None, None
        for key, q in admitted.items():
            if q and (bt is None or (q[0].arrival, q[0].rid) < bt):
                best, bt = key, (q[0].arrival, q[0].rid)
        return best


class ModelSet:
    """Device copies of the models of one (nx, ny) a server can be asked for;
    a launch gathers its requests' models by index (no host transfer)."""

    def __init__(self, models, device="cuda"):
        import numpy as np
        f32, f64 = torch.float32, torch.float64

        def stack(name, dtype):
            return torch.as_tensor(np.stack([np.asarray(getattr(m, name)) for m in models]), dtype=dtype,
                                   device=device).contiguous()

        self.F, self.Q, self.H, self.R = (stack(n, f32) for n in ("F", "Q", "H", "R"))
        self.u = stack("u", f32) if all(getattr(m, "u", None) is not None for m in models) else None
        self.d = stack("d", f32) if all(getattr(m, "d", None) is not None for m in models) else None
        self.m0, self.P0 = stack("m0", f64), stack("P0", f64)
        self.nx, self.ny = int(self.F.shape[1]), int(self.H.shape[1])

    def batch(self, idx: torch.Tensor, lengths: list) -> ModelBatch:
        off = torch.zeros(len(lengths) + 1, dtype=torch.int64)
        off[1:] = torch.cumsum(torch.as_tensor(lengths, dtype=torch.int64), 0)

        def g(t):
            return None if t is None else t.index_select(0, idx).contiguous()

        return ModelBatch(F=g(self.F), Q=g(self.Q), H=g(self.H), R=g(self.R), m0=g(self.m0), P0=g(self.P0),
                          offsets=off.to(self.F.device, non_blocking=True), u=g(self.u), d=g(self.d))


class GpuLauncher:
    """Launches request groups as ``ks_smooth_batch`` calls on its streams.

    Per launch: the requests' measurements are gathered into a pinned staging
    buffer of the stream (host copy) and moved with one host-to-device copy;
    the models are gathered on the device; the workspace and outputs come from
    torch's caching allocator on that stream; an event recorded after the
    call marks completion.  A stream's staging buffer is reused only after
    its previous launch completed.
    """

    def __init__(self, model_sets: dict, streams: int = 3, device="cuda"):
        self.sets = model_sets
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.staging = [None] * streams
        self.ref = None
        self.log = []              # per launch: (nx, requests, steps, host s, device ms)

    def start(self, t0_host: float):
        """Pin the event clock to the host clock at the start of a run."""
        torch.cuda.synchronize(self.device)
        self.ref = torch.cuda.Event(enable_timing=True)
        self.ref.record(torch.cuda.current_stream(self.device))
        self.ref.synchronize()
        self.ref_host = time.perf_counter() - t0_host

    def _stage(self, s: int, n: int, ny: int, ys: list) -> torch.Tensor:
        buf = self.staging[s]
        if buf is None or buf.numel() < n * ny:
            buf = torch.empty(max(n * ny, 1 << 20), dtype=torch.float32, pin_memory=True)
            self.staging[s] = buf
        view = buf[:n * ny].view(n, ny)
        torch.cat(ys, dim=0, out=view)
        return view

    def launch(self, key, reqs, s: int):
        h0 = time.perf_counter()
        nx, ny = key
        ms = self.sets[key]
        lengths = [r.T for r in reqs]
        total = sum(lengths)
        stream = self.streams[s]
        host_y = [r.y for r in reqs]
        with torch.cuda.stream(stream):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            if all(y.is_cuda for y in host_y):
                y = torch.cat(host_y, dim=0)
            elif all(y.is_pinned() for y in host_y):          # one DMA copy per request
                y = torch.empty((total, ny), dtype=torch.float32, device=self.device)
                o = 0
                for t in host_y:
                    y[o:o + t.shape[0]].copy_(t, non_blocking=True)
                    o += t.shape[0]
            else:                                            # pageable: gather into pinned staging
                y = torch.empty((total, ny), dtype=torch.float32, device=self.device)
                y.copy_(self._stage(s, total, ny, [t.cpu() if t.is_cuda else t for t in host_y]),
                        non_blocking=True)
            idx = torch.as_tensor([r.model for r in reqs], dtype=torch.int64).to(self.device, non_blocking=True)
            mb = ms.batch(idx, lengths)
            nbytes = workspace_bytes_batch(nx, ny, len(reqs), total)
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            _check(lib().ks_workspace_init(_p(ws), nbytes, _stream(stream)), "ks_workspace_init")
            out = smooth_batch(mb, y, ws, stream=stream)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        return {"ev": ev, "ev0": ev0, "ws": ws, "out": out, "y": y, "mb": mb, "stream": stream,
                "lengths": lengths, "nx": nx, "host_s": time.perf_counter() - h0}

    def poll(self, h):
        if not h["ev"].query():
            return None
        return self.ref_host + self.ref.elapsed_time(h["ev"]) / 1e3

    def finish(self, h, reqs, keep: bool):
        st = int(lib().ks_status(_p(h["ws"]), _stream(h["stream"])))
        if st != KS_OK:
            raise RuntimeError(f"batched launch reported status {st}")
        self.log.append((h["nx"], len(reqs), sum(h["lengths"]), h["host_s"], h["ev0"].elapsed_time(h["ev"])))
        if keep:
            _, _, sm, sc = h["out"]
            o = 0
            for r, T in zip(reqs, h["lengths"]):
                r.result = (sm[o:o + T], sc[o:o + T])
                o += T
        h.clear()


def percentiles(values, ps=(50, 99)) -> dict:
    """Nearest-rank percentiles of a list of numbers."""
    v = sorted(values)
    out = {}
    for p in ps:
        if not v:
            out[p] = float("nan")
            continue
        k = max(0, min(len(v) - 1, int(-(-p * len(v) // 100)) - 1))
        out[p] = v[k]
    return out
