"""Tuner of the fused scans' block length (Section III-C's block-level
elements: each thread folds l consecutive steps, a tile is 128 threads) and
of how a block is folded.

The nx <= 6 kernels are compiled for l in {4, 8, 16, 32}; short inputs need
short blocks to fill the 152 SMs, long inputs gain from long ones (less
per-block look-back and prefix work per step).  A full block of a
time-invariant model can be folded element by element or through
per-position coefficients built once per call (the linear block fold: fewer
operations per step, a longer preparation).  The library picks (l, fold) per
call from the call's total number of steps through a rule table per state
size (``ks_set_chunk_rules``).  This module

* measures, on the device it runs on, every (l, fold) variant at a grid of
  sizes for nx = 2, 4, 6 (one sequence through ``ks_smooth``) and for
  mixed-size batches (``ks_smooth_batched``, keyed by their total steps),
  timing each call with CUDA events after warm-up, L2 flushed between calls;
* turns the measurements into rules: the fastest variant at each measured
  size (keeping the smaller size's choice while it is within 2 % of the
  fastest), with the switch between two neighbouring sizes at their
  geometric mean;
* writes them to a versioned JSON cache, which the binding loads when the
  library is first used (``load_default``) if it was measured on the same
  device model and library version; otherwise the library's built-in table
  applies.

Run ``python -m paper_1905_13002_gb300.tune`` on the target GPU to refresh
``tuning/<device>.json``.
"""
from __future__ import annotations

import json
import math
import os
import time

CACHE_VERSION = 2
STEPS = (4, 8, 16, 32)
VARIANTS = tuple((s, f) for f in (0, 1) for s in STEPS)   # (steps per thread, block fold)
T_NEVER = 1 << 62                      # T_below of a last rule: "every larger size"
GRID = [1 << 10, 1 << 12, 1 << 14, 1 << 16, 98304, 1 << 17, 196608, 1 << 18, 1 << 19, 655360, 1 << 20,
        1 << 21, 1 << 22]
MIXED_B = [64, 256, 1024, 4096]        # sequences of the mixed batches (log-uniform lengths in [256, 16384])
SLOTS = (0, 2, 4, 6)                   # 0: mixed-size batches
HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")


# ---------------------------------------------------------------- selection logic
HYSTERESIS = 0.02   # keep the smaller size's choice while it is within 2 % of the fastest


def vkey(v) -> str:
    """Cache key of a variant: "32" (element by element) or "32f" (block fold)."""
    return f"{v[0]}{'f' if v[1] else ''}"


def vparse(k: str) -> tuple:
    return (int(k.rstrip("f")), 1 if k.endswith("f") else 0)


def rules_from(measured: dict) -> list:
    """measured: {size: {(steps, fold): ms}} -> [(T_below, steps, fold), ...]
    (sizes ascending).  The fastest variant at each size, except that the choice of the next
    smaller size is kept while it is within HYSTERESIS of the fastest (timing
    noise then does not flip the table back and forth); where neighbouring
    sizes disagree the switch sits at their geometric mean; equal neighbours
    merge."""
    sizes = sorted(measured)
    if not sizes:
        return []
    best = []
    for T in sizes:
        row = measured[T]
        fastest = min(row, key=lambda s: (row[s], s))
        if best and best[-1] in row and row[best[-1]] <= (1.0 + HYSTERESIS) * row[fastest]:
            fastest = best[-1]
        best.append(fastest)
    rules = []
    for i in range(len(sizes) - 1):
        if best[i] != best[i + 1]:
            rules.append((int(math.ceil(math.sqrt(sizes[i] * sizes[i + 1]))), int(best[i][0]), int(best[i][1])))
    rules.append((T_NEVER, int(best[-1][0]), int(best[-1][1])))
    return rules


def choose(rules: list, T: int) -> tuple:
    """The (steps, fold) the library uses for T steps under `rules` (the
    first rule whose T_below exceeds T, else the last one's)."""
    for tb, steps, fold in rules:
        if T < tb:
            return steps, fold
    return rules[-1][1], rules[-1][2]


def builtin(T: int, nx: int = 4) -> tuple:
    """The library's built-in (steps, fold) choice (nx = 0: mixed batches)."""
    steps = 4 if T < 96 * 1024 else 8 if T < 192 * 1024 else 16 if T < 640 * 1024 else 32
    return steps, int(nx != 0 and steps == 32)


def cache_path(device_name: str) -> str:
    slug = "".join(c.lower() if c.isalnum() else "_" for c in device_name).strip("_")
    return os.path.join(TUNING_DIR, f"{slug}.json")


def valid_cache(d: dict, device_name: str, lib_version: int) -> bool:
    return (d.get("version") == CACHE_VERSION and d.get("device") == device_name
            and d.get("library_version") == lib_version and isinstance(d.get("rules"), dict))


def apply(d: dict) -> None:
    from . import set_chunk_rules
    for key, rules in d["rules"].items():
        set_chunk_rules(int(key), [(int(tb), int(s), int(f)) for tb, s, f in rules])


def load_default() -> str | None:
    """Apply the cache of this device, if any (called when the library is
    first loaded).  KS_TUNING=off keeps the built-in table; KS_TUNING=<path>
    names another cache.  Returns the path applied, or None."""
    env = os.environ.get("KS_TUNING", "")
    if env.lower() in ("off", "0", "none"):
        return None
    try:
        import torch
        if not torch.cuda.is_available():
            return None
        name = torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return None
    path = env or cache_path(name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    from . import lib
    if not valid_cache(d, name, int(lib().ks_version())):
        return None
    apply(d)
    global APPLIED
    APPLIED = path
    return path


APPLIED = None


# ---------------------------------------------------------------- measurement
def _wiener(dim: int, dt: float = 0.1, q: float = 1.0, r: float = 1.0):
    """A d-axis Wiener-velocity model (positions observed) as numpy arrays:
    a representative time-invariant model for timing."""
    import numpy as np
    n = 2 * dim
    F = np.eye(n)
    F[:dim, dim:] = dt * np.eye(dim)
    Q = np.zeros((n, n))
    Q[:dim, :dim] = q * dt ** 3 / 3 * np.eye(dim)
    Q[:dim, dim:] = Q[dim:, :dim] = q * dt ** 2 / 2 * np.eye(dim)
    Q[dim:, dim:] = q * dt * np.eye(dim)
    H = np.zeros((dim, n))
    H[:, :dim] = np.eye(dim)
    return dict(F=F, Q=Q, H=H, R=r * np.eye(dim), m0=np.zeros(n), P0=np.eye(n))


def _measurements(T: int, dim: int, rng):
    """Positions of a slowly turning track with unit noise, FP32 [T, dim]."""
    import numpy as np
    t = np.arange(T, dtype=np.float64) * 0.1
    y = np.stack([np.cumsum(np.cos(1e-3 * t + a)) * 0.1 for a in range(dim)], 1)
    return (y + rng.standard_normal((T, dim))).astype(np.float32)


class _Timer:
    def __init__(self, torch, dev, reps: int, warmup: int):
        self.torch, self.reps, self.warmup = torch, reps, warmup
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def __call__(self, fn) -> float:
        torch = self.torch
        for _ in range(self.warmup):
            fn()
        ts = []
        for _ in range(self.reps):
            self.flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ts.sort()
        return ts[len(ts) // 2]


def measure_single(nx: int, sizes=GRID, reps: int = 7, warmup: int = 2, log=print) -> dict:
    import numpy as np
    import torch
    from . import KS_OK, Model, alloc_workspace, set_chunk_rules, smooth, status
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(1905130020 + nx)
    m = _wiener(nx // 2)
    model = Model.create(m["F"], m["Q"], m["H"], m["R"], m["m0"], m["P0"], device=dev)
    timer = _Timer(torch, dev, reps, warmup)
    out = {}
    for T in sizes:
        y = torch.as_tensor(_measurements(T, nx // 2, rng), device=dev)
        ws = alloc_workspace(model, T)
        outs = dict(fmean=torch.empty(T, nx, device=dev), fcov=torch.empty(T, nx, nx, device=dev),
                    smean=torch.empty(T, nx, device=dev), scov=torch.empty(T, nx, nx, device=dev))
        row = {}
        for v in VARIANTS:
            set_chunk_rules(nx, [(T_NEVER, v[0], v[1])])
            row[v] = timer(lambda: smooth(model, y, ws, **outs))
        if status(ws) != KS_OK:
            raise RuntimeError(f"device status not OK while tuning nx={nx} T={T}")
        out[T] = row
        log(f"nx={nx} T={T}: " + ", ".join(f"{vkey(v)}: {row[v]:.4f} ms" for v in VARIANTS))
        del ws, outs, y
    set_chunk_rules(nx, [])
    return out


def measure_mixed(batches=MIXED_B, reps: int = 5, warmup: int = 2, log=print) -> dict:
    import numpy as np
    import torch
    from . import KS_OK, ModelBatch, set_chunk_rules, smooth_batched, status, workspace_bytes_batched
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(1905130023)
    timer = _Timer(torch, dev, reps, warmup)

    class _M:   # attribute access for ModelBatch.create
        def __init__(self, d):
            self.__dict__.update(d)

    out = {}
    for B in batches:
        lengths = np.rint(np.exp(rng.uniform(math.log(256), math.log(16384), size=B))).astype(np.int64)
        nxs = rng.choice([2, 4, 6], size=B)
        groups = []
        for nx in (6, 4, 2):
            sel = [int(L) for L, n in zip(lengths, nxs) if n == nx]
            if not sel:
                continue
            batch = ModelBatch.create([_M(_wiener(nx // 2)) for _ in sel], sel, device=dev)
            y = torch.as_tensor(_measurements(int(sum(sel)), nx // 2, rng), device=dev)
            groups.append((batch, y))
        total = int(lengths.sum())
        ws = torch.zeros(workspace_bytes_batched([(b.nx, b.ny, b.B, int(y.shape[0])) for b, y in groups]),
                         dtype=torch.uint8, device=dev)
        outs = [(torch.empty(int(y.shape[0]), b.nx, device=dev), torch.empty(int(y.shape[0]), b.nx, b.nx, device=dev),
                 torch.empty(int(y.shape[0]), b.nx, device=dev), torch.empty(int(y.shape[0]), b.nx, b.nx, device=dev))
                for b, y in groups]
        row = {}
        for v in VARIANTS:
            set_chunk_rules(0, [(T_NEVER, v[0], v[1])])
            row[v] = timer(lambda: smooth_batched(groups, ws, outs=outs))
        if status(ws) != KS_OK:
            raise RuntimeError(f"device status not OK while tuning the mixed batch of {B} sequences")
        out[total] = row
        log(f"mixed B={B} total={total}: " + ", ".join(f"{vkey(v)}: {row[v]:.4f} ms" for v in VARIANTS))
        del ws, outs, groups
    set_chunk_rules(0, [])
    return out


def tune(quick: bool = False, log=print) -> dict:
    import torch
    from . import lib
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    sizes = GRID[::2] if quick else GRID
    meas = {}
    t0 = time.perf_counter()
    for nx in (2, 4, 6):
        meas[nx] = measure_single(nx, sizes, log=log)
    meas[0] = measure_mixed(MIXED_B[-2:] if quick else MIXED_B, log=log)
    rules = {str(k): rules_from(v) for k, v in meas.items()}
    return {"version": CACHE_VERSION, "library_version": int(lib().ks_version()), "device": name,
            "sm_count": torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count,
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "seconds": round(time.perf_counter() - t0, 1),
            "rules": rules,
            "measured_ms": {str(k): {str(T): {vkey(s): round(ms, 5) for s, ms in row.items()} for T, row in v.items()}
                            for k, v in meas.items()}}


def main(argv=None) -> int:
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=None, help="cache file (default: tuning/<device>.json in the package)")
    ap.add_argument("--quick", action="store_true", help="every other size, two mixed batches")
    args = ap.parse_args(argv)
    import torch
    os.environ["KS_TUNING"] = "off"       # measure against explicit rules only
    d = tune(quick=args.quick)
    path = args.out or cache_path(d["device"])
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    print(json.dumps({"cache": path, "rules": d["rules"], "seconds": d["seconds"]}))
    apply(d)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
