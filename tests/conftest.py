import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Worst parity measures per test (GPU runs): relative error, error in
    posterior sd, and the sd bound's use (<= 1 passes)."""
    try:
        import parity
    except Exception:  # pragma: no cover
        return
    if not parity.RECORD:
        return
    worst = {}
    for tid, e in parity.RECORD:
        w = worst.setdefault(tid, {"rel": 0.0, "sd": 0.0, "sdx": 0.0, "where": ""})
        w["rel"] = max(w["rel"], *(v for k, v in e.items() if k in ("fmean", "fcov", "smean", "scov", "mean")))
        w["sd"] = max(w["sd"], *(v for k, v in e.items() if k.endswith("_sd")))
        sdx = max(v for k, v in e.items() if k.endswith("_sdx"))
        if sdx >= w["sdx"]:
            w["sdx"], w["where"] = sdx, e.get("where", "")
    tr = terminalreporter
    tr.write_sep("-", "parity summary (max over steps and checks)")
    tr.write_line(f"{'rel':>9} {'sd':>9} {'sd-bound':>9}  test")
    for tid, w in sorted(worst.items(), key=lambda kv: -kv[1]["sdx"]):
        tr.write_line(f"{w['rel']:9.2e} {w['sd']:9.2e} {w['sdx']:9.3f}  {tid}")
        if w["sdx"] > 0.8 and w["where"]:
            tr.write_line(f"{'':30}{w['where']}")
