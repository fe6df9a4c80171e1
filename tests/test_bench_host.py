"""Host-side pieces of bench.py that shape its JSON line: the work models
behind the roofline fields and the gating of the recorded ncu traffic."""
import json

import bench


def test_flop_model_nx4():
    """Per-step flops of the fused nx = 4, ny = 2 scans (the roofline's
    algorithmic work): forward 1402 with the linear block fold (innovation and
    two 4 x 2 products, advance, measurement element, Lemma 5 element, fused
    Lemma 6 fold), 2230 when each step is folded by the rank-2 combine instead
    (time-varying models); reverse 744."""
    f = bench.flops_per_step(4, 2)
    assert f == {"filter": 1402, "smoother": 744}
    assert bench.flops_per_step(4, 2, block_fold=False) == {"filter": 2230, "smoother": 744}
    # without the fused smoothing fold the reverse scan builds its elements twice
    g = bench.flops_per_step(4, 2, fused_smoothing=False)
    assert g["filter"] < f["filter"] and g["smoother"] > f["smoother"]


def test_time_varying_bytes_nx4():
    """Algorithmic bytes per step of the time-varying path at nx = 4, ny = 2
    (u = d = 0): element kernel 344, forward scan 368, reverse scan 288."""
    assert bench.tv_bytes_per_step(4, 2) == {"elements": 344, "filter": 368, "smoother": 288}


def test_recorded_traffic_only_for_its_length_and_sources(tmp_path, monkeypatch):
    """The ncu traffic goes into the bench line only for the sequence length it
    was captured at and while the kernel's sources hash as recorded."""
    key = "filter_scan_kernel"
    rec = {key: {"source_hash": bench.source_hash(key), "T": 1 << 20, "dram_bytes_per_launch_full": 123.0}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda k: rec[key]["source_hash"] if k == key else "x")
    assert bench.recorded_traffic(key, 1 << 20) == 123.0
    assert bench.recorded_traffic(key, 1024) is None
    assert bench.recorded_traffic("smoother_scan_kernel", 1 << 20) is None
    monkeypatch.setattr(bench, "source_hash", lambda k: "changed")
    assert bench.recorded_traffic(key, 1 << 20) is None


def test_launch_counts():
    """Kernels per ks_smooth call in the bench's gpu_launches: 4 for the fused
    nx <= 6 path (preparation, forward, refinement retry, reverse); at nx = 32
    the preparation and per scan a reduce, the spine levels over tiles of 216
    steps and an apply (T = 65536: 304 tiles, 9 levels)."""
    assert bench.launches_per_call(4, 1 << 20) == 4
    assert bench.launches_per_call(32, 65536) == 1 + 2 * (2 + 9)
    assert bench.launches_per_call(32, 216) == 1 + 2 * 2


def test_output_errors_measure_the_means_in_posterior_sd():
    """The bench line's max_err: FP32 rounding of the oracle's own outputs
    stays far inside the sd bound; a mean moved by one posterior sd along the
    least certain direction reads as 1 sd."""
    import numpy as np
    import oracle
    import workloads
    seq = workloads.tracking_sequence(2000, seed=9)
    ref = oracle.kf_rts(seq.model, seq.y)
    got = [np.asarray(x, dtype=np.float32) for x in ref]
    e = bench.output_errors(got, ref)
    assert e["fmean"]["rel"] < 1e-6 and e["scov"]["rel"] < 1e-6
    assert e["fmean"]["sd_bound_use"] < 0.2 and e["smean"]["sd_bound_use"] < 0.2
    k = 1234
    w, V = np.linalg.eigh(ref[1][k])
    moved = got[0].astype(np.float64)
    moved[k] += np.sqrt(w[0]) * V[:, 0]
    e = bench.output_errors([moved, got[1], got[2], got[3]], ref)
    assert abs(e["fmean"]["sd"] - 1.0) < 1e-3
    assert e["fmean"]["sd_bound_use"] > 1.0
