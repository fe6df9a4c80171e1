"""GPU parity of time-varying models: per-step (F_k, u_k, Q_k) and
(H_k, d_k, R_k) (Section II's model), through ks_smooth, against the FP64
oracle's sequential filter and smoother on the same per-step arrays."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import parity
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    return ks


def gpu_model(ks, m):
    return ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, u=m.u, d=m.d, device="cuda")


def run(ks, m, y, filter_only=False):
    model = gpu_model(ks, m)
    yt = torch.as_tensor(np.asarray(y), dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, yt.shape[0])
    out = ks.smooth(model, yt, ws, filter_only=filter_only)
    assert ks.status(ws) == ks.KS_OK
    return out


def check(ks, seq, tol=parity.TOL):
    got = run(ks, seq.model, seq.y)
    ref = oracle.kf_rts(seq.model, np.asarray(seq.y, dtype=np.float64))
    return parity.check_all(got, ref, tol)


# Irregularly sampled tracking (nx = 4): sizes span the ragged first tile,
# many tiles, and each of the four steps-per-thread choices (switching at
# 96 Ki, 192 Ki and 640 Ki steps).
@pytest.mark.parametrize("T", [1, 2, 3, 33, 511, 513, 4097, 20001, 98304, 200001, 700001])
def test_irregular_tracking_sizes(ks, T):
    check(ks, workloads.irregular_tracking(T, seed=7000 + T))


@pytest.mark.parametrize("dim,T", [(1, 1), (1, 3000), (1, 150001), (3, 2), (3, 2500), (3, 150001),
                                   (4, 2), (4, 63), (4, 64), (4, 65), (4, 5000), (4, 40001)])
def test_irregular_tracking_other_state_sizes(ks, dim, T):
    check(ks, workloads.irregular_tracking(T, seed=7100 + T + dim, dim=dim))


@pytest.mark.parametrize("nx,ny,T", [(2, 1, 700), (4, 2, 1), (4, 2, 900), (6, 3, 700), (8, 4, 1), (8, 4, 65),
                                     (8, 4, 700)])
def test_random_time_varying_dense(ks, nx, ny, T):
    """Dense per-step F_k, Q_k, H_k, R_k with non-zero u_k, d_k."""
    check(ks, workloads.random_time_varying(nx, ny, T, np.random.default_rng(7200 + T + nx)))


def test_constant_per_step_arrays_match_time_invariant_call(ks):
    """A time-varying model whose steps all repeat one model gives the
    time-invariant call's posteriors (the two paths differ only in how the
    Lemma 3 and 5 elements are formed)."""
    seq = workloads.tracking_sequence(5000, seed=7300)
    m = seq.model
    T = seq.T
    tv = workloads.Model(F=np.broadcast_to(m.F, (T,) + m.F.shape).copy(), u=np.broadcast_to(m.u, (T, m.nx)).copy(),
                         Q=np.broadcast_to(m.Q, (T,) + m.Q.shape).copy(), H=np.broadcast_to(m.H, (T,) + m.H.shape).copy(),
                         d=np.broadcast_to(m.d, (T, m.ny)).copy(), R=np.broadcast_to(m.R, (T,) + m.R.shape).copy(),
                         m0=m.m0, P0=m.P0)
    a = run(ks, m, seq.y)
    b = run(ks, tv, seq.y)
    ref = oracle.kf_rts(m, seq.y)
    for x, y, r, P in zip(a, b, ref, (ref[1], None, ref[3], None)):
        x = x.cpu().numpy()
        y = y.cpu().numpy()
        if P is not None:
            parity.check_mean(x, y, P, parity.TOL)
        else:
            parity.check_cov(x, y, parity.TOL)


def test_filter_only(ks):
    seq = workloads.irregular_tracking(30000, seed=7400)
    fm, fP, sm, sP = run(ks, seq.model, seq.y, filter_only=True)
    assert sm is None and sP is None
    rfm, rfP = oracle.kf(seq.model, seq.y)
    parity.check_mean(fm.cpu().numpy(), rfm, rfP, parity.TOL)
    parity.check_cov(fP.cpu().numpy(), rfP, parity.TOL)


def test_too_few_steps_rejected_before_launch(ks):
    seq = workloads.irregular_tracking(100, seed=7500)
    model = gpu_model(ks, seq.model)
    y = torch.zeros(101, 2, device="cuda")
    with pytest.raises(ValueError):
        ks.smooth(model, y)


def test_entry_points_without_time_varying_support(ks):
    """Entry points other than ks_smooth reject time-varying models, and so
    does the nx = 32 smoother; the workspace query returns 0 there."""
    seq = workloads.irregular_tracking(64, seed=7600)
    model = gpu_model(ks, seq.model)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, 64, ks.KS_WS_ELEMENTS)
    m = model.struct()
    L = ks.lib()
    st = ks._stream(None)
    assert L.ks_build_elements(ctypes.byref(m), ks._p(y), 64, ks._p(ws), ws.numel(), st) == ks.KS_EUNSUPPORTED
    fm = torch.empty(64, 4, device="cuda")
    fP = torch.empty(64, 4, 4, device="cuda")
    assert L.ks_smooth_scan(ctypes.byref(m), 64, ks._p(fm), ks._p(fP), ks._p(ws), ws.numel(), ks._p(fm),
                            ks._p(fP), st) == ks.KS_EUNSUPPORTED
    big = ks._KsModel(32, 8, 1, 0, m.F, 0, m.Q, m.H, 0, m.R, m.m0, m.P0)
    assert L.ks_workspace_bytes(ctypes.byref(big), 64, ks.KS_WS_SMOOTH) == 0
    assert L.ks_smooth(ctypes.byref(big), ks._p(y), 64, ks._p(ws), ws.numel(), None, None, ks._p(fm), ks._p(fP),
                       st) == ks.KS_EUNSUPPORTED
    torch.cuda.synchronize()


def test_bench_workload_full_size(ks):
    """The time-varying bench workload at its full size (T = 2^20, the launch
    configuration bench.py times), every step against the oracle."""
    import workloads as w
    e = check(ks, w.irregular_tracking(1 << 20, seed=w.SEED_BASE + 6))
    print("time-varying T=2^20 errors", e)
