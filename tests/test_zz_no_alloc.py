"""ks_smooth_noalloc: the end-to-end call with its scratch in a static device
array, for callers that cannot allocate device memory.

Called through the C ABI and compared with ks_smooth (the workspace entry
point) on the same inputs, on two calls in a row with different sequences,
so the second call runs on whatever the first left in the shared array.
"""
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
    fn = ks.lib().ks_smooth_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.POINTER(ks._KsModel), vp, ctypes.c_int64, vp, vp, vp, vp, vp, vp]
    fn.restype = ctypes.c_int
    return ks


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_workspace_entry_point_on_two_calls(ks):
    fn = ks.lib().ks_smooth_noalloc
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (T, seed) in enumerate([(50001, 11), (1 << 20, 12)]):
        seq = workloads.tracking_sequence(T, seed=seed)
        m = seq.model
        model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, device="cuda")
        y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
        ref = ks.smooth(model, y)
        outs = [torch.full_like(r, float("nan")) for r in ref]
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        st = model.struct()
        rc = fn(ctypes.byref(st), _ptr(y), T, *(_ptr(o) for o in outs), _ptr(status), stream)
        assert rc == ks.KS_OK, f"call {call}: rc {rc}"
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"call {call}: device status {int(status.item())}"
        got = [o.cpu().numpy() for o in outs]
        want = [r.cpu().numpy().astype(np.float64) for r in ref]
        assert all(np.isfinite(g).all() for g in got), f"call {call}: unwritten outputs"
        parity.check_mean(got[0], want[0], want[1], parity.TOL)
        parity.check_cov(got[1], want[1], parity.TOL)
        parity.check_mean(got[2], want[2], want[3], parity.TOL)
        parity.check_cov(got[3], want[3], parity.TOL)
        # and, like every other entry point, against the FP64 oracle
        parity.check_all(got, oracle.kf_rts(m, seq.y))


def test_noalloc_filter_only(ks):
    """smean = scov = NULL runs the forward scan alone, as ks_smooth does."""
    fn = ks.lib().ks_smooth_noalloc
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    seq = workloads.tracking_sequence(9001, seed=13)
    m = seq.model
    model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, device="cuda")
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    fm = torch.full((seq.T, 4), float("nan"), device="cuda")
    fP = torch.full((seq.T, 4, 4), float("nan"), device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = model.struct()
    rc = fn(ctypes.byref(st), _ptr(y), seq.T, _ptr(fm), _ptr(fP), None, None, _ptr(status), stream)
    assert rc == ks.KS_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    rfm, rfP = oracle.kf(m, seq.y)
    parity.check_mean(fm.cpu().numpy(), rfm, rfP)
    parity.check_cov(fP.cpu().numpy(), rfP)


def test_noalloc_rejects_out_of_range_sizes(ks):
    fn = ks.lib().ks_smooth_noalloc
    seq = workloads.tracking_sequence(16, seed=3)
    m = seq.model
    model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, device="cuda")
    st = model.struct()
    dummy = ctypes.c_void_p(16)
    assert fn(ctypes.byref(st), dummy, (1 << 20) + 1, dummy, dummy, dummy, dummy, None, None) == ks.KS_EINVAL
    assert fn(ctypes.byref(st), dummy, 0, dummy, dummy, dummy, dummy, None, None) == ks.KS_EINVAL
    # one of the two smoothed outputs missing
    assert fn(ctypes.byref(st), dummy, 16, dummy, dummy, dummy, None, None, None) == ks.KS_EINVAL
    assert fn(ctypes.byref(st), dummy, 16, dummy, dummy, None, dummy, None, None) == ks.KS_EINVAL
    assert fn(ctypes.byref(st), dummy, 16, None, dummy, dummy, dummy, None, None) == ks.KS_EINVAL
    other = ks._KsModel(6, 3, 0, 0, 1, 0, 1, 1, 0, 1, 1, 1)
    assert fn(ctypes.byref(other), dummy, 16, dummy, dummy, dummy, dummy, None, None) == ks.KS_EUNSUPPORTED
