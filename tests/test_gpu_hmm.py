"""GPU parity of the discrete-state (HMM) filter and smoother (Section III
with the counting measure) through the C ABI, against the FP64 oracle's
sequential forward filter / backward smoother (oracle/hmm.py)."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from oracle import hmm as ohmm

pytestmark = pytest.mark.gpu

# Probabilities in [0, 1]: absolute error per entry.  The log-likelihood
# log p(y_1:k) grows like k: error relative to max(1, |ll_k|).
TOL_P = 1e-4
TOL_LL = 1e-4


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    return ks


def run(ks, seq, **kw):
    model = ks.HmmModel.create(seq.pi, seq.Pi)
    lik = torch.as_tensor(seq.lik, dtype=torch.float32, device="cuda")
    filt, smooth, ll, ws = ks.hmm_smooth(model, lik, **kw)
    return filt, smooth, ll, ks.status(ws)


def check(ks, seq):
    filt, smooth, ll, st = run(ks, seq)
    assert st == ks.KS_OK
    rf, rs, rll = ohmm.forward_backward(seq.pi, seq.Pi, seq.lik)
    ef = np.abs(filt.cpu().numpy() - rf).max()
    es = np.abs(smooth.cpu().numpy() - rs).max()
    el = (np.abs(ll.cpu().numpy() - rll) / np.maximum(1.0, np.abs(rll))).max()
    assert ef < TOL_P and es < TOL_P and el < TOL_LL, (ef, es, el)
    return ef, es, el


# K = 8: sizes span one thread's steps (4, 16 or 32), a 512-, 2048- or
# 4096-step tile, many tiles with ragged tails, and all three steps-per-thread
# choices (switching at 256 Ki and 768 Ki steps).
@pytest.mark.parametrize("T", [1, 2, 3, 33, 511, 512, 513, 2049, 65537, 262143, 262144, 300001, 786431,
                               786432, 800001])
def test_regime_switching_k8(ks, T):
    check(ks, workloads.hmm_sequence(8, T, seed=8000 + T))


@pytest.mark.parametrize("K,T", [(2, 1), (2, 5000), (2, 300001), (2, 800001), (4, 7), (4, 40000), (4, 270001),
                                 (4, 790001)])
def test_other_state_counts(ks, K, T):
    check(ks, workloads.hmm_sequence(K, T, seed=8100 + T + K))


# K = 16 and 32 run one K-lane group per chain of 64 steps (8 or 4 chains
# per tile) with reduce / spine / apply launches: sizes span one chain, one
# tile (512 or 256 steps), ragged tails and many spine levels.
@pytest.mark.parametrize("T", [1, 2, 63, 64, 65, 255, 256, 257, 5000, 70001])
def test_k32(ks, T):
    check(ks, workloads.hmm_sequence(32, T, seed=8500 + T))


@pytest.mark.parametrize("T", [1, 2, 64, 65, 511, 512, 513, 5000, 70001])
def test_k16(ks, T):
    check(ks, workloads.hmm_sequence(16, T, seed=8700 + T))


def test_k32_filter_only(ks):
    seq = workloads.hmm_sequence(32, 9000, seed=8600)
    filt, smooth, ll, st = run(ks, seq, filter_only=True)
    assert st == ks.KS_OK and smooth is None
    rf, _, rll = ohmm.forward_backward(seq.pi, seq.Pi, seq.lik)
    assert np.abs(filt.cpu().numpy() - rf).max() < TOL_P
    assert (np.abs(ll.cpu().numpy() - rll) / np.maximum(1.0, np.abs(rll))).max() < TOL_LL


@pytest.mark.parametrize("stay", [0.999, 0.9999])
def test_nearly_static_chain(ks, stay):
    """Long runs in one state with weak evidence per step (sigma = 1.5).  A
    smoothed marginal then pools about tau = 1 / (1 - stay) steps whose
    transition matrices are close to the identity, so FP32 rounding adds up
    over tau steps without being damped: the bound is ~2 tau eps32 (1.2e-4
    and 1.2e-3 here), so the tolerance is the larger of that and 1e-4."""
    tol = max(TOL_P, 2.0 / (1.0 - stay) * np.finfo(np.float32).eps)
    seq = workloads.hmm_sequence(4, 50000, seed=8200, stay=stay, sigma=1.5)
    filt, smooth, ll, st = run(ks, seq)
    assert st == ks.KS_OK
    rf, rs, rll = ohmm.forward_backward(seq.pi, seq.Pi, seq.lik)
    ef = np.abs(filt.cpu().numpy() - rf).max()
    es = np.abs(smooth.cpu().numpy() - rs).max()
    el = (np.abs(ll.cpu().numpy() - rll) / np.maximum(1.0, np.abs(rll))).max()
    assert ef < TOL_P and es < tol and el < TOL_LL, (ef, es, el, tol)


def test_filter_only_and_no_loglik(ks):
    seq = workloads.hmm_sequence(8, 30000, seed=8300)
    filt, smooth, ll, st = run(ks, seq, filter_only=True, want_loglik=False)
    assert st == ks.KS_OK and smooth is None and ll is None
    rf, _, _ = ohmm.forward_backward(seq.pi, seq.Pi, seq.lik)
    assert np.abs(filt.cpu().numpy() - rf).max() < TOL_P


def test_impossible_observation_is_reported(ks):
    """A likelihood row with no positive entry has no posterior: the device
    status reports it (no fault, no hang)."""
    seq = workloads.hmm_sequence(4, 3000, seed=8400)
    seq.lik[1234] = 0.0
    _, _, _, st = run(ks, seq)
    assert st == ks.KS_ENUMERIC


def test_unsupported_state_count(ks):
    pi = torch.full((3,), 1 / 3, device="cuda")
    Pi = torch.full((3, 3), 1 / 3, device="cuda")
    h = ks._KsHmm(3, 0, pi.data_ptr(), Pi.data_ptr())
    lik = torch.ones(10, 3, device="cuda")
    out = torch.empty(10, 3, device="cuda")
    assert not ks.hmm_supported(3) and ks.hmm_supported(16) and ks.hmm_supported(32)
    assert ks.lib().ks_hmm_workspace_bytes(3, 10) == 0
    assert ks.lib().ks_hmm_smooth(ctypes.byref(h), ks._p(lik), 10, None, 0, ks._p(out), None, None,
                                  ks._stream(None)) == ks.KS_EUNSUPPORTED


def test_bench_workload_full_size(ks):
    """The discrete-state bench workload at its full size (K = 8, T = 2^20),
    every step against the oracle."""
    e = check(ks, workloads.hmm_sequence(8, 1 << 20, seed=workloads.SEED_BASE + 7))
    print("HMM K=8 T=2^20 errors (filt, smooth, loglik)", e)
