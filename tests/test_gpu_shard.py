"""GPU: time sharding through libks (ks_filter_aggregate, ks_smoother_aggregate,
the filter-only ks_smooth and the operator batches).  Ranks are emulated in
one process, phase by phase (every rank's aggregate, then the exchange); the
concatenated shards must match the FP64 oracle on the whole sequence."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads
from shard_ops import NumpyOps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    return ks


def gpu_model(ks, m):
    return ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, u=m.u, d=m.d, device="cuda")


def data(dim, T, seed):
    rng = np.random.default_rng(seed)
    m = workloads.wiener_velocity(dim, dt=0.1, q=float(rng.uniform(0.5, 2)), r=float(rng.uniform(0.1, 1)))
    _, y = workloads.simulate(m, T, rng)
    return m, y


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("first", [True, False])
@pytest.mark.parametrize("T", [1, 37, 5000, 9000])
def test_filter_aggregate_equals_lemma_fold(ks, first, T):
    m, y = data(2, T, 40 + T)
    got = ks.filter_aggregate(gpu_model(ks, m), torch.as_tensor(y, dtype=torch.float32, device="cuda"), first)[0]
    ref = NumpyOps().filter_aggregate(m, y, first).numpy()
    n = 4
    g = got.cpu().numpy()
    # b and C carry the shard's posterior information; A, eta, J as well
    for lo, hi in [(0, n * n), (n * n, n * n + n), (n * n + n, 2 * n * n + n), (2 * n * n + n, 2 * n * n + 2 * n),
                   (2 * n * n + 2 * n, 3 * n * n + 2 * n)]:
        assert rel(g[lo:hi], ref[lo:hi]) < 2e-4, (lo, hi, rel(g[lo:hi], ref[lo:hi]))


@pytest.mark.parametrize("last", [True, False])
@pytest.mark.parametrize("T", [1, 37, 5000])
def test_smoother_aggregate_equals_lemma_fold(ks, last, T):
    m, y = data(2, T, 60 + T)
    fm, fc = oracle.kf(m, y)
    got = ks.smoother_aggregate(gpu_model(ks, m), torch.as_tensor(fm, dtype=torch.float32, device="cuda"),
                                torch.as_tensor(fc, dtype=torch.float32, device="cuda"), last)[0].cpu().numpy()
    ref = NumpyOps().smoother_aggregate(m, torch.from_numpy(fm.astype(np.float32).astype(np.float64)),
                                        torch.from_numpy(fc.astype(np.float32).astype(np.float64)), last).numpy()
    n = 4
    for lo, hi in [(0, n * n), (n * n, n * n + n), (n * n + n, 2 * n * n + n)]:
        assert rel(got[lo:hi], ref[lo:hi]) < 2e-4, (lo, hi, rel(got[lo:hi], ref[lo:hi]))


def test_filter_only_smooth_equals_full(ks):
    m, y = data(2, 20000, 81)
    model = gpu_model(ks, m)
    yt = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    fm1, fc1, sm, sc = ks.smooth(model, yt, filter_only=True)
    assert sm is None and sc is None
    fm2, fc2, _, _ = ks.smooth(model, yt)
    assert torch.equal(fm1, fm2) and torch.equal(fc1, fc2)


@pytest.mark.parametrize("dim,T,world", [(2, 20001, 2), (2, 20001, 3), (2, 50000, 5), (1, 9000, 4), (3, 12345, 3)])
def test_emulated_ranks_equal_the_oracle(ks, dim, T, world):
    from paper_1905_13002_gb300 import shard
    m, y = data(dim, T, 90 + dim + world)
    model = gpu_model(ks, m)
    yt = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    n = 2 * dim
    parts = [shard.ShardSmoother(shard.DeviceOps(), model, yt[s:e].contiguous(), r, world, n)
             for r, (s, e) in enumerate(shard.shard_bounds(T, world))]
    aggs = [p.filter_aggregate() for p in parts]
    for p in parts:
        p.forward(aggs)
    saggs = [p.smoother_aggregate() for p in parts]
    outs = [p.reverse(saggs) for p in parts]
    got = [torch.cat([o[i] for o in outs]).cpu().numpy() for i in range(4)]
    e = parity.check_all(got, oracle.kf_rts(m, y))
    print(f"nx={n} T={T} world={world} errors", e)
