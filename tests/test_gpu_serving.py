"""GPU: the serving loop (continuous batching over ks_smooth_batch on two
streams).  Each request's result in the mix equals its result alone (plain
ks_smooth on its own) and the FP64 oracle, within the parity tolerance."""
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


@pytest.fixture(scope="module")
def setup(ks):
    from paper_1905_13002_gb300 import serving
    models = workloads.serving_models(n_per_size=4, seed=workloads.SEED_BASE + 5)
    ys = workloads.serving_measurements(models, 6000, seed=workloads.SEED_BASE + 5)
    sets = {(nx, nx // 2): serving.ModelSet(ms) for nx, ms in models.items()}
    return serving, models, ys, sets


def make_requests(serving, models, ys, n, seed, lo=64, hi=6000, spread=0.02):
    arr = workloads.serving_arrivals(rate=n / spread, n=n, seed=seed, lo=lo, hi=hi, n_models=4)
    out = []
    for i, a in enumerate(arr):
        y = torch.from_numpy(ys[a.nx][a.model][:a.T]).pin_memory()
        out.append(serving.Request(rid=i, nx=a.nx, ny=a.nx // 2, T=a.T, model=a.model, y=y, arrival=a.t))
    return out


def alone(ks, models, r):
    m = models[r.nx][r.model]
    model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, u=m.u, d=m.d, device="cuda")
    ws = ks.alloc_workspace(model, r.T)
    out = ks.smooth(model, r.y.cuda(), ws)
    assert ks.status(ws) == ks.KS_OK
    return out[2].cpu().numpy(), out[3].cpu().numpy()


def test_mix_equals_alone_and_oracle(ks, setup):
    serving, models, ys, sets = setup
    reqs = make_requests(serving, models, ys, 40, seed=901)
    srv = serving.Server(serving.GpuLauncher(sets, streams=2), budget_bytes=8 << 30, streams=2)
    done = srv.run(reqs, keep_results=True)
    assert len(done) == 40
    assert srv.stats.launches >= 2                       # requests arrived while launches ran
    worst_alone = worst_oracle = 0.0
    for r in done:
        sm, sc = (t.cpu().numpy() for t in r.result)
        am, ac = alone(ks, models, r)
        m = models[r.nx][r.model]
        _, _, rsm, rsc = oracle.kf_rts(m, ys[r.nx][r.model][:r.T].astype(np.float64))
        worst_alone = max(worst_alone, parity.mean_err(sm, am, rsc), parity.cov_err(sc, ac))
        worst_oracle = max(worst_oracle, parity.mean_err(sm, rsm, rsc), parity.cov_err(sc, rsc))
        parity.check_mean(sm, rsm, rsc)
        assert parity.sd_excess(sm, am, rsc) <= 1.0
    print("mix vs alone", worst_alone, "mix vs oracle", worst_oracle)
    assert worst_alone < parity.TOL
    assert worst_oracle < parity.TOL


def test_tight_budget_queues_but_serves_everything(ks, setup):
    serving, models, ys, sets = setup
    reqs = make_requests(serving, models, ys, 30, seed=902, spread=0.005)
    need = sorted(serving.request_bytes(r.nx, r.ny, r.T) for r in reqs)
    budget = need[-1] + need[-2]                           # room for about two requests at a time
    srv = serving.Server(serving.GpuLauncher(sets, streams=2), budget_bytes=budget, streams=2)
    done = srv.run(reqs)
    assert len(done) == 30
    assert srv.stats.max_reserved <= budget
    assert srv.stats.launches >= 10
    assert all(r.done >= r.launched >= r.admitted >= r.arrival for r in done)


def test_long_nx8_request_in_the_mix(ks, setup):
    """A served nx = 8 request of 150,000 steps (the serving workload draws T
    up to 2^18) among short requests of both sizes: each result equals its
    result alone and the FP64 oracle."""
    serving, models, ys, sets = setup
    long_T = 150000
    m8 = models[8][1]
    rng = np.random.default_rng(905)
    _, ylong = workloads.simulate(m8, long_T, rng)
    reqs = make_requests(serving, models, ys, 12, seed=906)
    reqs.append(serving.Request(rid=len(reqs), nx=8, ny=4, T=long_T, model=1,
                                y=torch.from_numpy(np.ascontiguousarray(ylong, dtype=np.float32)).pin_memory(),
                                arrival=0.0))
    srv = serving.Server(serving.GpuLauncher(sets, streams=2), budget_bytes=8 << 30, streams=2)
    done = srv.run(reqs, keep_results=True)
    assert len(done) == len(reqs)
    for r in done:
        sm, sc = (t.cpu().numpy() for t in r.result)
        m = models[r.nx][r.model]
        y = ylong if r.T == long_T and r.nx == 8 else ys[r.nx][r.model][:r.T]
        am, ac = alone(ks, models, r)
        _, _, rsm, rsc = oracle.kf_rts(m, np.asarray(y, dtype=np.float64))
        parity.check_mean(sm, rsm, rsc)
        parity.check_cov(sc, rsc)
        assert parity.sd_excess(sm, am, rsc) <= 1.0
