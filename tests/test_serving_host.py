"""Host logic of the serving loop (admission, grouping, stream slots, timing)
driven by a launcher that completes each launch after a simulated duration."""
import time

import pytest

torch = pytest.importorskip("torch")

from paper_1905_13002_gb300.serving import Request, Server, percentiles


class FakeLauncher:
    """Completes a launch after `per_step` seconds per step (no device)."""

    def __init__(self, per_step=2e-7, base=2e-4):
        self.per_step, self.base = per_step, base
        self.launches = []

    def start(self, t0):
        self.t0 = t0

    def launch(self, key, reqs, s):
        now = time.perf_counter() - self.t0
        h = {"done": now + self.base + self.per_step * sum(r.T for r in reqs), "key": key, "s": s,
             "rids": [r.rid for r in reqs], "t": now}
        self.launches.append(h)
        return h

    def poll(self, h):
        now = time.perf_counter() - self.t0
        return h["done"] if now >= h["done"] else None

    def finish(self, h, reqs, keep):
        if keep:
            for r in reqs:
                r.result = ("ok", r.rid)


def reqs(n, gap=1e-4, seed=0):
    import random
    rnd = random.Random(seed)
    out = []
    for i in range(n):
        nx = rnd.choice([4, 8])
        T = rnd.randint(64, 4000)
        out.append(Request(rid=i, nx=nx, ny=nx // 2, T=T, model=rnd.randrange(4), y=None, arrival=i * gap))
    return out


def nbytes(nx, ny, T):
    return 100 * T


def test_every_request_completes_in_order_of_its_stages():
    rs = reqs(200)
    srv = Server(FakeLauncher(), budget_bytes=10 ** 9, streams=2, bytes_fn=nbytes)
    done = srv.run(rs)
    assert sorted(r.rid for r in done) == list(range(200))
    for r in done:
        assert r.arrival <= r.admitted + 1e-9 <= r.launched + 2e-9 <= r.done + 3e-9
        assert r.latency >= 0


def test_budget_is_never_exceeded_and_admission_is_fifo():
    rs = reqs(150, gap=2e-5)
    budget = 100 * 12000                     # about three average requests
    srv = Server(FakeLauncher(per_step=1e-6), budget_bytes=budget, streams=2, bytes_fn=nbytes)
    done = srv.run(rs)
    assert len(done) == 150
    assert srv.stats.max_reserved <= budget
    by_rid = sorted(done, key=lambda r: r.rid)                   # arrival order
    assert all(a.admitted <= b.admitted for a, b in zip(by_rid, by_rid[1:]))


def test_launches_hold_one_state_size_and_respect_stream_slots():
    rs = reqs(300, gap=1e-5)
    la = FakeLauncher(per_step=5e-7)
    srv = Server(la, budget_bytes=10 ** 9, streams=3, bytes_fn=nbytes)
    done = srv.run(rs)
    by = {r.rid: r for r in done}
    for h in la.launches:
        assert len({(by[i].nx, by[i].ny) for i in h["rids"]}) == 1
        assert {(by[i].nx, by[i].ny) for i in h["rids"]} == {h["key"]}
    assert srv.stats.max_in_flight <= 3
    # a stream slot is reused only after its previous launch completed
    for s in range(3):
        hs = sorted((h for h in la.launches if h["s"] == s), key=lambda h: h["t"])
        for a, b in zip(hs, hs[1:]):
            assert b["t"] >= a["done"] - 1e-9


def test_requests_arriving_during_a_launch_join_a_later_one():
    # one long request, then short ones arriving while it runs
    rs = [Request(0, 4, 2, 200000, 0, None, 0.0)]
    rs += [Request(i, 4, 2, 100, 0, None, 0.002 + 1e-4 * i) for i in range(1, 20)]
    la = FakeLauncher(per_step=1e-7, base=1e-4)          # the long launch lasts ~20 ms
    srv = Server(la, budget_bytes=10 ** 9, streams=2, bytes_fn=nbytes)
    done = srv.run(rs)
    by = {r.rid: r for r in done}
    assert by[0].batch == 0
    late = [by[i] for i in range(1, 20)]
    # the short requests ran on the second stream while the long one was in flight
    assert any(r.done < by[0].done for r in late)
    assert max(r.batch for r in late) >= 1


def test_max_batch_steps_splits_groups():
    rs = [Request(i, 4, 2, 1000, 0, None, 0.0) for i in range(10)]
    la = FakeLauncher()
    srv = Server(la, budget_bytes=10 ** 9, streams=1, max_batch_steps=3000, bytes_fn=nbytes)
    srv.run(rs)
    assert all(len(h["rids"]) <= 3 for h in la.launches)
    assert sum(len(h["rids"]) for h in la.launches) == 10


def test_request_larger_than_budget_is_rejected():
    srv = Server(FakeLauncher(), budget_bytes=1000, bytes_fn=nbytes)
    with pytest.raises(ValueError):
        srv.run([Request(0, 4, 2, 100, 0, None, 0.0)])


def test_kept_results_that_fill_the_budget_raise_instead_of_spinning():
    rs = [Request(i, 4, 2, 100, 0, None, 0.0) for i in range(3)]
    srv = Server(FakeLauncher(), budget_bytes=25000, streams=1, bytes_fn=nbytes)
    with pytest.raises(RuntimeError):
        srv.run(rs, keep_results=True)


def test_percentiles_nearest_rank():
    v = list(range(1, 101))
    p = percentiles(v, (50, 99, 100))
    assert p[50] == 50 and p[99] == 99 and p[100] == 100
    assert percentiles([7.0])[99] == 7.0
