"""The paper's only experiment (Section V, Figs. 3-5): span and work flops of
the sequential and parallel filter and smoother on the nx = 4, ny = 2 tracking
model, from a counted-flop model of the algorithms (oracle/flops.py).

Section V states: the parallel filter's span falls below the sequential
filter's flops from about T = 20 on; its work is about 8x the sequential
filter's; the parallel smoother matches the sequential smoother already below
T = 10; its work is about 4x; the span grows logarithmically, the sequential
flops linearly.  The paper does not give its counter's per-operation costs;
with the costs stated in oracle/flops.py the model gives 8.2x, 27, 3.25x and 7.
The bands below allow for the counter conventions, not for a wrong order of
magnitude or a wrong growth law."""
import math

from oracle import flops as F

N, M = 4, 2


def test_filter_work_ratio_is_about_eight():
    for T in (1 << 10, 1 << 16, 1 << 20):
        r = F.pkf(T, N, M)[1] / F.kf(T, N, M)
        assert 7.0 <= r <= 9.5, (T, r)


def test_smoother_work_ratio_is_about_four():
    for T in (1 << 10, 1 << 16, 1 << 20):
        r = F.prts(T, N)[1] / F.rts(T, N)
        assert 3.0 <= r <= 5.0, (T, r)


def test_filter_span_crossover_near_twenty():
    t = F.crossover(lambda T: F.pkf(T, N, M)[0], lambda T: F.kf(T, N, M))
    assert 12 <= t <= 40, t


def test_smoother_span_crossover_below_ten():
    t = F.crossover(lambda T: F.prts(T, N)[0], lambda T: F.rts(T, N))
    assert t < 10, t


def test_span_grows_logarithmically_and_work_linearly():
    for fn in (lambda T: F.pkf(T, N, M), lambda T: F.prts(T, N)):
        spans = [fn(1 << k)[0] for k in range(4, 16)]
        steps = {round(b - a, 6) for a, b in zip(spans, spans[1:])}
        assert len(steps) == 1                              # constant increment per doubling
        works = [fn(1 << k)[1] for k in (12, 13)]
        assert abs(works[1] / works[0] - 2.0) < 0.01


def test_scan_schedule_counts():
    # Fig. 1: n - 1 combines up, n - 1 down, n in the final pass; 2 log2 n + 1 levels
    assert F.scan_counts(8) == (2 * 7 + 8, 2 * 3 + 1)
    assert F.scan_counts(9) == (2 * 15 + 9, 2 * 4 + 1)
    assert F.scan_counts(1) == (0, 0)
    assert F.scan_counts(2) == (2 * 1 + 2, 2 * 1 + 1)


def test_operation_costs():
    c = F.Count()
    c.mul(2, 3, 4)
    assert c.f == 2 * 4 * 5
    c = F.Count()
    c.lu(3)
    assert math.isclose(c.f, 18.0)
