"""Counted-flop model of the sequential and parallel filter and smoother
(Section V: span and work flops of KF vs PKF and RTS vs PRTS).

TEST INFRASTRUCTURE / ANALYSIS: it evaluates no posterior; it counts the
floating-point operations of each matrix operation of the algorithms, the
way Section V describes its counter (multiplication, summation and LU
factorisation costs, added after every operation).  Costs:
  product (n x m)(m x p): n p (2m - 1);  sum of n x m: n m;
  LU of n x n: (2/3) n^3;  solve with an LU factor, k right-hand sides: 2 n^2 k;
  vector ops as the corresponding products.
The parallel algorithms run the all-prefix-sums scan of Fig. 1 (Section
II-B): an up-sweep and a down-sweep over n' = 2^ceil(log2 n) elements and a
final pass a_i (x) b_i giving the inclusive sums.  Span counts one element
build and one combine per level (the operations of a level run in parallel);
work counts all of them.
"""
from __future__ import annotations

import math


class Count:
    def __init__(self):
        self.f = 0.0

    def mul(self, n, m, p):
        self.f += n * p * (2 * m - 1)

    def add(self, n, m=1):
        self.f += n * m

    def lu(self, n):
        self.f += 2.0 / 3.0 * n ** 3

    def solve(self, n, k):
        self.f += 2.0 * n * n * k


def kf_step(n: int, m: int) -> float:
    """One Kalman filter step (prediction and update)."""
    c = Count()
    c.mul(n, n, 1); c.add(n)                       # m- = F m + u
    c.mul(n, n, n); c.mul(n, n, n); c.add(n, n)    # P- = F P F^T + Q
    c.mul(m, n, n); c.mul(m, n, m); c.add(m, m)    # S = H P- H^T + R
    c.lu(m); c.mul(n, n, m); c.solve(m, n)         # K = P- H^T S^-1
    c.mul(m, n, 1); c.add(m); c.add(m)             # v = y - H m- - d
    c.mul(n, m, 1); c.add(n)                       # m = m- + K v
    c.mul(n, m, m); c.mul(n, m, n); c.add(n, n)    # P = P- - K S K^T
    return c.f


def rts_step(n: int) -> float:
    """One RTS smoother step, reusing the filter's predicted moments
    (m-, P-) of the next step, as the sequential smoother does."""
    c = Count()
    c.lu(n); c.mul(n, n, n); c.solve(n, n)         # G = P F^T (P-)^-1
    c.add(n); c.mul(n, n, 1); c.add(n)             # m_s = m + G (m_s' - m-)
    c.add(n, n); c.mul(n, n, n); c.mul(n, n, n); c.add(n, n)   # P_s = P + G (Ps' - P-) G^T
    return c.f


def lemma3(n: int, m: int) -> float:
    """One filtering element (Lemma 3, k > 1)."""
    c = Count()
    c.mul(m, n, n); c.mul(m, n, m); c.add(m, m)    # S = H Q H^T + R
    c.lu(m); c.mul(n, n, m); c.solve(m, n)         # K = Q H^T S^-1
    c.mul(m, n, n); c.mul(n, m, n); c.add(n, n); c.mul(n, n, n)   # A = (I - K H) F
    c.mul(m, n, 1); c.add(m); c.add(m); c.mul(n, m, 1); c.add(n)  # b = u + K (y - H u - d)
    c.mul(n, m, n); c.mul(n, n, n); c.add(n, n)    # C = (I - K H) Q
    c.mul(n, n, m); c.solve(m, 1); c.mul(n, m, 1)  # eta = F^T H^T S^-1 (y - H u - d)
    c.mul(n, m, m); c.solve(m, n); c.mul(n, m, n)  # J = F^T H^T S^-1 H F
    return c.f


def lemma4(n: int) -> float:
    """One application of the filtering operator (Lemma 4)."""
    c = Count()
    c.mul(n, n, n); c.add(n)                       # M = I + C_i J_j
    c.lu(n)
    c.mul(n, n, 1); c.add(n); c.solve(n, 1); c.mul(n, n, 1); c.add(n)   # b_ij
    c.solve(n, n); c.mul(n, n, n)                  # A_j M^-1 (one factorisation serves both)
    c.mul(n, n, n)                                 # A_ij = (A_j M^-1) A_i
    c.mul(n, n, n); c.mul(n, n, n); c.add(n, n)    # C_ij
    c.mul(n, n, 1); c.add(n); c.solve(n, 1); c.mul(n, n, 1); c.add(n)   # eta_ij
    c.solve(n, n); c.mul(n, n, n); c.mul(n, n, n); c.add(n, n)          # J_ij
    return c.f


def lemma5(n: int) -> float:
    """One smoothing element (Lemma 5, k < n)."""
    c = Count()
    c.mul(n, n, n); c.mul(n, n, n); c.add(n, n)    # P- = F P F^T + Q
    c.lu(n); c.mul(n, n, n); c.solve(n, n)         # E = P F^T (P-)^-1
    c.mul(n, n, 1); c.add(n); c.mul(n, n, 1); c.add(n)   # g = xbar - E (F xbar + u)
    c.mul(n, n, n); c.add(n, n)                    # L = P - E F P (with F P above)
    return c.f


def lemma6(n: int) -> float:
    """One application of the smoothing operator (Lemma 6)."""
    c = Count()
    c.mul(n, n, n)                                 # E_i E_j
    c.mul(n, n, 1); c.add(n)                       # E_i g_j + g_i
    c.mul(n, n, n); c.mul(n, n, n); c.add(n, n)    # E_i L_j E_i^T + L_i
    return c.f


def scan_counts(T: int) -> tuple[int, int]:
    """(work, span) in operator applications of the Fig. 1 scan plus its
    final pass, over T elements padded to a power of two."""
    if T <= 1:
        return 0, 0
    lev = math.ceil(math.log2(T))
    npad = 1 << lev
    return 2 * (npad - 1) + T, 2 * lev + 1


def kf(T: int, n: int, m: int) -> float:
    return T * kf_step(n, m)


def rts(T: int, n: int) -> float:
    return (T - 1) * rts_step(n)


def pkf(T: int, n: int, m: int) -> tuple[float, float]:
    """(span, work) flops of the parallel Kalman filter."""
    w, s = scan_counts(T)
    return lemma3(n, m) + s * lemma4(n), T * lemma3(n, m) + w * lemma4(n)


def prts(T: int, n: int) -> tuple[float, float]:
    """(span, work) flops of the parallel RTS smoother."""
    w, s = scan_counts(T)
    return lemma5(n) + s * lemma6(n), (T - 1) * lemma5(n) + w * lemma6(n)


def crossover(span_fn, seq_fn, Tmax: int = 4096) -> int:
    """Smallest T from which the parallel span stays below the sequential
    flops up to Tmax."""
    last = None
    for T in range(Tmax, 1, -1):
        if span_fn(T) >= seq_fn(T):
            return T + 1 if last is None else last
        last = T
    return 2
