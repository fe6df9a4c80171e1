"""Discrete-state (hidden Markov model) instance of the general parallel
filter and smoother of Section III, in plain numpy FP64.

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke check
and the benchmark's CPU baseline use this module.

Section VI notes that the framework holds for discrete state spaces once the
integrals are taken against the counting measure.  Every integral of
Definitions 1 and 2 and Theorems 1 and 2 becomes a sum over the K states.

Model
-----
x_0 ~ pi (the prior before the first measurement, as N(m0, P0) in Section
IV), p(x_k = j | x_{k-1} = i) = Pi[i, j] for k = 1..n, and the measurement
enters only through its likelihoods lik[k-1, j] = p(y_k | x_k = j) >= 0
(so any emission model fits).  Arrays are indexed from 0: row k of `lik` is
step k + 1 of the paper.

Element representations
-----------------------
* filtering element (Definition 1): the pair (f, g) as a row-stochastic
  matrix f[z, x] = f(x | z) and a vector g[z] = g(z);
* smoothing element (Definition 2): a row-stochastic matrix a[z, x] = a(x | z).
"""
from __future__ import annotations

import itertools
from typing import NamedTuple

import numpy as np


class HElem(NamedTuple):
    f: np.ndarray    # [K, K], f[z, x] = f(x | z)
    g: np.ndarray    # [K],    g[z]


# ---------------------------------------------------------------- sequential
def forward_backward(pi, Pi, lik):
    """The sequential Bayesian filter and smoother (Section II-A's prediction,
    update and backward recursions with sums).

    Returns (filt [n, K] = p(x_k | y_1:k), smooth [n, K] = p(x_k | y_1:n),
    loglik [n] = log p(y_1:k)).
    """
    pi = np.asarray(pi, dtype=np.float64)
    Pi = np.asarray(Pi, dtype=np.float64)
    lik = np.asarray(lik, dtype=np.float64)
    n, K = lik.shape
    filt = np.empty((n, K))
    ll = np.empty(n)
    prev = pi
    total = 0.0
    for k in range(n):
        pred = prev @ Pi                       # p(x_k | y_1:k-1)
        w = pred * lik[k]                      # update
        c = w.sum()                            # p(y_k | y_1:k-1)
        filt[k] = w / c
        total += np.log(c)
        ll[k] = total
        prev = filt[k]
    smooth = np.empty((n, K))
    smooth[n - 1] = filt[n - 1]
    for k in range(n - 2, -1, -1):
        pred = filt[k] @ Pi                    # p(x_k+1 | y_1:k)
        smooth[k] = filt[k] * (Pi @ (smooth[k + 1] / pred))
    return filt, smooth, ll


# ---------------------------------------------------------------- Section III elements and operators
def filter_elements(pi, Pi, lik) -> list[HElem]:
    """Theorem 1's elements with sums: f_k(x | z) = p(x_k = x | y_k, x_k-1 = z)
    and g_k(z) = p(y_k | x_k-1 = z); for k = 1 both are conditioned on nothing
    (f_1(x | z) = p(x_1 = x | y_1) for every z, g_1 = p(y_1))."""
    pi = np.asarray(pi, dtype=np.float64)
    Pi = np.asarray(Pi, dtype=np.float64)
    lik = np.asarray(lik, dtype=np.float64)
    n, K = lik.shape
    out = []
    for k in range(n):
        if k == 0:
            joint = (pi @ Pi) * lik[0]             # p(x_1, y_1)
            py = joint.sum()
            f = np.tile(joint / py, (K, 1))
            g = np.full(K, py)
        else:
            joint = Pi * lik[k][None, :]           # joint[z, x] = p(x_k = x, y_k | x_k-1 = z)
            g = joint.sum(axis=1)
            f = joint / g[:, None]
        out.append(HElem(f, g))
    return out


def filter_combine(ai: HElem, aj: HElem) -> HElem:
    """Definition 1 with sums:
    f_ij(x | z) = sum_y g_j(y) f_j(x | y) f_i(y | z) / sum_y g_j(y) f_i(y | z),
    g_ij(z) = g_i(z) sum_y g_j(y) f_i(y | z)."""
    K = ai.g.shape[0]
    f = np.empty((K, K))
    g = np.empty(K)
    for z in range(K):
        den = sum(aj.g[y] * ai.f[z, y] for y in range(K))
        for x in range(K):
            f[z, x] = sum(aj.g[y] * aj.f[y, x] * ai.f[z, y] for y in range(K)) / den
        g[z] = ai.g[z] * den
    return HElem(f, g)


def filter_identity(K: int) -> HElem:
    """(f(x | z) = [x = z], g = 1): a two-sided identity of Definition 1."""
    return HElem(np.eye(K), np.ones(K))


def smoother_elements(Pi, filt) -> list[np.ndarray]:
    """Theorem 2's elements with sums: a_k(x | z) = p(x_k = x | y_1:k,
    x_k+1 = z) = filt_k(x) Pi[x, z] / sum_x' filt_k(x') Pi[x', z] for k < n,
    and a_n(x | z) = p(x_n = x | y_1:n)."""
    Pi = np.asarray(Pi, dtype=np.float64)
    filt = np.asarray(filt, dtype=np.float64)
    n, K = filt.shape
    out = []
    for k in range(n):
        if k == n - 1:
            out.append(np.tile(filt[k], (K, 1)))
        else:
            joint = filt[k][None, :] * Pi.T        # joint[z, x] = p(x_k = x, x_k+1 = z | y_1:k)
            out.append(joint / joint.sum(axis=1, keepdims=True))
    return out


def smoother_combine(ai: np.ndarray, aj: np.ndarray) -> np.ndarray:
    """Definition 2 with sums: a_ij(x | z) = sum_y a_i(x | y) a_j(y | z)."""
    K = ai.shape[0]
    out = np.empty((K, K))
    for z in range(K):
        for x in range(K):
            out[z, x] = sum(ai[y, x] * aj[z, y] for y in range(K))
    return out


def smoother_identity(K: int) -> np.ndarray:
    return np.eye(K)


def parallel_filter(pi, Pi, lik):
    """Theorem 1: the prefix a_1 (x) ... (x) a_k has f(. | z) = p(x_k | y_1:k)
    for every z and g = p(y_1:k).  Returns (filt [n, K], loglik [n])."""
    from .lemmas import all_prefix_sums
    pre = all_prefix_sums(filter_elements(pi, Pi, lik), filter_combine)
    return np.array([p.f[0] for p in pre]), np.array([np.log(p.g[0]) for p in pre])


def parallel_smoother(Pi, filt):
    """Theorem 2: the suffix a_k (x) ... (x) a_n has a(. | z) = p(x_k | y_1:n)
    for every z.  Returns smooth [n, K]."""
    from .lemmas import all_suffix_sums
    suf = all_suffix_sums(smoother_elements(Pi, filt), smoother_combine)
    return np.array([s[0] for s in suf])


# ---------------------------------------------------------------- brute force (pins)
def enumerate_posteriors(pi, Pi, lik):
    """Exact p(x_k | y_1:k), p(x_k | y_1:n) and log p(y_1:k) from the joint
    p(x_0:k, y_1:k) = pi(x_0) prod_j Pi[x_j-1, x_j] lik[j-1, x_j], summed
    over every state path (tiny n and K only)."""
    pi = np.asarray(pi, dtype=np.float64)
    Pi = np.asarray(Pi, dtype=np.float64)
    lik = np.asarray(lik, dtype=np.float64)
    n, K = lik.shape

    def joint(path):
        p = pi[path[0]]
        for j in range(1, len(path)):
            p *= Pi[path[j - 1], path[j]] * lik[j - 1, path[j]]
        return p

    filt = np.zeros((n, K))
    evid = np.zeros(n)
    for k in range(1, n + 1):                  # paths x_0..x_k
        for path in itertools.product(range(K), repeat=k + 1):
            p = joint(path)
            filt[k - 1, path[k]] += p
            evid[k - 1] += p
    smooth = np.zeros((n, K))
    for path in itertools.product(range(K), repeat=n + 1):
        p = joint(path)
        for k in range(1, n + 1):
            smooth[k - 1, path[k]] += p
    return filt / evid[:, None], smooth / smooth.sum(axis=1, keepdims=True), np.log(evid)
