"""Pins of the discrete-state (HMM) oracle, oracle/hmm.py (no GPU).

The oracle's sequential filter/smoother and its Section III elements and
operators (counting measure) are checked against what the mathematics fixes:
exhaustive sums over all state paths on tiny problems, closed forms of two
degenerate chains, the associativity and identities of both operators, and
Theorems 1-2 (prefix / suffix sums equal the sequential posteriors).  The
last test plants mistakes in the oracle and checks that a pin catches each.
"""
import numpy as np
import pytest

from oracle import hmm


def rand_hmm(K, n, rng, lo=0.05, hi=3.0):
    pi = rng.dirichlet(np.ones(K))
    Pi = rng.dirichlet(np.ones(K), size=K)
    lik = rng.uniform(lo, hi, size=(n, K))
    return pi, Pi, lik


@pytest.mark.parametrize("K,n", [(2, 1), (2, 4), (3, 5), (4, 3)])
def test_forward_backward_equals_enumeration(K, n):
    pi, Pi, lik = rand_hmm(K, n, np.random.default_rng(10 * K + n))
    f, s, ll = hmm.forward_backward(pi, Pi, lik)
    bf, bs, bll = hmm.enumerate_posteriors(pi, Pi, lik)
    assert np.allclose(f, bf, atol=1e-13, rtol=0)
    assert np.allclose(s, bs, atol=1e-13, rtol=0)
    assert np.allclose(ll, bll, atol=1e-12, rtol=0)


def test_static_chain_closed_form():
    """Pi = I (the state never moves): p(x | y_1:k) is proportional to
    pi(x) prod_j lik_j(x), and every smoothed marginal is the last filtered one."""
    rng = np.random.default_rng(1)
    K, n = 5, 12
    pi, _, lik = rand_hmm(K, n, rng)
    f, s, ll = hmm.forward_backward(pi, np.eye(K), lik)
    w = pi[None, :] * np.cumprod(lik, axis=0)
    assert np.allclose(f, w / w.sum(1, keepdims=True), atol=1e-14)
    assert np.allclose(ll, np.log(w.sum(1)), atol=1e-12)
    assert np.allclose(s, np.tile(f[-1], (n, 1)), atol=1e-14)


def test_independent_states_closed_form():
    """Every row of Pi equal to r (states drawn independently each step):
    filtered and smoothed marginals are both proportional to r(x) lik_k(x)."""
    rng = np.random.default_rng(2)
    K, n = 4, 9
    pi, _, lik = rand_hmm(K, n, rng)
    r = rng.dirichlet(np.ones(K))
    f, s, ll = hmm.forward_backward(pi, np.tile(r, (K, 1)), lik)
    w = r[None, :] * lik
    assert np.allclose(f, w / w.sum(1, keepdims=True), atol=1e-14)
    assert np.allclose(s, f, atol=1e-14)
    assert np.allclose(ll, np.cumsum(np.log(w.sum(1))), atol=1e-12)


@pytest.mark.parametrize("K", [2, 4])
def test_parallel_formulation_equals_sequential(K):
    """Theorem 1 (prefix sums of the filtering elements give p(x_k | y_1:k) and
    p(y_1:k)) and Theorem 2 (suffix sums of the smoothing elements give
    p(x_k | y_1:n)), with Definitions 1-2 written with sums."""
    pi, Pi, lik = rand_hmm(K, 25, np.random.default_rng(3 + K))
    f, s, ll = hmm.forward_backward(pi, Pi, lik)
    pf, pll = hmm.parallel_filter(pi, Pi, lik)
    ps = hmm.parallel_smoother(Pi, f)
    assert np.allclose(pf, f, atol=1e-13)
    assert np.allclose(pll, ll, atol=1e-11)
    assert np.allclose(ps, s, atol=1e-13)


def rand_felem(K, rng):
    return hmm.HElem(rng.dirichlet(np.ones(K), size=K), rng.uniform(0.1, 2.0, size=K))


def test_operators_associative_and_identity():
    rng = np.random.default_rng(4)
    K = 4
    a, b, c = (rand_felem(K, rng) for _ in range(3))
    l = hmm.filter_combine(hmm.filter_combine(a, b), c)
    r = hmm.filter_combine(a, hmm.filter_combine(b, c))
    assert np.allclose(l.f, r.f, atol=1e-14) and np.allclose(l.g, r.g, atol=1e-14)
    e = hmm.filter_identity(K)
    for x in (hmm.filter_combine(a, e), hmm.filter_combine(e, a)):
        assert np.allclose(x.f, a.f, atol=1e-15) and np.allclose(x.g, a.g, atol=1e-15)
    A, B, C = (rng.dirichlet(np.ones(K), size=K) for _ in range(3))
    assert np.allclose(hmm.smoother_combine(hmm.smoother_combine(A, B), C),
                       hmm.smoother_combine(A, hmm.smoother_combine(B, C)), atol=1e-14)
    I = hmm.smoother_identity(K)
    assert np.allclose(hmm.smoother_combine(A, I), A) and np.allclose(hmm.smoother_combine(I, A), A)
    # both operators keep their elements in their sets (rows sum to one)
    assert np.allclose(hmm.filter_combine(a, b).f.sum(1), 1) and np.allclose(hmm.smoother_combine(A, B).sum(1), 1)


# ---------------------------------------------------------------- planted mistakes
def _fb_transposed(pi, Pi, lik):
    return _orig_fb(pi, np.asarray(Pi).T, lik)


def _fcomb_drop_gj(ai, aj):
    return _orig_fc(ai, hmm.HElem(aj.f, np.ones_like(aj.g)))


def _scomb_swapped(ai, aj):
    return _orig_sc(aj, ai)


def _selem_no_transpose(Pi, filt):
    return _orig_se(np.asarray(Pi).T, filt)


_orig_fb = hmm.forward_backward
_orig_fc = hmm.filter_combine
_orig_sc = hmm.smoother_combine
_orig_se = hmm.smoother_elements

CASES = {
    "forward_backward_transposed_Pi": ("forward_backward", _fb_transposed,
                                       [lambda: test_forward_backward_equals_enumeration(3, 5)]),
    "filter_combine_drops_g_j": ("filter_combine", _fcomb_drop_gj,
                                 [lambda: test_parallel_formulation_equals_sequential(4)]),
    "smoother_combine_swapped": ("smoother_combine", _scomb_swapped,
                                 [lambda: test_parallel_formulation_equals_sequential(4)]),
    "smoother_elements_untransposed": ("smoother_elements", _selem_no_transpose,
                                       [lambda: test_parallel_formulation_equals_sequential(4)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, mutant, checks = CASES[name]
    monkeypatch.setattr(hmm, attr, mutant)
    for check in checks:
        with pytest.raises(AssertionError):
            check()
