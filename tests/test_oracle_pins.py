"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check reaches its expected value by a route that shares no formula with
the oracle: dense joint-Gaussian algebra over the whole trajectory, numerical
integration of the paper's general operators (Definitions 1 and 2), closed
forms of special models, and the paper's own worked prefix-sum example.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import lemmas as L
import pins
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------ golden
def _read_golden_prefix():
    rows = []
    with open(os.path.join(GOLDEN, "prefix_sums_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split("|")
            op, *a = lhs.split()
            rows.append((op, [float(v) for v in a], [float(v) for v in rhs.split()]))
    return rows


def test_prefix_sums_worked_example():
    """Section II-B example: a_i = i, n = 4 -> (1,3,6,10) for +, (1,-1,-4,-8) for -."""
    ops = {"add": lambda x, y: x + y, "sub": lambda x, y: x - y}
    rows = _read_golden_prefix()
    assert len(rows) == 2
    for op, a, expect in rows:
        assert L.all_prefix_sums(a, ops[op]) == expect


def test_suffix_sums_keep_left_operand_earlier():
    """Theorem 2's suffix sums a_k ⊗ ... ⊗ a_n on a non-commutative operator
    (string concatenation): the earlier element must stay on the left."""
    got = L.all_suffix_sums(list("abcd"), lambda x, y: x + y)
    assert got == ["abcd", "bcd", "cd", "d"]
    assert L.all_prefix_sums(list("abcd"), lambda x, y: x + y) == ["a", "ab", "abc", "abcd"]


def _read_golden_model():
    out = {}
    with open(os.path.join(GOLDEN, "tracking_model.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split("=")
            out[k.strip()] = np.array([[float(t) for t in r.split()] for r in v.split(";")])
    return out


def test_tracking_model_matches_section_v():
    g = _read_golden_model()
    m = workloads.wiener_velocity(2, dt=0.1, q=1.0, r=0.25, m0=np.array([0, 0, 1.0, -1.0]))
    for k in ("F", "Q", "H", "R", "P0"):
        np.testing.assert_allclose(getattr(m, k), g[k], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(m.m0, g["m0"].reshape(-1))


# ------------------------------------------------------------------ dense posterior
@pytest.mark.parametrize("n,m,T,tv", [(1, 1, 6, False), (2, 1, 5, False), (3, 2, 6, False),
                                      (4, 2, 8, False), (3, 2, 5, True), (4, 3, 4, True)])
def test_kf_rts_equals_dense_posterior(n, m, T, tv):
    """Filtered and smoothed marginals of the sequential oracle equal the
    marginals of the dense joint posterior of the whole trajectory."""
    rng = np.random.default_rng(100 + 10 * n + T + tv)
    model = pins.rand_model(n, m, rng, T if tv else None)
    y = rng.standard_normal((T, m))
    fm, fP, sm, sP = oracle.kf_rts(model, y)
    dfm, dfP, dsm, dsP = pins.dense_filter_smoother(model, y)
    assert relerr(fm, dfm) < 1e-10
    assert relerr(fP, dfP) < 1e-10
    assert relerr(sm, dsm) < 1e-10
    assert relerr(sP, dsP) < 1e-10


def test_tracking_model_equals_dense_posterior():
    seq = workloads.tracking_sequence(8, seed=7)
    fm, fP, sm, sP = oracle.kf_rts(seq.model, seq.y)
    dfm, dfP, dsm, dsP = pins.dense_filter_smoother(seq.model, seq.y)
    for a, b in ((fm, dfm), (fP, dfP), (sm, dsm), (sP, dsP)):
        assert relerr(a, b) < 1e-9


@pytest.mark.parametrize("tv", [False, True])
def test_loglik_equals_dense_marginal(tv):
    """Σ_k log p(y_k | y_{1:k-1}) (Section III-C) = log of the stacked
    Gaussian marginal p(y_{1:T})."""
    rng = np.random.default_rng(5 + tv)
    T = 7
    model = pins.rand_model(3, 2, rng, T if tv else None)
    y = rng.standard_normal((T, 2))
    _, _, ll = oracle.kf(model, y, loglik=True)
    assert abs(ll.sum() - pins.dense_loglik(model, y)) < 1e-9 * max(1.0, abs(ll.sum()))


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("q,r", [(1.0, 1.0), (0.1, 2.0), (3.0, 0.2)])
def test_scalar_random_walk_riccati(q, r):
    """F = H = 1: the filter covariance converges to P = P- r/(P- + r) with
    P- = (q + sqrt(q^2 + 4qr))/2, and the smoothed covariance in the middle of
    a long sequence to P/(1 + G) with G = P/P-."""
    T = 4000
    model = pins.TinyModel(np.eye(1), np.zeros(1), q * np.eye(1), np.eye(1), np.zeros(1),
                           r * np.eye(1), np.zeros(1), np.eye(1))
    y = np.random.default_rng(3).standard_normal((T, 1))
    fm, fP, sm, sP = oracle.kf_rts(model, y)
    Pm = (q + np.sqrt(q * q + 4 * q * r)) / 2
    Pf = Pm * r / (Pm + r)
    G = Pf / Pm
    Ps = Pf / (1 + G)
    assert abs(fP[-1, 0, 0] - Pf) < 1e-12 * Pf
    assert abs(sP[T // 2, 0, 0] - Ps) < 1e-12 * Ps
    assert abs(sP[-1, 0, 0] - Pf) < 1e-12 * Pf


def test_no_measurement_information():
    """H = 0: nothing is learned, so filtered = smoothed = the prior marginal
    m_k = F^k m0 + Σ F^j u, P_k = F^k P0 F^kT + Σ_{j<k} F^j Q F^jT."""
    rng = np.random.default_rng(11)
    n, m, T = 3, 2, 12
    F = rng.standard_normal((n, n)) * 0.5
    u = rng.standard_normal(n)
    Q = pins.rand_spd(n, rng)
    model = pins.TinyModel(F, u, Q, np.zeros((m, n)), np.zeros(m), np.eye(m),
                           rng.standard_normal(n), pins.rand_spd(n, rng))
    y = rng.standard_normal((T, m))
    fm, fP, sm, sP = oracle.kf_rts(model, y)
    Fk = np.eye(n)
    for k in range(1, T + 1):
        Fk = F @ Fk
        mk = Fk @ model.m0 + sum(np.linalg.matrix_power(F, j) @ u for j in range(k))
        Pk = Fk @ model.P0 @ Fk.T + sum(np.linalg.matrix_power(F, j) @ Q @ np.linalg.matrix_power(F, j).T
                                        for j in range(k))
        assert relerr(fm[k - 1], mk) < 1e-11
        assert relerr(fP[k - 1], Pk) < 1e-11
    assert relerr(sm, fm) < 1e-11
    assert relerr(sP, fP) < 1e-11


def test_static_parameter_is_bayesian_regression():
    """F = I, Q = 0 with time-varying H_k: the filter is Bayesian linear
    regression, P_k^{-1} = P0^{-1} + Σ_{j<=k} H_j^T R^{-1} H_j and
    m_k = P_k (P0^{-1} m0 + Σ H_j^T R^{-1} (y_j - d)); every smoothed
    marginal equals the final filtered one."""
    rng = np.random.default_rng(13)
    n, m, T = 3, 1, 20
    Hs = rng.standard_normal((T, m, n))
    R = np.array([[0.3]])
    model = pins.TinyModel(np.eye(n), np.zeros(n), np.zeros((n, n)), Hs, np.zeros(m), R,
                           rng.standard_normal(n), pins.rand_spd(n, rng))
    y = rng.standard_normal((T, m))
    fm, fP, sm, sP = oracle.kf_rts(model, y)
    info = np.linalg.inv(model.P0)
    vec = info @ model.m0
    for k in range(T):
        info = info + Hs[k].T @ np.linalg.inv(R) @ Hs[k]
        vec = vec + Hs[k].T @ np.linalg.inv(R) @ y[k]
        Pk = np.linalg.inv(info)
        assert relerr(fP[k], Pk) < 1e-10
        assert relerr(fm[k], Pk @ vec) < 1e-10
    for k in range(T):
        assert relerr(sm[k], fm[-1]) < 1e-9
        assert relerr(sP[k], fP[-1]) < 1e-9


def test_invariants_on_tracking_workload():
    """Symmetry, positive definiteness, Ps_k <= P_k (Loewner) and Ps_T = P_T."""
    seq = workloads.config_single(T=512)
    fm, fP, sm, sP = oracle.kf_rts(seq.model, seq.y)
    for P in (fP, sP):
        assert np.max(np.abs(P - P.transpose(0, 2, 1))) < 1e-12 * np.max(np.abs(P))
        assert np.min(np.linalg.eigvalsh(0.5 * (P + P.transpose(0, 2, 1)))) > 0
    D = fP - sP
    assert np.min(np.linalg.eigvalsh(0.5 * (D + D.transpose(0, 2, 1)))) > -1e-12
    assert np.array_equal(sP[-1], fP[-1]) and np.array_equal(sm[-1], fm[-1])


# ------------------------------------------------------------------ lemmas
def rand_felem(n, rng, first=False):
    A = np.zeros((n, n)) if first else rng.standard_normal((n, n)) / np.sqrt(n)
    return L.FElem(A, rng.standard_normal(n), pins.rand_spd(n, rng, 0.5),
                   rng.standard_normal(n), pins.rand_psd(n, rng, scale=0.7))


def rand_selem(n, rng):
    return L.SElem(rng.standard_normal((n, n)) / np.sqrt(n), rng.standard_normal(n),
                   pins.rand_spd(n, rng, 0.5))


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lemma3_equals_joint_conditioning(n):
    """Lemma 3's (A, b, C) is p(x_k | y_k, x_{k-1}) and (eta, J) the quadratic
    of log p(y_k | x_{k-1}), both obtained here by textbook conditioning."""
    rng = np.random.default_rng(20 + n)
    m = max(1, n // 2)
    mod = pins.rand_model(n, m, rng)
    y = rng.standard_normal(m)
    got = L.filter_element(mod.F, mod.u, mod.Q, mod.H, mod.d, mod.R, y)
    A, b, C, eta, J = pins.filter_element_by_joint(mod.F, mod.u, mod.Q, mod.H, mod.d, mod.R, y)
    for x, ref in zip(got, (A, b, C, eta, J)):
        assert relerr(x, ref) < 1e-7


def test_lemma3_first_element_is_one_kalman_step():
    """k = 1: (A_1, b_1, C_1) = (0, m_1, P_1) of one prediction + update from
    N(m0, P0), cross-checked against the dense posterior with T = 1."""
    rng = np.random.default_rng(31)
    mod = pins.rand_model(3, 2, rng)
    y = rng.standard_normal((1, 2))
    a1 = L.filter_element_first(mod.F, mod.u, mod.Q, mod.H, mod.d, mod.R, y[0], mod.m0, mod.P0)
    dm, dP = pins.dense_posterior(mod, y)
    assert np.all(a1.A == 0)
    assert relerr(a1.b, dm[1]) < 1e-10 and relerr(a1.C, dP[1]) < 1e-10


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lemma4_equals_definition1_joint(n):
    """Lemma 4 equals Definition 1 evaluated on Gaussian (f, g) pairs by
    joint-Gaussian algebra (Appendix C's identities not used)."""
    rng = np.random.default_rng(40 + n)
    ai, aj = rand_felem(n, rng), rand_felem(n, rng)
    got = L.filter_combine(ai, aj)
    ref = pins.filter_combine_by_joint(ai, aj)
    for x, r in zip(got, ref):
        assert relerr(x, r) < 1e-6


def test_lemma4_equals_definition1_quadrature():
    """Scalar case: Definition 1's integrals by numerical quadrature."""
    rng = np.random.default_rng(50)
    ai, aj = rand_felem(1, rng), rand_felem(1, rng)
    c = L.filter_combine(ai, aj)
    xs = np.array([-1.0, 0.3, 1.2])
    zs = np.array([0.5, -0.7, 1.1])
    f, lg = pins.filter_combine_by_quadrature(ai, aj, xs, zs)
    A, b, C, eta, J = (float(np.asarray(v).reshape(-1)[0]) for v in c)
    np.testing.assert_allclose(f, pins.gauss(xs, A * zs + b, C), rtol=1e-7)
    np.testing.assert_allclose(lg, -0.5 * J * zs ** 2 + eta * zs, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_lemma5_equals_joint_conditioning(n):
    rng = np.random.default_rng(60 + n)
    F = rng.standard_normal((n, n)) / np.sqrt(n)
    u = rng.standard_normal(n)
    Q = pins.rand_spd(n, rng, 0.3)
    xbar = rng.standard_normal(n)
    P = pins.rand_spd(n, rng)
    got = L.smoother_element(F, u, Q, xbar, P)
    ref = pins.smoother_element_by_joint(F, u, Q, xbar, P)
    for x, r in zip(got, ref):
        assert relerr(x, r) < 1e-8


def test_lemma6_equals_definition2_quadrature():
    rng = np.random.default_rng(70)
    ai, aj = rand_selem(1, rng), rand_selem(1, rng)
    c = L.smoother_combine(ai, aj)
    xs = np.array([-0.4, 0.2, 1.5])
    zs = np.array([1.0, -2.0, 0.3])
    got = pins.smoother_combine_by_quadrature(ai, aj, xs, zs)
    E, g, Lv = (float(np.asarray(v).reshape(-1)[0]) for v in c)
    np.testing.assert_allclose(got, pins.gauss(xs, E * zs + g, Lv), rtol=1e-7)


def test_lemma6_equals_definition2_monte_carlo():
    """Definition 2 by sampling y ~ a_j(.|z), x ~ a_i(.|y) (n = 3)."""
    rng = np.random.default_rng(71)
    n, N = 3, 400_000
    ai, aj = rand_selem(n, rng), rand_selem(n, rng)
    z = rng.standard_normal(n)
    y = (aj.E @ z + aj.g) + rng.standard_normal((N, n)) @ np.linalg.cholesky(aj.L).T
    x = y @ ai.E.T + ai.g + rng.standard_normal((N, n)) @ np.linalg.cholesky(ai.L).T
    c = L.smoother_combine(ai, aj)
    se = np.sqrt(np.max(np.diag(c.L)) / N)
    assert np.max(np.abs(x.mean(0) - (c.E @ z + c.g))) < 6 * se
    assert np.max(np.abs(np.cov(x.T) - c.L)) < 0.02 * np.max(np.abs(c.L))


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32])
def test_filter_operator_associative(n):
    """Appendix A: [a_i ⊗ a_j] ⊗ a_k = a_i ⊗ [a_j ⊗ a_k] (Lemma 4)."""
    rng = np.random.default_rng(80 + n)
    a, b, c = (rand_felem(n, rng) for _ in range(3))
    lhs = L.filter_combine(L.filter_combine(a, b), c)
    rhs = L.filter_combine(a, L.filter_combine(b, c))
    for x, y in zip(lhs, rhs):
        assert relerr(x, y) < 1e-9


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32])
def test_smoother_operator_associative(n):
    """Appendix B: [a_i ⊗ a_j] ⊗ a_k = a_i ⊗ [a_j ⊗ a_k] (Lemma 6)."""
    rng = np.random.default_rng(90 + n)
    a, b, c = (rand_selem(n, rng) for _ in range(3))
    lhs = L.smoother_combine(L.smoother_combine(a, b), c)
    rhs = L.smoother_combine(a, L.smoother_combine(b, c))
    for x, y in zip(lhs, rhs):
        assert relerr(x, y) < 1e-10


@pytest.mark.parametrize("n", [2, 4])
def test_identity_elements(n):
    rng = np.random.default_rng(95 + n)
    a = rand_felem(n, rng)
    e = L.filter_identity(n)
    for x, y in zip(L.filter_combine(e, a), a):
        assert relerr(x, y) < 1e-14
    for x, y in zip(L.filter_combine(a, e), a):
        assert relerr(x, y) < 1e-14
    s = rand_selem(n, rng)
    es = L.smoother_identity(n)
    for x, y in zip(L.smoother_combine(es, s), s):
        assert relerr(x, y) < 1e-14
    for x, y in zip(L.smoother_combine(s, es), s):
        assert relerr(x, y) < 1e-14


# ------------------------------------------------------------------ Theorems 1 and 2
@pytest.mark.parametrize("case", ["tracking", "random", "time_varying"])
def test_parallel_formulation_equals_sequential(case):
    """Section V's claim that the parallel algorithms give exactly the
    sequential KF/RTS result: prefix sums of Lemma 3 elements under Lemma 4
    and suffix sums of Lemma 5 elements under Lemma 6 equal the C oracle."""
    rng = np.random.default_rng(123)
    if case == "tracking":
        seq = workloads.tracking_sequence(64, seed=9)
        model, y = seq.model, seq.y
    elif case == "random":
        model = pins.rand_model(3, 2, rng)
        y = rng.standard_normal((50, 2))
    else:
        model = pins.rand_model(3, 2, rng, T=30)
        y = rng.standard_normal((30, 2))
    fm, fP, sm, sP = oracle.kf_rts(model, y)
    pfm, pfP = L.parallel_filter(model, y)
    psm, psP = L.parallel_smoother(model, fm, fP)
    assert relerr(pfm, fm) < 1e-10 and relerr(pfP, fP) < 1e-10
    assert relerr(psm, sm) < 1e-10 and relerr(psP, sP) < 1e-10


def test_first_element_information_reading_is_irrelevant():
    """eta_1 and J_1 cannot reach any filtering mean or covariance because
    A_1 = 0: using Lemma 3's k > 1 formulas for them at k = 1 changes nothing."""
    seq = workloads.tracking_sequence(40, seed=21)
    m = seq.model
    el = L.filter_elements(m, seq.y)
    alt = L.filter_element(m.F, m.u, m.Q, m.H, m.d, m.R, seq.y[0])
    el_alt = [el[0]._replace(eta=alt.eta, J=alt.J)] + el[1:]
    p1 = L.all_prefix_sums(el, L.filter_combine)
    p2 = L.all_prefix_sums(el_alt, L.filter_combine)
    for a, b in zip(p1, p2):
        assert relerr(a.b, b.b) < 1e-12 and relerr(a.C, b.C) < 1e-12
