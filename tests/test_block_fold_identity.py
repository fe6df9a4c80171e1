"""The identity the linear block fold is built on (no GPU), checked with the
oracle's Lemma 3/4 functions in FP64.

For a time-invariant model the Lemma 4 fold of a block of measurement
elements has (b, eta) affine in the block's measurements.  Its terms in the
first measurement y_0 come from a noise-free trajectory: for any state z,
the trajectory x_i = F x_{i-1} + u from x_prev = z yields measurements
ybar_i = H x_i + d for which b = x_end - A z and eta = J z, so

    b   = x_end - A L y_0 + sum_i Bc_i (y_i - ybar_i),
    eta = J L y_0 + sum_i Ec_i (y_i - ybar_i)

with z = L y_0, for every N x M matrix L.  The kernels take
L = H^T (H H^T)^{-1}."""
import zlib
from functools import reduce

import numpy as np
import pytest

import workloads
from oracle import lemmas as lm


def fold(m, u, d, ys):
    return reduce(lm.filter_combine, [lm.filter_element(m.F, u, m.Q, m.H, d, m.R, y) for y in ys])


def coefficients(m, u, d, ch):
    """Per-position responses Bc_i, Ec_i of (b, eta) to y_i, by unit impulses."""
    p = m.H.shape[0]
    base = fold(m, u, d, np.zeros((ch, p)))
    Bc, Ec = [], []
    for i in range(ch):
        cb, ce = [], []
        for r in range(p):
            ys = np.zeros((ch, p))
            ys[i, r] = 1.0
            a = fold(m, u, d, ys)
            cb.append(a.b - base.b)
            ce.append(a.eta - base.eta)
        Bc.append(np.array(cb).T)
        Ec.append(np.array(ce).T)
    return base, Bc, Ec


@pytest.mark.parametrize("case", ["wiener2", "wiener4", "stable6", "stable5"])
@pytest.mark.parametrize("lift", ["pinv", "random", "zero"])
def test_lifted_trajectory_gives_the_terms_in_y0(case, lift):
    rng = np.random.default_rng(zlib.crc32(f"{case}-{lift}".encode()))
    if case.startswith("wiener"):
        m = workloads.wiener_velocity(int(case[-1]) // 2, dt=0.1, q=1.3, r=0.4)
    else:
        n = int(case[-1])
        m = workloads.random_stable(n, n // 2, rng)
    n, p = m.F.shape[0], m.H.shape[0]
    u, d = rng.standard_normal(n), rng.standard_normal(p)
    ch = 8
    base, Bc, Ec = coefficients(m, u, d, ch)
    L = {"pinv": m.H.T @ np.linalg.inv(m.H @ m.H.T), "random": rng.standard_normal((n, p)),
         "zero": np.zeros((n, p))}[lift]
    V, c = L.copy(), np.zeros(n)
    Bs, Es, bc, ec = np.zeros((n, p)), np.zeros((n, p)), np.zeros(n), np.zeros(n)
    for i in range(ch):
        V, c = m.F @ V, m.F @ c + u            # F^{i+1} L, c_{i+1}
        G, g = m.H @ V, m.H @ c + d            # ybar_i = G y_0 + g
        Bs += Bc[i] @ (G - np.eye(p))
        Es += Ec[i] @ (G - np.eye(p))
        bc += Bc[i] @ g
        ec += Ec[i] @ g
    Bs, bc = V - base.A @ L - Bs, c - bc
    Es, ec = base.J @ L - Es, -ec
    for trial in range(3):
        ys = rng.standard_normal((ch, p)) * 5 + 40 * trial
        ref = fold(m, u, d, ys)
        b = bc + Bs @ ys[0] + sum(Bc[i] @ (ys[i] - ys[0]) for i in range(1, ch))
        eta = ec + Es @ ys[0] + sum(Ec[i] @ (ys[i] - ys[0]) for i in range(1, ch))
        np.testing.assert_allclose(b, ref.b, rtol=1e-10, atol=1e-10 * np.abs(ref.b).max())
        np.testing.assert_allclose(eta, ref.eta, rtol=1e-10, atol=1e-10 * np.abs(ref.eta).max())


def test_tracking_lift_is_stationary():
    """With L = H^T (H H^T)^{-1} on the tracking model the lifted state has
    zero velocity, so its trajectory stays put: G_i = I, g_i = 0 (u = d = 0)
    and the coefficient of y_0 is (I - A) L, built from the block's own A."""
    m = workloads.wiener_velocity(2, dt=0.1, q=1.0, r=1.0)
    L = m.H.T @ np.linalg.inv(m.H @ m.H.T)
    V = L.copy()
    for _ in range(32):
        V = m.F @ V
        np.testing.assert_array_equal(m.H @ V, np.eye(2))
    np.testing.assert_array_equal(V, L)
