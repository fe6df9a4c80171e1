"""Lemmas 3-6 and the scans of Sections II-B / III in plain numpy FP64.

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke check
and the benchmark's CPU baseline use this module.

Each function states the formulas of the paper it writes out, in the paper's
order and notation, with no fusion or reordering.  Matrix inverses are taken
with ``numpy.linalg.inv`` where the paper writes an inverse.

Element representations
-----------------------
* filtering element  a = (A, b, C, eta, J)   (Lemma 3): the pair
  f(x | z) = N(x; A z + b, C),  g(z) ∝ N_I(z; eta, J)
* smoothing element  a = (E, g, L)           (Lemma 5):
  a(x | z) = N(x; E z + g, L)
"""
from __future__ import annotations

from typing import Callable, NamedTuple, Sequence

import numpy as np

inv = np.linalg.inv


class FElem(NamedTuple):
    A: np.ndarray
    b: np.ndarray
    C: np.ndarray
    eta: np.ndarray
    J: np.ndarray


class SElem(NamedTuple):
    E: np.ndarray
    g: np.ndarray
    L: np.ndarray


_KIND = {"F": 2, "u": 1, "Q": 2, "H": 2, "d": 1, "R": 2}


def _step(model, name, i):
    """Parameter ``name`` at step index i: a time-varying parameter carries one
    extra leading axis over its time-invariant shape."""
    x = np.asarray(getattr(model, name), dtype=np.float64)
    return x[i] if x.ndim == _KIND[name] + 1 else x


# ---------------------------------------------------------------- Lemma 3
def filter_element(F, u, Q, H, d, R, y) -> FElem:
    """Lemma 3, k > 1 (Section IV-A): parameters of
    f_k(x_k | x_{k-1}) = N(x_k; A_k x_{k-1} + b_k, C_k) and
    g_k(x_{k-1}) ∝ N_I(x_{k-1}; eta_k, J_k), with F = F_{k-1}, u = u_{k-1},
    Q = Q_{k-1}, H = H_k, d = d_k, R = R_k:

        S_k   = H Q H^T + R
        K_k   = Q H^T S_k^{-1}
        A_k   = (I - K_k H) F
        b_k   = u + K_k (y_k - H u - d)
        C_k   = (I - K_k H) Q
        eta_k = F^T H^T S_k^{-1} (y_k - H u - d)
        J_k   = F^T H^T S_k^{-1} H F
    """
    F, u, Q, H, d, R, y = (np.asarray(v, dtype=np.float64) for v in (F, u, Q, H, d, R, y))
    n = F.shape[0]
    I = np.eye(n)
    S = H @ Q @ H.T + R
    Sinv = inv(S)
    K = Q @ H.T @ Sinv
    A = (I - K @ H) @ F
    b = u + K @ (y - H @ u - d)
    C = (I - K @ H) @ Q
    eta = F.T @ H.T @ Sinv @ (y - H @ u - d)
    J = F.T @ H.T @ Sinv @ H @ F
    return FElem(A, b, C, eta, J)


def filter_element_first(F, u, Q, H, d, R, y, m0, P0) -> FElem:
    """Lemma 3, k = 1: Kalman prediction and update from x_0 ~ N(m0, P0),

        m1- = F m0 + u,   P1- = F P0 F^T + Q,   S_1 = H P1- H^T + R
        K_1 = P1- H^T S_1^{-1}
        A_1 = 0,   b_1 = m1- + K_1 (y_1 - H m1- - d),   C_1 = P1- - K_1 S_1 K_1^T

    and eta_1 = 0, J_1 = 0: with A_1 = 0 the term g_1 is p(y_1), a constant in
    x_0 (Theorem 1), so its information-form parameters vanish.  (Lemma 3's
    formula for eta_k, J_k at k = 1 is ambiguous about which S_1 it means;
    since A_1 = 0 neither value can reach any filtering mean or covariance.)
    """
    F, u, Q, H, d, R, y, m0, P0 = (np.asarray(v, dtype=np.float64)
                                   for v in (F, u, Q, H, d, R, y, m0, P0))
    n = F.shape[0]
    mm = F @ m0 + u
    Pm = F @ P0 @ F.T + Q
    S = H @ Pm @ H.T + R
    K = Pm @ H.T @ inv(S)
    A = np.zeros((n, n))
    b = mm + K @ (y - H @ mm - d)
    C = Pm - K @ S @ K.T
    return FElem(A, b, C, np.zeros(n), np.zeros((n, n)))


def filter_elements(model, y) -> list[FElem]:
    """Lemma 3 for k = 1..n (time-invariant or time-varying model)."""
    y = np.asarray(y, dtype=np.float64)
    T = y.shape[0]
    out = []
    for i in range(T):
        F, u, Q, H, d, R = (_step(model, name, i) for name in "F u Q H d R".split())
        if i == 0:
            out.append(filter_element_first(F, u, Q, H, d, R, y[0], model.m0, model.P0))
        else:
            out.append(filter_element(F, u, Q, H, d, R, y[i]))
    return out


# ---------------------------------------------------------------- Lemma 4
def filter_combine(ai: FElem, aj: FElem) -> FElem:
    """Lemma 4: (f_i, g_i) ⊗ (f_j, g_j) = (f_ij, g_ij) with

        A_ij   = A_j (I + C_i J_j)^{-1} A_i
        b_ij   = A_j (I + C_i J_j)^{-1} (b_i + C_i eta_j) + b_j
        C_ij   = A_j (I + C_i J_j)^{-1} C_i A_j^T + C_j
        eta_ij = A_i^T (I + J_j C_i)^{-1} (eta_j - J_j b_i) + eta_i
        J_ij   = A_i^T (I + J_j C_i)^{-1} J_j A_i + J_i
    """
    n = ai.A.shape[0]
    I = np.eye(n)
    M1 = inv(I + ai.C @ aj.J)
    M2 = inv(I + aj.J @ ai.C)
    A = aj.A @ M1 @ ai.A
    b = aj.A @ M1 @ (ai.b + ai.C @ aj.eta) + aj.b
    C = aj.A @ M1 @ ai.C @ aj.A.T + aj.C
    eta = ai.A.T @ M2 @ (aj.eta - aj.J @ ai.b) + ai.eta
    J = ai.A.T @ M2 @ aj.J @ ai.A + ai.J
    return FElem(A, b, C, eta, J)


def filter_identity(n: int) -> FElem:
    """Two-sided identity of Lemma 4's operator: (I, 0, 0, 0, 0).

    The paper gives no identity element (Fig. 1 needs one for its down-sweep);
    substituting into Lemma 4 shows e ⊗ a = a ⊗ e = a for this choice.
    """
    return FElem(np.eye(n), np.zeros(n), np.zeros((n, n)), np.zeros(n), np.zeros((n, n)))


# ---------------------------------------------------------------- Lemma 5
def smoother_element(F, u, Q, xbar, P) -> SElem:
    """Lemma 5, k < n: with F = F_k, u = u_k, Q = Q_k and the filtering mean
    and covariance (xbar_k, P_k),

        E_k = P_k F^T (F P_k F^T + Q)^{-1}
        g_k = xbar_k - E_k (F xbar_k + u)
        L_k = P_k - E_k F P_k
    """
    F, u, Q, xbar, P = (np.asarray(v, dtype=np.float64) for v in (F, u, Q, xbar, P))
    E = P @ F.T @ inv(F @ P @ F.T + Q)
    g = xbar - E @ (F @ xbar + u)
    L = P - E @ F @ P
    return SElem(E, g, L)


def smoother_element_last(xbar, P) -> SElem:
    """Lemma 5, k = n: E_n = 0, g_n = xbar_n, L_n = P_n."""
    xbar = np.asarray(xbar, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    n = xbar.shape[0]
    return SElem(np.zeros((n, n)), xbar.copy(), P.copy())


def smoother_elements(model, fmean, fcov) -> list[SElem]:
    """Lemma 5 for k = 1..n from filtered means/covariances.  The element at
    step i uses the transition out of step i (F_k in Lemma 5), which in the
    step-indexed arrays of the time-varying case is entry i + 1."""
    fmean = np.asarray(fmean, dtype=np.float64)
    fcov = np.asarray(fcov, dtype=np.float64)
    T = fmean.shape[0]
    out = []
    for i in range(T - 1):
        F, u, Q = (_step(model, name, i + 1) for name in "F u Q".split())
        out.append(smoother_element(F, u, Q, fmean[i], fcov[i]))
    out.append(smoother_element_last(fmean[T - 1], fcov[T - 1]))
    return out


# ---------------------------------------------------------------- Lemma 6
def smoother_combine(ai: SElem, aj: SElem) -> SElem:
    """Lemma 6: a_i ⊗ a_j = a_ij with

        E_ij = E_i E_j,   g_ij = E_i g_j + g_i,   L_ij = E_i L_j E_i^T + L_i
    """
    return SElem(ai.E @ aj.E, ai.E @ aj.g + ai.g, ai.E @ aj.L @ ai.E.T + ai.L)


def smoother_identity(n: int) -> SElem:
    """Two-sided identity of Lemma 6's operator: (I, 0, 0)."""
    return SElem(np.eye(n), np.zeros(n), np.zeros((n, n)))


# ---------------------------------------------------------------- scans
def all_prefix_sums(elems: Sequence, op: Callable) -> list:
    """Definition of all-prefix-sums (Section II-B):
    (a_1, a_1 ⊗ a_2, ..., a_1 ⊗ ... ⊗ a_n), evaluated left to right."""
    out = []
    acc = None
    for a in elems:
        acc = a if acc is None else op(acc, a)
        out.append(acc)
    return out


def all_suffix_sums(elems: Sequence, op: Callable) -> list:
    """Theorem 2's sums a_k ⊗ a_{k+1} ⊗ ... ⊗ a_n for k = 1..n.

    The operator is not commutative, so the earlier element stays the left
    operand: s_n = a_n, s_k = a_k ⊗ s_{k+1}.  (Running a prefix scan on the
    reversed sequence, as Section III-B suggests, gives the same sums only if
    the operands of each ⊗ are swapped back.)
    """
    out = [None] * len(elems)
    acc = None
    for k in range(len(elems) - 1, -1, -1):
        acc = elems[k] if acc is None else op(elems[k], acc)
        out[k] = acc
    return out


def parallel_filter(model, y):
    """Theorem 1 for the linear/Gaussian case: all-prefix-sums of the Lemma 3
    elements under Lemma 4; the filtering mean and covariance are b and C of
    each prefix (its A is 0 because A_1 = 0).  Returns (fmean, fcov)."""
    pre = all_prefix_sums(filter_elements(model, y), filter_combine)
    return np.array([p.b for p in pre]), np.array([p.C for p in pre])


def parallel_smoother(model, fmean, fcov):
    """Theorem 2 for the linear/Gaussian case: suffix sums of the Lemma 5
    elements under Lemma 6; the smoothed mean and covariance are g and L of
    each suffix (its E is 0 because E_n = 0).  Returns (smean, scov)."""
    suf = all_suffix_sums(smoother_elements(model, fmean, fcov), smoother_combine)
    return np.array([s.g for s in suf]), np.array([s.L for s in suf])
