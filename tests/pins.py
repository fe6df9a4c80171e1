"""Independent reference computations that pin the oracle.

Nothing here reuses the oracle's formulas: every quantity is obtained by a
different route fixed by the mathematics (dense joint-Gaussian algebra,
numerical integration of the paper's general definitions, closed forms).
"""
from __future__ import annotations

import numpy as np


def rand_spd(n, rng, scale=1.0, floor=0.05):
    G = rng.standard_normal((n, n))
    return scale * (G @ G.T / n + floor * np.eye(n))


def rand_psd(n, rng, rank=None, scale=1.0):
    rank = n if rank is None else rank
    G = rng.standard_normal((n, rank))
    return scale * (G @ G.T / n)


class TinyModel:
    """Plain attribute container for a (possibly time-varying) model."""

    def __init__(self, F, u, Q, H, d, R, m0, P0):
        self.F, self.u, self.Q, self.H, self.d, self.R = F, u, Q, H, d, R
        self.m0, self.P0 = m0, P0


def rand_model(n, m, rng, T=None):
    """Random model; with T, every parameter varies per step."""
    def mat(shape):
        return rng.standard_normal(shape) / np.sqrt(shape[-1])

    if T is None:
        return TinyModel(mat((n, n)) * 0.9, rng.standard_normal(n) * 0.1, rand_spd(n, rng, 0.3),
                         mat((m, n)), rng.standard_normal(m) * 0.1, rand_spd(m, rng, 0.5),
                         rng.standard_normal(n), rand_spd(n, rng))
    return TinyModel(np.array([mat((n, n)) * 0.9 for _ in range(T)]),
                     rng.standard_normal((T, n)) * 0.1,
                     np.array([rand_spd(n, rng, 0.3) for _ in range(T)]),
                     np.array([mat((m, n)) for _ in range(T)]),
                     rng.standard_normal((T, m)) * 0.1,
                     np.array([rand_spd(m, rng, 0.5) for _ in range(T)]),
                     rng.standard_normal(n), rand_spd(n, rng))


def _at(x, i, base_ndim):
    x = np.asarray(x, dtype=np.float64)
    return x[i] if x.ndim == base_ndim + 1 else x


def dense_posterior(model, y):
    """Joint Gaussian posterior of (x_0, ..., x_T) given y_{1:T}, by assembling
    the joint precision of the whole trajectory and solving densely.

    Negative log density = 1/2 |x_0 - m0|^2_{P0^-1}
                         + sum_k 1/2 |x_k - F_{k-1} x_{k-1} - u_{k-1}|^2_{Q^-1}
                         + sum_k 1/2 |y_k - H_k x_k - d_k|^2_{R^-1}.
    Returns (mean[T+1, n], cov[T+1, n, n]) block marginals.
    """
    y = np.asarray(y, dtype=np.float64)
    T = y.shape[0]
    n = np.asarray(model.m0).shape[0]
    N = (T + 1) * n
    Lam = np.zeros((N, N))
    nu = np.zeros(N)

    def add(G, W, h):
        # residual r = G z - h with weight W
        nonlocal Lam, nu
        Lam += G.T @ W @ G
        nu += G.T @ W @ h

    G = np.zeros((n, N)); G[:, :n] = np.eye(n)
    add(G, np.linalg.inv(model.P0), np.asarray(model.m0, dtype=np.float64))
    for k in range(1, T + 1):
        i = k - 1
        F, u, Q = _at(model.F, i, 2), _at(model.u, i, 1), _at(model.Q, i, 2)
        H, d, R = _at(model.H, i, 2), _at(model.d, i, 1), _at(model.R, i, 2)
        G = np.zeros((n, N))
        G[:, k * n:(k + 1) * n] = np.eye(n)
        G[:, (k - 1) * n:k * n] = -F
        add(G, np.linalg.inv(Q), u)
        G = np.zeros((H.shape[0], N))
        G[:, k * n:(k + 1) * n] = H
        add(G, np.linalg.inv(R), y[i] - d)
    cov = np.linalg.inv(Lam)
    mean = cov @ nu
    means = mean.reshape(T + 1, n)
    covs = np.array([cov[k * n:(k + 1) * n, k * n:(k + 1) * n] for k in range(T + 1)])
    return means, covs


def dense_filter_smoother(model, y):
    """Filtered marginals p(x_k | y_{1:k}) (dense posterior of the first k
    measurements, last block) and smoothed marginals p(x_k | y_{1:T})."""
    y = np.asarray(y, dtype=np.float64)
    T = y.shape[0]
    sm, sP = dense_posterior(model, y)
    fm, fP = [], []
    for k in range(1, T + 1):
        sub = TinyModel(*(_prefix(getattr(model, a), k, nd) for a, nd in
                          (("F", 2), ("u", 1), ("Q", 2), ("H", 2), ("d", 1), ("R", 2))),
                        model.m0, model.P0)
        m_k, P_k = dense_posterior(sub, y[:k])
        fm.append(m_k[k]); fP.append(P_k[k])
    return np.array(fm), np.array(fP), sm[1:], sP[1:]


def _prefix(x, k, base_ndim):
    x = np.asarray(x, dtype=np.float64)
    return x[:k] if x.ndim == base_ndim + 1 else x


def dense_loglik(model, y):
    """log p(y_{1:T}) from the stacked Gaussian marginal of all measurements."""
    from scipy.stats import multivariate_normal
    y = np.asarray(y, dtype=np.float64)
    T, m = y.shape
    n = np.asarray(model.m0).shape[0]
    # x = Phi xi + c with xi = (x_0 - m0, q_1, ..., q_T) ~ N(0, blockdiag(P0, Q_0..))
    N = (T + 1) * n
    Phi = np.zeros((N, N)); c = np.zeros(N)
    Sxi = np.zeros((N, N))
    Phi[:n, :n] = np.eye(n); c[:n] = model.m0; Sxi[:n, :n] = model.P0
    for k in range(1, T + 1):
        F, u, Q = _at(model.F, k - 1, 2), _at(model.u, k - 1, 1), _at(model.Q, k - 1, 2)
        Phi[k * n:(k + 1) * n] = F @ Phi[(k - 1) * n:k * n]
        Phi[k * n:(k + 1) * n, k * n:(k + 1) * n] += np.eye(n)
        c[k * n:(k + 1) * n] = F @ c[(k - 1) * n:k * n] + u
        Sxi[k * n:(k + 1) * n, k * n:(k + 1) * n] = Q
    Sx = Phi @ Sxi @ Phi.T
    Hb = np.zeros((T * m, N)); db = np.zeros(T * m); Rb = np.zeros((T * m, T * m))
    for k in range(1, T + 1):
        H, d, R = _at(model.H, k - 1, 2), _at(model.d, k - 1, 1), _at(model.R, k - 1, 2)
        Hb[(k - 1) * m:k * m, k * n:(k + 1) * n] = H
        db[(k - 1) * m:k * m] = d
        Rb[(k - 1) * m:k * m, (k - 1) * m:k * m] = R
    mu = Hb @ c + db
    S = Hb @ Sx @ Hb.T + Rb
    return multivariate_normal(mu, S).logpdf(y.reshape(-1))


# ---------------------------------------------------------------- joint-Gaussian routes
def condition_joint(mu, Sigma, idx_keep, idx_obs, obs):
    """Conditional of a joint Gaussian through its precision matrix:
    p(x_keep | x_obs) has covariance Lam_kk^{-1} and mean
    mu_k - Lam_kk^{-1} Lam_ko (obs - mu_o)."""
    Lam = np.linalg.inv(Sigma)
    Lkk = Lam[np.ix_(idx_keep, idx_keep)]
    Lko = Lam[np.ix_(idx_keep, idx_obs)]
    cov = np.linalg.inv(Lkk)
    mean = mu[idx_keep] - cov @ Lko @ (obs - mu[idx_obs])
    return mean, cov


def affine_from_function(fun, n_in):
    """Recover (A, b) of an affine map z -> A z + b from evaluations."""
    b = fun(np.zeros(n_in))
    A = np.stack([fun(np.eye(n_in)[i]) - b for i in range(n_in)], axis=1)
    return A, b


def quadratic_from_function(fun, n_in):
    """Recover (J, eta) of q(z) = -1/2 z^T J z + eta^T z + c from evaluations
    (finite differences are exact for a quadratic up to rounding)."""
    f0 = fun(np.zeros(n_in))
    e = np.eye(n_in)
    fi = np.array([fun(e[i]) for i in range(n_in)])
    fmi = np.array([fun(-e[i]) for i in range(n_in)])
    J = np.zeros((n_in, n_in))
    for i in range(n_in):
        J[i, i] = -(fi[i] + fmi[i] - 2 * f0)
    for i in range(n_in):
        for j in range(i + 1, n_in):
            fij = fun(e[i] + e[j])
            # q(ei+ej) - q(ei) - q(ej) + q(0) = -J_ij
            J[i, j] = J[j, i] = -(fij - fi[i] - fi[j] + f0)
    eta = (fi - fmi) / 2.0
    return J, eta


def log_info_integral(J, eta, mu, C):
    """log of  ∫ exp(-1/2 y^T J y + eta^T y) N(y; mu, C) dy  for SPD C, by
    completing the square: with Lam = J + C^{-1}, h = eta + C^{-1} mu,
    value = 1/2 h^T Lam^{-1} h - 1/2 mu^T C^{-1} mu - 1/2 log det(C Lam)."""
    Ci = np.linalg.inv(C)
    Lam = J + Ci
    h = eta + Ci @ mu
    sign, ld = np.linalg.slogdet(C @ Lam)
    return 0.5 * h @ np.linalg.solve(Lam, h) - 0.5 * mu @ Ci @ mu - 0.5 * ld


def filter_combine_by_joint(ai, aj):
    """Definition 1 evaluated for Gaussian (f, g) pairs through the joint
    density of (y, x) given z, without Lemma 4's formulas.

    f_ij(x | z): y | z ~ N(A_i z + b_i, C_i), x | y ~ N(A_j y + b_j, C_j), the
    factor g_j(y) adds J_j / eta_j to the y-block of the joint precision; the
    x-block of the resulting Gaussian is f_ij.  g_ij(z) = g_i(z) ∫ g_j f_i dy
    is evaluated in closed form and its quadratic read off.
    """
    n = ai.A.shape[0]

    def joint_xgivenz(z):
        my = ai.A @ z + ai.b
        mx = aj.A @ my + aj.b
        S = np.block([[ai.C, ai.C @ aj.A.T], [aj.A @ ai.C, aj.A @ ai.C @ aj.A.T + aj.C]])
        Lam = np.linalg.inv(S)
        h = Lam @ np.concatenate([my, mx])
        Lam[:n, :n] += aj.J
        h[:n] += aj.eta
        cov = np.linalg.inv(Lam)
        mean = cov @ h
        return mean[n:], cov[n:, n:]

    A, b = affine_from_function(lambda z: joint_xgivenz(z)[0], n)
    C = joint_xgivenz(np.zeros(n))[1]

    def log_g(z):
        return (-0.5 * z @ ai.J @ z + ai.eta @ z
                + log_info_integral(aj.J, aj.eta, ai.A @ z + ai.b, ai.C))

    J, eta = quadratic_from_function(log_g, n)
    return A, b, C, eta, J


def smoother_element_by_joint(F, u, Q, xbar, P):
    """p(x_k | y_{1:k}, x_{k+1}) by conditioning the joint Gaussian of
    (x_k, x_{k+1}), x_k ~ N(xbar, P), x_{k+1} = F x_k + u + q."""
    n = xbar.shape[0]
    mu = np.concatenate([xbar, F @ xbar + u])
    S = np.block([[P, P @ F.T], [F @ P, F @ P @ F.T + Q]])
    keep, obs = np.arange(n), np.arange(n, 2 * n)
    E, g = affine_from_function(lambda x1: condition_joint(mu, S, keep, obs, x1)[0], n)
    L = condition_joint(mu, S, keep, obs, np.zeros(n))[1]
    return E, g, L


def filter_element_by_joint(F, u, Q, H, d, R, y):
    """p(x_k | y_k, x_{k-1}) by conditioning the joint of (x_k, y_k) given
    x_{k-1}; p(y_k | x_{k-1}) as a log density whose quadratic is read off."""
    from scipy.stats import multivariate_normal
    n, m = F.shape[0], H.shape[0]

    def cond(xprev):
        mx = F @ xprev + u
        mu = np.concatenate([mx, H @ mx + d])
        S = np.block([[Q, Q @ H.T], [H @ Q, H @ Q @ H.T + R]])
        return condition_joint(mu, S, np.arange(n), np.arange(n, n + m), y)

    A, b = affine_from_function(lambda z: cond(z)[0], n)
    C = cond(np.zeros(n))[1]
    S = H @ Q @ H.T + R
    J, eta = quadratic_from_function(
        lambda z: multivariate_normal(H @ (F @ z + u) + d, S).logpdf(y), n)
    return A, b, C, eta, J


# ---------------------------------------------------------------- 1-D quadrature
def gauss(x, m, v):
    return np.exp(-0.5 * (x - m) ** 2 / v) / np.sqrt(2 * np.pi * v)


def quad_grid(center, spread, npts=200001):
    y = np.linspace(center - spread, center + spread, npts)
    return y, y[1] - y[0]


def filter_combine_by_quadrature(ai, aj, xs, zs):
    """Definition 1 for scalar elements by numerical integration over y.

    Returns (f_ij(x|z) for each (x, z) pair, log g_ij(z) - log g_ij(0) for zs)."""
    s = lambda a: float(np.asarray(a).reshape(-1)[0])
    Ai, bi, Ci, ei, Ji = map(s, ai)
    Aj, bj, Cj, ej, Jj = map(s, aj)
    gj = lambda y: np.exp(-0.5 * Jj * y * y + ej * y)
    f = []
    for x, z in zip(xs, zs):
        y, dy = quad_grid(Ai * z + bi, 40 * np.sqrt(Ci))
        w = gj(y) * gauss(y, Ai * z + bi, Ci)
        num = np.trapezoid(w * gauss(x, Aj * y + bj, Cj), dx=dy)
        den = np.trapezoid(w, dx=dy)
        f.append(num / den)

    def log_g(z):
        y, dy = quad_grid(Ai * z + bi, 40 * np.sqrt(Ci))
        return (-0.5 * Ji * z * z + ei * z
                + np.log(np.trapezoid(gj(y) * gauss(y, Ai * z + bi, Ci), dx=dy)))

    lg0 = log_g(0.0)
    return np.array(f), np.array([log_g(z) - lg0 for z in zs])


def smoother_combine_by_quadrature(ai, aj, xs, zs):
    """Definition 2 for scalar elements: a_ij(x|z) = ∫ a_i(x|y) a_j(y|z) dy."""
    s = lambda a: float(np.asarray(a).reshape(-1)[0])
    Ei, gi, Li = map(s, ai)
    Ej, gj_, Lj = map(s, aj)
    out = []
    for x, z in zip(xs, zs):
        y, dy = quad_grid(Ej * z + gj_, 40 * np.sqrt(Lj))
        out.append(np.trapezoid(gauss(x, Ei * y + gi, Li) * gauss(y, Ej * z + gj_, Lj), dx=dy))
    return np.array(out)
