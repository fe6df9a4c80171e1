"""Seeded synthetic workloads for the temporally parallel Kalman filter / RTS smoother.

This module is shared by the tests, the benchmark and the smoke check.  It only
builds state-space models and simulates them: it holds no filtering or
smoothing arithmetic.  Both the CUDA path and the FP64 oracle are fed from here.

Models follow the linear/Gaussian state-space form of Section IV,

    x_k = F x_{k-1} + u + q_{k-1},  q ~ N(0, Q)
    y_k = H x_k + d + r_k,          r ~ N(0, R),   x_0 ~ N(m0, P0),

with time-invariant parameters, except the time-varying workloads at the end
(one parameter set per step, Section II's F_{k-1}, Q_{k-1}, H_k, R_k).

Precision convention: F, u, Q, H, d, R and y are rounded to FP32 once (the
GPU computes in FP32) and kept as float64 arrays holding those FP32 values, so
that the oracle sees exactly the inputs the GPU sees.  m0 and P0 stay FP64,
because the k = 1 element is built in FP64 on the GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1905130020


def _f32(a) -> np.ndarray:
    """Round to FP32 and return as float64 (exactly the values the GPU reads)."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Model:
    """Time-invariant linear/Gaussian state-space model (Section IV)."""

    F: np.ndarray
    u: np.ndarray
    Q: np.ndarray
    H: np.ndarray
    d: np.ndarray
    R: np.ndarray
    m0: np.ndarray
    P0: np.ndarray
    name: str = ""

    @property
    def nx(self) -> int:
        return self.F.shape[-1]

    @property
    def ny(self) -> int:
        return self.H.shape[-2]

    @property
    def time_varying(self) -> bool:
        return self.F.ndim == 3

    def f32(self) -> dict:
        """The FP32 arrays the GPU path reads (m0, P0 stay FP64)."""
        return {
            "F": self.F.astype(np.float32), "u": self.u.astype(np.float32),
            "Q": self.Q.astype(np.float32), "H": self.H.astype(np.float32),
            "d": self.d.astype(np.float32), "R": self.R.astype(np.float32),
            "m0": self.m0.astype(np.float64), "P0": self.P0.astype(np.float64),
        }


def make_model(F, Q, H, R, m0, P0, u=None, d=None, name="") -> Model:
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    H = np.atleast_2d(np.asarray(H, dtype=np.float64))
    nx, ny = F.shape[0], H.shape[0]
    u = np.zeros(nx) if u is None else np.asarray(u, dtype=np.float64)
    d = np.zeros(ny) if d is None else np.asarray(d, dtype=np.float64)
    return Model(F=_f32(F), u=_f32(u), Q=_f32(Q), H=_f32(H), d=_f32(d), R=_f32(R),
                 m0=np.asarray(m0, dtype=np.float64).reshape(nx),
                 P0=np.asarray(P0, dtype=np.float64).reshape(nx, nx), name=name)


def wiener_velocity(dim: int = 2, dt: float = 0.1, q: float = 1.0, r: float = 1.0,
                    m0=None, P0=None) -> Model:
    """Constant-velocity (Wiener-velocity) tracking model of Section V.

    State = (positions_1..dim, velocities_1..dim), measurement = positions.
    F and Q are the Section V matrices generalised from 2-D to ``dim`` axes
    (each axis independent); R = r I.
    """
    I = np.eye(dim)
    Z = np.zeros((dim, dim))
    F = np.block([[I, dt * I], [Z, I]])
    Q = q * np.block([[dt ** 3 / 3 * I, dt ** 2 / 2 * I], [dt ** 2 / 2 * I, dt * I]])
    H = np.hstack([I, Z])
    R = r * np.eye(dim)
    nx = 2 * dim
    m0 = np.zeros(nx) if m0 is None else m0
    P0 = np.eye(nx) if P0 is None else P0
    return make_model(F, Q, H, R, m0, P0, name=f"wiener_velocity_{dim}d")


def random_stable(nx: int, ny: int, rng: np.random.Generator, q: float = 0.1,
                  r: float = 0.5, lo: float = 0.9, hi: float = 0.99) -> Model:
    """Random stable model: F = O diag(U[lo, hi]), O Haar-orthogonal, Q = qI,
    H_ij ~ N(0, 1/nx) (variance 1/nx), R = rI, m0 = 0, P0 = I."""
    G = rng.standard_normal((nx, nx))
    O, Rq = np.linalg.qr(G)
    O = O * np.sign(np.diag(Rq))[None, :]
    F = O @ np.diag(rng.uniform(lo, hi, size=nx))
    H = rng.standard_normal((ny, nx)) / math.sqrt(nx)
    return make_model(F, q * np.eye(nx), H, r * np.eye(ny), np.zeros(nx), np.eye(nx),
                      name=f"random_stable_{nx}x{ny}")


def _chol_psd(S: np.ndarray) -> np.ndarray:
    try:
        return np.linalg.cholesky(S)
    except np.linalg.LinAlgError:
        w, V = np.linalg.eigh(S)
        return V * np.sqrt(np.clip(w, 0.0, None))[None, :]


def simulate(model: Model, T: int, rng: np.random.Generator, block: int = 256):
    """Draw x_0 ~ N(m0, P0), x_k = F x_{k-1} + u + q, y_k = H x_k + d + r.

    Returns (x[T+1, nx] FP64 states including x_0, y[T, ny] FP32-representable).
    The linear recursion is evaluated blockwise (exact in FP64 up to rounding
    order), so that T = 2^20 takes well under a second.
    """
    nx, ny = model.nx, model.ny
    x0 = model.m0 + _chol_psd(model.P0) @ rng.standard_normal(nx)
    W = rng.standard_normal((T, nx)) @ _chol_psd(model.Q).T + model.u[None, :]
    V = rng.standard_normal((T, ny)) @ _chol_psd(model.R).T + model.d[None, :]
    X = np.empty((T, nx))
    if T <= block:
        x = x0
        for k in range(T):
            x = model.F @ x + W[k]
            X[k] = x
    else:
        nb = -(-T // block)
        Wp = np.zeros((nb * block, nx))
        Wp[:T] = W
        Wp = Wp.reshape(nb, block, nx)
        Z = np.empty_like(Wp)
        carry = np.zeros((nb, nx))
        for i in range(block):          # within-block response from a zero state
            carry = carry @ model.F.T + Wp[:, i]
            Z[:, i] = carry
        Fpow = np.empty((block, nx, nx))
        P = np.eye(nx)
        for i in range(block):
            P = model.F @ P
            Fpow[i] = P
        s = x0
        Xp = np.empty((nb, block, nx))
        for b in range(nb):             # carry the block-start state
            Xp[b] = np.einsum("ijk,k->ij", Fpow, s) + Z[b]
            s = Xp[b, -1]
        X = Xp.reshape(nb * block, nx)[:T]
    Y = X @ model.H.T + V
    return np.vstack([x0[None, :], X]), _f32(Y)


@dataclass
class Sequence:
    model: Model
    y: np.ndarray          # [T, ny], FP32-representable float64
    x: np.ndarray = field(default=None, repr=False)   # true states [T+1, nx]

    @property
    def T(self) -> int:
        return self.y.shape[0]


def tracking_sequence(T: int, seed: int, r: float = 1.0, q: float = 1.0,
                      dt: float = 0.1) -> Sequence:
    """Single-sequence workload: 2-D Wiener-velocity model (nx=4, ny=2),
    dt=0.1, q=1, R=rI, m0=0, P0=I, simulated from ``seed``."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    m = wiener_velocity(2, dt=dt, q=q, r=r)
    x, y = simulate(m, T, rng)
    return Sequence(m, y, x)


def config_single(T: int = 1024) -> Sequence:
    """nx=4 tracking workload, T=1024 (seed SEED_BASE+1)."""
    return tracking_sequence(T, SEED_BASE + 1)


def config_long(T: int = 1 << 20) -> Sequence:
    """nx=4 tracking workload, T=2^20 (seed SEED_BASE+2)."""
    return tracking_sequence(T, SEED_BASE + 2)


def config_precision(T: int = 65536, nx: int = 32, ny: int = 8) -> Sequence:
    """Random stable model nx=32, ny=8, Q=0.1I, R=0.5I (seed SEED_BASE+4)."""
    rng = np.random.default_rng(np.random.PCG64(SEED_BASE + 4))
    m = random_stable(nx, ny, rng)
    x, y = simulate(m, T, rng)
    return Sequence(m, y, x)


def batch_lengths(B: int, rng: np.random.Generator, lo: int, hi: int) -> np.ndarray:
    """T_i = round(exp(U[ln lo, ln hi])) (log-uniform lengths)."""
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=B))).astype(np.int64)


def config_batched(B: int = 4096, lo: int = 256, hi: int = 16384,
                   nx_choices=(2, 4, 6), seed: int = SEED_BASE + 3) -> list[Sequence]:
    """Batched workload: B independent sequences, log-uniform lengths in
    [lo, hi], nx uniform in ``nx_choices`` (Wiener-velocity in nx/2 axes,
    ny = nx/2), q ~ U[0.5, 2], R = rI with r ~ U[0.1, 1], dt = 0.1, m0=0, P0=I."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    Ts = batch_lengths(B, rng, lo, hi)
    nxs = rng.choice(np.asarray(nx_choices), size=B)
    qs = rng.uniform(0.5, 2.0, size=B)
    rs = rng.uniform(0.1, 1.0, size=B)
    out = []
    for i in range(B):
        m = wiener_velocity(int(nxs[i]) // 2, dt=0.1, q=float(qs[i]), r=float(rs[i]))
        x, y = simulate(m, int(Ts[i]), rng)
        out.append(Sequence(m, y, x))
    return out


def to_f32_y(seq: Sequence) -> np.ndarray:
    return np.ascontiguousarray(seq.y.astype(np.float32))


# ---------------------------------------------------------------- serving workload
@dataclass
class Arrival:
    """One request of the serving workload: scheduled arrival time (s), the
    state size, its length and which model of the size's model set it uses."""
    t: float
    nx: int
    T: int
    model: int


def serving_models(n_per_size: int = 16, seed: int = SEED_BASE + 5) -> dict:
    """Model sets of the serving workload: nx = 4 (2-D Wiener velocity, ny = 2,
    q ~ U[0.5, 2], R = rI with r ~ U[0.1, 1]) and nx = 8 (random stable, ny = 4,
    the nx = 32 recipe at nx = 8: F = O diag(U[0.9, 0.99]), Q = 0.1 I,
    H ~ N(0, 1/8), R = 0.5 I); dt = 0.1, m0 = 0, P0 = I."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    out = {4: [], 8: []}
    for _ in range(n_per_size):
        out[4].append(wiener_velocity(2, dt=0.1, q=float(rng.uniform(0.5, 2.0)), r=float(rng.uniform(0.1, 1.0))))
        out[8].append(random_stable(8, 4, rng))
    return out


def serving_arrivals(rate: float, n: int, seed: int, lo: int = 64, hi: int = 1 << 18,
                     sizes=(4, 8), n_models: int = 16) -> list:
    """Open-loop Poisson arrivals at ``rate`` requests/s: exponential gaps,
    T = round(exp(U[ln lo, ln hi])), nx uniform over ``sizes``, model index
    uniform over the size's set."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    Ts = batch_lengths(n, rng, lo, hi)
    nxs = rng.choice(np.asarray(sizes), size=n)
    ms = rng.integers(0, n_models, size=n)
    return [Arrival(float(t[i]), int(nxs[i]), int(Ts[i]), int(ms[i])) for i in range(n)]


def serving_measurements(models: dict, T: int, seed: int = SEED_BASE + 5) -> dict:
    """One simulated measurement sequence of length T per model (requests
    use a prefix of their model's sequence): {nx: [y (T, ny) FP32]}."""
    out = {}
    for nx, ms in models.items():
        out[nx] = []
        for i, m in enumerate(ms):
            rng = np.random.default_rng(np.random.PCG64(seed * 1000 + nx * 100 + i))
            _, y = simulate(m, T, rng)
            out[nx].append(np.ascontiguousarray(y.astype(np.float32)))
    return out


# ---------------------------------------------------------------- time-varying workloads
def _wiener_blocks(dts: np.ndarray, dim: int, q: float):
    """Per-step Wiener-velocity F_k, Q_k for sampling intervals dts [T]."""
    T = dts.shape[0]
    nx = 2 * dim
    I = np.eye(dim)
    F = np.zeros((T, nx, nx))
    F[:, :dim, :dim] = I
    F[:, dim:, dim:] = I
    F[:, :dim, dim:] = dts[:, None, None] * I
    Q = np.zeros((T, nx, nx))
    Q[:, :dim, :dim] = q * (dts ** 3 / 3)[:, None, None] * I
    Q[:, :dim, dim:] = q * (dts ** 2 / 2)[:, None, None] * I
    Q[:, dim:, :dim] = q * (dts ** 2 / 2)[:, None, None] * I
    Q[:, dim:, dim:] = q * dts[:, None, None] * I
    return F, Q


def irregular_tracking(T: int, seed: int, dim: int = 2, q: float = 1.0, dt_lo: float = 0.02,
                       dt_hi: float = 0.5, r_lo: float = 0.25, r_hi: float = 4.0) -> Sequence:
    """Time-varying workload: the Wiener-velocity model of Section V observed
    at irregular times.  The interval before step k is dt_k ~ log-uniform
    [dt_lo, dt_hi] (F_k, Q_k follow from it) and the sensor noise of step k is
    R_k = r_k I with r_k ~ log-uniform [r_lo, r_hi]; H = [I 0], u = d = 0,
    m0 = 0, P0 = I.  The states are drawn exactly (per axis, the velocity is a
    cumulative sum of its noise and the position integrates it), so T = 2^20
    takes well under a second."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    nx = 2 * dim
    dts = np.exp(rng.uniform(math.log(dt_lo), math.log(dt_hi), size=T))
    rs = np.exp(rng.uniform(math.log(r_lo), math.log(r_hi), size=T))
    F, Q = _wiener_blocks(dts, dim, q)
    H = np.broadcast_to(np.hstack([np.eye(dim), np.zeros((dim, dim))]), (T, dim, nx)).copy()
    R = rs[:, None, None] * np.eye(dim)[None]
    model = Model(F=_f32(F), u=np.zeros((T, nx)), Q=_f32(Q), H=_f32(H), d=np.zeros((T, dim)), R=_f32(R),
                  m0=np.zeros(nx), P0=np.eye(nx), name=f"irregular_tracking_{dim}d")
    # exact simulation with the FP32-rounded parameters: per axis the step
    # noise (w_p, w_v) ~ N(0, q [[dt^3/3, dt^2/2], [dt^2/2, dt]])
    Fd, Qd = model.F, model.Q
    x0 = rng.standard_normal(nx)
    a = Qd[:, 0, 0]
    c = Qd[:, 0, dim]
    b = Qd[:, dim, dim]
    l11 = np.sqrt(a)
    l21 = c / l11
    l22 = np.sqrt(np.maximum(b - l21 * l21, 0.0))
    z = rng.standard_normal((T, 2, dim))
    wp = l11[:, None] * z[:, 0]
    wv = l21[:, None] * z[:, 0] + l22[:, None] * z[:, 1]
    v = x0[dim:][None, :] + np.cumsum(wv, axis=0)                 # v_k
    vprev = np.vstack([x0[dim:][None, :], v[:-1]])
    p = x0[:dim][None, :] + np.cumsum(Fd[:, 0, dim][:, None] * vprev + wp, axis=0)
    X = np.hstack([p, v])
    Y = p + np.sqrt(model.R[:, 0, 0])[:, None] * rng.standard_normal((T, dim))
    return Sequence(model, _f32(Y), np.vstack([x0[None, :], X]))


def random_time_varying(nx: int, ny: int, T: int, rng: np.random.Generator, q: float = 0.1,
                        r: float = 0.5) -> Sequence:
    """Dense time-varying model: per step F_k = O_k diag(U[0.9, 0.99]) with
    O_k Haar-orthogonal, Q_k = q (I + G G^T / nx), H_k ~ N(0, 1/nx),
    R_k = r (I + G' G'^T / ny), u_k ~ N(0, 0.1), d_k ~ N(0, 0.1); m0 ~ N(0, 1),
    P0 = 2 I.  The states are simulated step by step (small T only)."""
    G = rng.standard_normal((T, nx, nx))
    O, Rq = np.linalg.qr(G)
    O = O * np.sign(np.diagonal(Rq, axis1=1, axis2=2))[:, None, :]
    F = O * rng.uniform(0.9, 0.99, size=(T, 1, nx))
    A = rng.standard_normal((T, nx, nx))
    Q = q * (np.eye(nx)[None] + A @ A.transpose(0, 2, 1) / nx)
    H = rng.standard_normal((T, ny, nx)) / math.sqrt(nx)
    B = rng.standard_normal((T, ny, ny))
    R = r * (np.eye(ny)[None] + B @ B.transpose(0, 2, 1) / ny)
    u = 0.3 * rng.standard_normal((T, nx))
    d = 0.3 * rng.standard_normal((T, ny))
    model = Model(F=_f32(F), u=_f32(u), Q=_f32(Q), H=_f32(H), d=_f32(d), R=_f32(R),
                  m0=rng.standard_normal(nx), P0=2.0 * np.eye(nx), name=f"random_time_varying_{nx}x{ny}")
    x = model.m0 + _chol_psd(model.P0) @ rng.standard_normal(nx)
    X = np.empty((T, nx))
    Y = np.empty((T, ny))
    for k in range(T):
        x = model.F[k] @ x + model.u[k] + _chol_psd(model.Q[k]) @ rng.standard_normal(nx)
        X[k] = x
        Y[k] = model.H[k] @ x + model.d[k] + _chol_psd(model.R[k]) @ rng.standard_normal(ny)
    return Sequence(model, _f32(Y), np.vstack([model.m0[None, :], X]))


# ---------------------------------------------------------------- discrete-state workloads
@dataclass
class HmmSequence:
    pi: np.ndarray     # [K] prior of x_0
    Pi: np.ndarray     # [K, K] row-stochastic transitions
    lik: np.ndarray    # [T, K] p(y_k | x_k = j), FP32-representable
    x: np.ndarray = field(default=None, repr=False)   # true states [T]

    @property
    def T(self) -> int:
        return self.lik.shape[0]

    @property
    def K(self) -> int:
        return self.pi.shape[0]


def hmm_sequence(K: int, T: int, seed: int, stay: float = 0.95, sigma: float = 0.6) -> HmmSequence:
    """Regime-switching workload: K states, each kept with probability `stay`
    per step and otherwise left for another drawn from a Dirichlet(1) row;
    the measurement is y_k ~ N(x_k, sigma^2) (state j has mean j), given to
    the filter as its Gaussian likelihood row lik[k, j] = N(y_k; j, sigma^2).
    pi uniform.  Pi and lik are rounded to FP32 (the rows of Pi renormalised
    in FP64 first)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    off = rng.dirichlet(np.ones(K - 1), size=K) if K > 1 else np.zeros((1, 0))
    Pi = np.zeros((K, K))
    for i in range(K):
        Pi[i, i] = stay if K > 1 else 1.0
        Pi[i, [j for j in range(K) if j != i]] = (1.0 - stay) * off[i]
    Pi = _f32(Pi / Pi.sum(axis=1, keepdims=True))
    pi = _f32(np.full(K, 1.0 / K))
    x = np.empty(T, dtype=np.int64)
    u = rng.random(T + 1)
    cum = np.cumsum(Pi, axis=1)
    s = int(np.searchsorted(np.cumsum(pi), u[0] * np.cumsum(pi)[-1]))
    for k in range(T):
        s = int(min(np.searchsorted(cum[s], u[k + 1] * cum[s, -1]), K - 1))
        x[k] = s
    y = x + sigma * rng.standard_normal(T)
    mu = np.arange(K, dtype=np.float64)
    lik = np.exp(-0.5 * ((y[:, None] - mu[None, :]) / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))
    return HmmSequence(pi, Pi, _f32(lik), x)
