"""Host checks of the time-varying workload generators (no GPU): shapes,
ranges, and that the simulated states follow the per-step model."""
import numpy as np

import workloads


def test_irregular_tracking_shapes_and_ranges():
    s = workloads.irregular_tracking(5000, seed=3)
    m = s.model
    assert m.time_varying and m.nx == 4 and m.ny == 2
    assert m.F.shape == (5000, 4, 4) and m.Q.shape == (5000, 4, 4)
    assert m.H.shape == (5000, 2, 4) and m.R.shape == (5000, 2, 2)
    dt = m.F[:, 0, 2]
    assert dt.min() >= 0.02 * (1 - 1e-6) and dt.max() <= 0.5 * (1 + 1e-6)
    r = m.R[:, 0, 0]
    assert r.min() >= 0.25 * (1 - 1e-6) and r.max() <= 4.0 * (1 + 1e-6)
    assert np.all(np.linalg.eigvalsh(m.Q) > 0)


def test_irregular_tracking_follows_its_model():
    """Whitened process and measurement residuals of the drawn states have
    unit variance (the exact per-axis simulation matches F_k, Q_k, R_k)."""
    s = workloads.irregular_tracking(20000, seed=4)
    m = s.model
    X = s.x
    res = X[1:] - np.einsum("tij,tj->ti", m.F, X[:-1])
    L = np.linalg.cholesky(m.Q)
    z = np.linalg.solve(L, res[..., None])[..., 0]
    assert np.all(np.abs(z.var(axis=0) - 1) < 0.05), z.var(axis=0)
    v = s.y - np.einsum("tij,tj->ti", m.H, X[1:])
    w = v / np.sqrt(m.R[:, [0, 1], [0, 1]])
    assert np.all(np.abs(w.var(axis=0) - 1) < 0.05), w.var(axis=0)


def test_random_time_varying_shapes_and_spd():
    rng = np.random.default_rng(5)
    s = workloads.random_time_varying(6, 3, 50, rng)
    m = s.model
    assert m.F.shape == (50, 6, 6) and m.u.shape == (50, 6) and m.d.shape == (50, 3)
    assert np.all(np.linalg.eigvalsh(m.Q) > 0) and np.all(np.linalg.eigvalsh(m.R) > 0)
    assert np.all(np.abs(np.linalg.eigvals(m.F)) < 1)
