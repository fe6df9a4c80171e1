"""GPU: marginal log-likelihood by one pass over the filtered moments
(ks_loglik) against the oracle's sequential log p(y_k | y_1:k-1).

The residual y_k - mu_k is formed in FP32, so the cases use stable models (or
a short Wiener-velocity sequence): at T = 2^20 the Wiener positions reach
~1e7, where one FP32 ulp is ~1 and the per-step term loses its digits."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    return ks


def gpu_model(ks, m):
    return ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, u=m.u, d=m.d, device="cuda")


def cases():
    out = []
    for nx, ny, T in [(4, 2, 5000), (8, 4, 3000), (32, 8, 2000), (2, 1, 1), (4, 2, 1)]:
        out.append(("stable", nx, ny, T))
    out.append(("wiener", 4, 2, 1000))
    out.append(("wiener", 6, 3, 700))
    return out


def make(kind, nx, ny, T, seed):
    rng = np.random.default_rng(seed)
    if kind == "stable":
        m = workloads.random_stable(nx, ny, rng)
        m = workloads.make_model(m.F, m.Q, m.H, m.R, 0.3 * rng.standard_normal(nx), np.eye(nx) * 1.5,
                                 u=0.05 * rng.standard_normal(nx), d=0.05 * rng.standard_normal(ny))
    else:
        m = workloads.wiener_velocity(nx // 2, dt=0.1, q=1.0, r=float(rng.uniform(0.1, 1)))
    _, y = workloads.simulate(m, T, rng)
    return m, y


@pytest.mark.parametrize("kind,nx,ny,T", cases())
def test_loglik_from_oracle_moments(ks, kind, nx, ny, T):
    """The kernel's arithmetic alone: FP32-rounded oracle filtered moments in."""
    m, y = make(kind, nx, ny, T, 700 + nx + T)
    fm, fc, ll_ref = oracle.kf(m, y, loglik=True)
    model = gpu_model(ks, m)
    dev = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()
    ll, total, st = ks.loglik(model, dev(y), dev(fm), dev(fc))
    assert int(st.item()) == 0
    ll = ll.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(ll, ll_ref, rtol=1e-4, atol=2e-4)
    assert abs(total.item() - ll_ref.sum()) <= 1e-5 * max(1.0, abs(ll_ref.sum())) + 2e-4 * np.sqrt(T)


@pytest.mark.parametrize("kind,nx,ny,T", cases())
def test_loglik_end_to_end(ks, kind, nx, ny, T):
    """The GPU filter's moments in: the total within 1e-4 relative of the oracle."""
    m, y = make(kind, nx, ny, T, 900 + nx + T)
    _, _, ll_ref = oracle.kf(m, y, loglik=True)
    model = gpu_model(ks, m)
    yt = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    fm, fc, _, _ = ks.smooth(model, yt, filter_only=True)
    ll, total, st = ks.loglik(model, yt, fm, fc)
    assert int(st.item()) == 0
    ref = ll_ref.sum()
    print(f"{kind} nx={nx} T={T} loglik {total.item():.6f} oracle {ref:.6f}")
    assert abs(total.item() - ref) <= 1e-4 * max(1.0, abs(ref))
    np.testing.assert_allclose(ll.cpu().numpy(), ll_ref, rtol=1e-3, atol=2e-3)


def test_loglik_rejects_missing_outputs(ks):
    import ctypes
    m, y = make("stable", 4, 2, 10, 1)
    model = gpu_model(ks, m)
    yt = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = ks.lib().ks_loglik(ctypes.byref(model.struct()), ks._p(yt), 10, ks._p(yt), ks._p(yt), None, None,
                            ks._p(st), ks._stream(None))
    assert rc == ks.KS_EINVAL
