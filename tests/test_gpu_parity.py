"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every comparison is element by element over all steps on seeded inputs.
Tolerances: tests/parity.py (1e-4 normwise per step for FP32, and the
posterior-sd bound on every mean).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import lemmas as L
import parity
import pins
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


def run_smooth(ks, m, y, with_ws=False):
    model = gpu_model(ks, m)
    yt = torch.as_tensor(np.asarray(y), dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, yt.shape[0])
    out = ks.smooth(model, yt, ws)
    assert ks.status(ws) == ks.KS_OK
    return (out, ws) if with_ws else out


def check(ks, m, y, tol=parity.TOL, refined=None):
    """Parity against the oracle; refined = True / False additionally asserts
    that some / no inverse got the FP64 refinement step."""
    got, ws = run_smooth(ks, m, y, with_ws=True)
    ref = oracle.kf_rts(m, np.asarray(y, dtype=np.float64))
    e = parity.check_all(got, ref, tol)
    n = ks.refinements(ws)
    e["refinements"] = n
    if refined is not None:
        assert (n > 0) == refined, ("refinement count", n)
    return e


def scaled_model(m, d):
    """The model in rescaled state coordinates x' = D x, D = diag(d) (state
    components in units of very different size): F' = D F D^-1, Q' = D Q D,
    H' = H D^-1, m0' = D m0, P0' = D P0 D, same measurements.  Its posteriors
    are D times the original's.  Lemma 4's I + C_i J_j becomes
    D (I + C_i J_j) D^-1, so its 1-norm condition number grows with the
    spread of d: the cross-block combines of these tests exceed the 1e3
    threshold of the FP64 refinement."""
    D = np.diag(np.asarray(d, dtype=np.float64))
    Di = np.diag(1.0 / np.asarray(d, dtype=np.float64))
    return workloads.make_model(D @ m.F @ Di, D @ m.Q @ D, m.H @ Di, m.R, D @ m.m0, D @ m.P0 @ D,
                                u=None if m.u is None else D @ m.u, d=m.d)


# Sizes span one tile (2048 steps) and many, with ragged tails, and the
# degenerate T = 1 and T = 2.
@pytest.mark.parametrize("T", [1, 2, 3, 15, 16, 17, 33, 511, 2047, 2048, 2049, 4096, 4097, 6150, 20001])
def test_tracking_model_sizes(ks, T):
    seq = workloads.tracking_sequence(T, seed=1000 + T)
    check(ks, seq.model, seq.y)



# The fused smooth picks 4, 8, 16 or 32 steps per thread by T (switching at
# 96 Ki, 192 Ki and 640 Ki steps): both sides of every switch, each with a
# ragged last tile, for nx = 4, and one size inside each band for nx = 2, 6.
# At 32 steps per thread a single sequence builds each step's Lemma 5 element
# one iteration late, and the reverse scan applies its elements in pairs from
# groups of 4: last blocks of 1 and 19 steps (groups of 4, 4, 4, 4, 3) cover both tails.
@pytest.mark.parametrize("dim,T", [(2, 98303), (2, 98304), (2, 196607), (2, 196608), (2, 655359),
                                   (2, 655360), (2, 655361), (2, 700019), (1, 150001), (1, 400003),
                                   (1, 655361), (3, 150001), (3, 400003), (3, 700001)])
def test_chunk_variants(ks, dim, T):
    rng = np.random.default_rng(4000 + T + dim)
    m = workloads.wiener_velocity(dim, dt=0.1, q=1.0, r=0.5)
    _, y = workloads.simulate(m, T, rng)
    check(ks, m, y)

# Every (steps per thread, block fold) variant of the fused scans, forced by a
# one-rule table, on sizes with ragged ends; the table is restored after.
@pytest.mark.parametrize("dim,T", [(1, 9001), (2, 70001), (3, 30001)])
@pytest.mark.parametrize("steps,fold", [(4, 1), (8, 1), (16, 1), (32, 1), (32, 0)])
def test_block_fold_variants(ks, dim, T, steps, fold):
    from paper_1905_13002_gb300 import tune
    rng = np.random.default_rng(4100 + T + dim)
    m = workloads.wiener_velocity(dim, dt=0.1, q=1.3, r=0.4)
    m.u = rng.standard_normal(2 * dim) * 0.1        # the affine terms of the fold
    m.d = rng.standard_normal(dim) * 0.1
    _, y = workloads.simulate(m, T, rng)
    ks.set_chunk_rules(2 * dim, [(tune.T_NEVER, steps, fold)])
    try:
        assert (ks.chunk_steps(2 * dim, T), ks.chunk_fold(2 * dim, T)) == (steps, fold)
        check(ks, m, y)
    finally:
        ks.set_chunk_rules(2 * dim, [])
        tune.load_default()                       # the device's tuned table, if any


def test_single_sequence_T1024(ks):
    seq = workloads.config_single()
    e = check(ks, seq.model, seq.y)
    print("T=1024 errors", e)


def test_long_sequence_T2pow20(ks):
    seq = workloads.config_long()
    e = check(ks, seq.model, seq.y, refined=False)
    print("T=2^20 errors", e)


def test_paper_experiment_model(ks):
    """Section V's printed parameters: sigma = 0.5 (R = 0.25 I), m0 = (0, 0, 1, -1)."""
    rng = np.random.default_rng(77)
    m = workloads.wiener_velocity(2, dt=0.1, q=1.0, r=0.25, m0=np.array([0.0, 0.0, 1.0, -1.0]))
    _, y = workloads.simulate(m, 3000, rng)
    check(ks, m, y)



@pytest.mark.parametrize("p0", [1e-4, 1e6])
def test_extreme_prior_first_element(ks, p0):
    """The k = 1 element (prediction and update of N(m0, P0)) is built in
    FP64: with a near-exact or a diffuse prior (P- ~ 1e6 against R = 0.5) its
    update P- - K S K^T keeps FP32 accuracy.  T = 1, so the output is that
    element alone."""
    rng = np.random.default_rng(79)
    m = workloads.wiener_velocity(2, dt=0.1, q=1.0, r=0.5, m0=np.array([30.0, -20.0, 1.0, 2.0]),
                                  P0=p0 * np.eye(4))
    _, y = workloads.simulate(m, 1, rng)
    check(ks, m, y)


@pytest.mark.parametrize("p0", [1e-4, 25.0])
def test_prior_scales(ks, p0):
    """A near-exact and a broad prior over a long sequence (m0 far from the
    data).  A very diffuse one (P0 ~ 1e6 I) is outside the FP32 scan's
    reach: Lemma 4's I + C_i J_j then has entries ~1e8."""
    rng = np.random.default_rng(80)
    m = workloads.wiener_velocity(2, dt=0.1, q=1.0, r=0.5, m0=np.array([30.0, -20.0, 1.0, 2.0]),
                                  P0=p0 * np.eye(4))
    _, y = workloads.simulate(m, 2000, rng)
    check(ks, m, y)


def test_random_model_with_offsets(ks):
    """A dense random stable model with non-zero u and d."""
    rng = np.random.default_rng(78)
    m0 = workloads.random_stable(4, 2, rng)
    m = workloads.make_model(m0.F, m0.Q, m0.H, m0.R, rng.standard_normal(4), 2.0 * np.eye(4),
                             u=0.3 * rng.standard_normal(4), d=0.5 * rng.standard_normal(2))
    _, y = workloads.simulate(m, 9000, rng)
    check(ks, m, y)


def test_materialised_elements_match_lemma3(ks):
    seq = workloads.tracking_sequence(300, seed=5)
    m = seq.model
    model = gpu_model(ks, m)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, 300, ks.KS_WS_ELEMENTS)
    ks.build_elements(model, y, ws)
    assert ks.status(ws) == ks.KS_OK
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in ks.elements(model, 300, ws).items()}
    ref = L.filter_elements(m, seq.y)
    for name in ("A", "b", "C", "eta", "J"):
        r = np.array([getattr(e, name) for e in ref])
        scale = max(np.abs(r).max(), 1e-30)
        assert np.abs(got[name] - r).max() / scale < 1e-5, name


@pytest.mark.parametrize("T", [1, 2, 2049, 70000])
def test_filter_scan_over_materialised_elements(ks, T):
    seq = workloads.tracking_sequence(T, seed=2000 + T)
    m = seq.model
    model = gpu_model(ks, m)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, T, ks.KS_WS_ELEMENTS)
    ks.build_elements(model, y, ws)
    fm, fP = ks.filter_scan(model, T, ws)
    assert ks.status(ws) == ks.KS_OK
    rfm, rfP = oracle.kf(m, seq.y)
    parity.check_mean(fm.cpu().numpy(), rfm, rfP, parity.TOL)
    parity.check_cov(fP.cpu().numpy(), rfP, parity.TOL)


@pytest.mark.parametrize("T", [1, 3, 2048, 50001])
def test_smooth_scan_from_given_filtered_moments(ks, T):
    """ks_smooth_scan on FP32 filtered moments vs the oracle's RTS pass on the
    very same (FP32-rounded) moments."""
    seq = workloads.tracking_sequence(T, seed=3000 + T)
    m = seq.model
    rfm, rfP = oracle.kf(m, seq.y)
    fm32 = rfm.astype(np.float32)
    fP32 = rfP.astype(np.float32)
    rsm, rsP = oracle.rts(m, fm32.astype(np.float64), fP32.astype(np.float64))
    model = gpu_model(ks, m)
    sm, sP = ks.smooth_scan(model, torch.as_tensor(fm32, device="cuda"), torch.as_tensor(fP32, device="cuda"))
    torch.cuda.synchronize()
    parity.check_mean(sm.cpu().numpy(), rsm, rsP, parity.TOL)
    parity.check_cov(sP.cpu().numpy(), rsP, parity.TOL)


def _pack_f(e):
    return np.concatenate([e.A.ravel(), e.b, e.C.ravel(), e.eta, e.J.ravel()])


def _pack_s(e):
    return np.concatenate([e.E.ravel(), e.g, e.L.ravel()])


def test_filter_operator_batch_matches_lemma4(ks):
    rng = np.random.default_rng(11)
    n, cnt = 4, 500
    lefts, rights, refs = [], [], []
    for i in range(cnt):
        a = L.FElem(rng.standard_normal((n, n)) / 2, rng.standard_normal(n), pins.rand_spd(n, rng, 0.5),
                    rng.standard_normal(n), pins.rand_psd(n, rng, scale=0.7))
        b = L.FElem(rng.standard_normal((n, n)) / 2, rng.standard_normal(n), pins.rand_spd(n, rng, 0.5),
                    rng.standard_normal(n), pins.rand_psd(n, rng, rank=2, scale=0.7))
        a32 = L.FElem(*(x.astype(np.float32).astype(np.float64) for x in a))
        b32 = L.FElem(*(x.astype(np.float32).astype(np.float64) for x in b))
        lefts.append(_pack_f(a32)); rights.append(_pack_f(b32)); refs.append(_pack_f(L.filter_combine(a32, b32)))
    lt = torch.as_tensor(np.array(lefts), dtype=torch.float32, device="cuda")
    rt = torch.as_tensor(np.array(rights), dtype=torch.float32, device="cuda")
    out, ws = ks.filter_combine_batch(n, lt, rt)
    assert ks.status(ws) == ks.KS_OK
    got = out.cpu().numpy().astype(np.float64)
    ref = np.array(refs)
    rel = np.abs(got - ref).max(1) / np.abs(ref).max(1)
    assert rel.max() < 1e-4, rel.max()


def test_smoother_operator_batch_matches_lemma6(ks):
    rng = np.random.default_rng(12)
    n, cnt = 4, 500
    lefts, rights, refs = [], [], []
    for i in range(cnt):
        a = L.SElem(rng.standard_normal((n, n)) / 2, rng.standard_normal(n), pins.rand_spd(n, rng))
        b = L.SElem(rng.standard_normal((n, n)) / 2, rng.standard_normal(n), pins.rand_spd(n, rng))
        a32 = L.SElem(*(x.astype(np.float32).astype(np.float64) for x in a))
        b32 = L.SElem(*(x.astype(np.float32).astype(np.float64) for x in b))
        lefts.append(_pack_s(a32)); rights.append(_pack_s(b32)); refs.append(_pack_s(L.smoother_combine(a32, b32)))
    lt = torch.as_tensor(np.array(lefts), dtype=torch.float32, device="cuda")
    rt = torch.as_tensor(np.array(rights), dtype=torch.float32, device="cuda")
    out, _ = ks.smoother_combine_batch(n, lt, rt)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = np.array(refs)
    rel = np.abs(got - ref).max(1) / np.abs(ref).max(1)
    assert rel.max() < 1e-5, rel.max()


def test_non_finite_measurement_is_reported(ks):
    seq = workloads.tracking_sequence(5000, seed=4)
    y = seq.y.copy()
    y[1234, 0] = np.nan
    model = gpu_model(ks, seq.model)
    yt = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, 5000)
    ks.smooth(model, yt, ws)
    assert ks.status(ws) == ks.KS_ENUMERIC
    assert ks.status(ws) == ks.KS_OK          # the status word was cleared


@pytest.mark.parametrize("nx,ny", [(2, 1), (4, 2), (6, 3), (8, 4)])
def test_non_positive_first_innovation_covariance_is_reported(ks, nx, ny):
    """The FP64 k = 1 element checks that S1 = H P- H^T + R is positive
    definite (leading minors for ny <= 3, pivots of the unpivoted elimination
    above): a prior covariance P0 = -10 I, which no valid model has, makes S1
    negative definite while S = H Q H^T + R of the later steps stays valid."""
    rng = np.random.default_rng(nx)
    if nx <= 6:
        m = workloads.wiener_velocity(nx // 2, dt=0.1, q=1.0, r=0.5)
    else:
        m = workloads.random_stable(nx, ny, rng)
    m.P0 = -10.0 * np.eye(nx)
    y = rng.standard_normal((300, ny))
    model = gpu_model(ks, m)
    yt = torch.as_tensor(np.asarray(y), dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, 300)
    ks.smooth(model, yt, ws)
    assert ks.status(ws) == ks.KS_ENUMERIC


def test_bad_arguments_raise(ks):
    seq = workloads.tracking_sequence(100, seed=4)
    model = gpu_model(ks, seq.model)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    small = torch.zeros(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ks.KsError) as ei:
        ks.smooth(model, y, small)
    assert ei.value.code == ks.KS_EINVAL
    mis = torch.empty(2 * 100 + 1, dtype=torch.float32, device="cuda")[1:].view(100, 2)
    with pytest.raises(ks.KsError) as ei:
        ks.smooth(model, mis)
    assert ei.value.code == ks.KS_EINVAL


def test_repeated_calls_agree(ks):
    """Two calls on the same workspace agree (the look-back may combine tiles
    in a different grouping from run to run, so agreement is to rounding)."""
    seq = workloads.tracking_sequence(100000, seed=6)
    model = gpu_model(ks, seq.model)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, 100000)
    a = [t.clone() for t in ks.smooth(model, y, ws)]
    b = ks.smooth(model, y, ws)
    assert ks.status(ws) == ks.KS_OK
    ref = oracle.kf_rts(seq.model, seq.y)
    parity.check_all(a, ref)
    parity.check_all(b, ref)


@pytest.mark.parametrize("dim,T", [(1, 3000), (1, 1), (3, 2500), (3, 4097)])
def test_other_state_sizes_wiener(ks, dim, T):
    """nx = 2 (ny = 1) and nx = 6 (ny = 3) Wiener-velocity models."""
    rng = np.random.default_rng(300 + dim + T)
    m = workloads.wiener_velocity(dim, dt=0.1, q=float(rng.uniform(0.5, 2)), r=float(rng.uniform(0.1, 1)))
    _, y = workloads.simulate(m, T, rng)
    check(ks, m, y)


@pytest.mark.parametrize("T", [1, 700, 5000])
def test_random_stable_nx8(ks, T):
    if not ks.supported(8, 4):
        pytest.skip("nx = 8 is not compiled into this library")
    rng = np.random.default_rng(400 + T)
    m = workloads.random_stable(8, 4, rng)
    _, y = workloads.simulate(m, T, rng)
    check(ks, m, y)


@pytest.mark.parametrize("T", [1, 2, 31, 32, 33, 95, 96, 97, 289, 1000, 5000])
def test_random_stable_nx32_sizes(ks, T):
    """nx = 32 (tensor-core operators, one warp per chain): edge sizes around a
    chain (32 steps) and a tile (3 chains), and several tiles with a ragged tail."""
    rng = np.random.default_rng(500 + T)
    m = workloads.random_stable(32, 8, rng)
    _, y = workloads.simulate(m, T, rng)
    e = check(ks, m, y, tol=parity.TOL_NX32)
    print(f"nx=32 T={T} errors", e)


def test_nx32_accurate_measurements(ks):
    """Accurate measurements against a large process noise (q = 1, R = 1e-3 I).
    The tile combines' I + C_i J_j stay near cond_1 = 21 here (the oracle's
    FP64 lemmas give the same), below the refinement threshold."""
    rng = np.random.default_rng(515)
    m = workloads.random_stable(32, 8, rng, q=1.0, r=1e-3)
    _, y = workloads.simulate(m, 3000, rng)
    e = check(ks, m, y, tol=parity.TOL_NX32)
    print("nx=32 accurate-measurement errors", e)


def test_nx32_ill_conditioned_combine_is_refined(ks):
    """Half of the 32 state components in units 100 times smaller: the tile
    combines' I + C_i J_j reach cond_1 ~ 5e3 (FP64 lemmas), above the 1e3
    threshold, so the FP64-residual refinement runs, and the result still
    matches the oracle."""
    rng = np.random.default_rng(515)
    d = np.ones(32)
    d[:16] = 100.0
    m = scaled_model(workloads.random_stable(32, 8, rng), d)
    _, y = workloads.simulate(m, 3000, rng)
    e = check(ks, m, y, tol=parity.TOL_NX32, refined=True)
    print("nx=32 ill-conditioned errors", e)


# Positions in units 300 (100) times smaller than velocities: the
# cross-block combines' I + C_i J_j reach cond_1 ~ 4e3 at 4 steps per thread
# (T < 96 Ki) and ~3e3 at 32 steps per thread (scale 100, T >= 640 Ki), and
# ~9e3 at nx = 8 (FP64 lemmas): the register and lane-group paths refine them.
@pytest.mark.parametrize("nx,scale,T", [(4, 300.0, 20000), (4, 100.0, 700001), (8, 300.0, 6000)])
def test_ill_conditioned_combines_are_refined(ks, nx, scale, T):
    rng = np.random.default_rng(520 + nx)
    if nx == 4:
        base = workloads.wiener_velocity(2, dt=0.1, q=1.0, r=1.0)
        d = [scale, scale, 1.0, 1.0]
    else:
        base = workloads.random_stable(8, 4, rng)
        d = [scale] * 4 + [1.0] * 4
    m = scaled_model(base, d)
    _, y = workloads.simulate(m, T, rng)
    e = check(ks, m, y, refined=True)
    print(f"nx={nx} scale={scale} T={T} errors", e)


@pytest.mark.parametrize("T", [1, 97, 3000])
def test_smooth_scan_nx32_from_given_moments(ks, T):
    rng = np.random.default_rng(650 + T)
    m = workloads.random_stable(32, 8, rng)
    _, y = workloads.simulate(m, T, rng)
    rfm, rfP = oracle.kf(m, y)
    fm32, fP32 = rfm.astype(np.float32), rfP.astype(np.float32)
    rsm, rsP = oracle.rts(m, fm32.astype(np.float64), fP32.astype(np.float64))
    model = gpu_model(ks, m)
    sm, sP = ks.smooth_scan(model, torch.as_tensor(fm32, device="cuda"), torch.as_tensor(fP32, device="cuda"))
    torch.cuda.synchronize()
    parity.check_mean(sm.cpu().numpy(), rsm, rsP, parity.TOL_NX32)
    parity.check_cov(sP.cpu().numpy(), rsP, parity.TOL_NX32)


def test_precision_workload_nx32(ks):
    """The nx = 32, ny = 8, T = 65536 random stable workload against the FP64
    oracle; its combines stay well conditioned, so nothing is refined."""
    seq = workloads.config_precision()
    e = check(ks, seq.model, seq.y, tol=parity.TOL_NX32, refined=False)
    print("nx=32 T=65536 errors", e)


@pytest.mark.parametrize("T", [1, 2048, 9000])
def test_smooth_scan_nx8_from_given_moments(ks, T):
    rng = np.random.default_rng(600 + T)
    m = workloads.random_stable(8, 4, rng)
    _, y = workloads.simulate(m, T, rng)
    rfm, rfP = oracle.kf(m, y)
    fm32, fP32 = rfm.astype(np.float32), rfP.astype(np.float32)
    rsm, rsP = oracle.rts(m, fm32.astype(np.float64), fP32.astype(np.float64))
    model = gpu_model(ks, m)
    sm, sP = ks.smooth_scan(model, torch.as_tensor(fm32, device="cuda"), torch.as_tensor(fP32, device="cuda"))
    torch.cuda.synchronize()
    parity.check_mean(sm.cpu().numpy(), rsm, rsP, parity.TOL)
    parity.check_cov(sP.cpu().numpy(), rsP, parity.TOL)


def test_lookback_wait_runs_out_and_is_reported(ks):
    """A look-back wait on a flag that nothing sets: the forward scan numbers
    its tiles from 1 (ks_workspace_set_waits), so tile 0 is never published
    and tile 1's wait must give up after its 2000 polls.  The call returns in
    bounded time, ks_status reports KS_ETIMEOUT, and a freshly initialised
    workspace then gives the oracle's result."""
    import time
    seq = workloads.tracking_sequence(20000, seed=91)     # 4 steps per thread: 40 tiles of 512 steps
    model = gpu_model(ks, seq.model)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device="cuda")
    ws = ks.alloc_workspace(model, seq.T)
    ks.set_waits(ws, wait_polls=2000, first_tile=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ks.smooth(model, y, ws)
    rc = ks.status(ws)
    dt = time.perf_counter() - t0
    assert rc == ks.KS_ETIMEOUT, rc
    assert dt < 2.0, dt
    assert ks.lib().ks_workspace_init(ks._p(ws), ws.numel(), ks._stream(None)) == ks.KS_OK
    out = ks.smooth(model, y, ws)
    assert ks.status(ws) == ks.KS_OK
    parity.check_all(out, oracle.kf_rts(seq.model, seq.y))


def test_wait_settings_are_checked(ks):
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ks.KsError) as ei:
        ks.set_waits(ws, wait_polls=10, first_tile=2)
    assert ei.value.code == ks.KS_EINVAL
