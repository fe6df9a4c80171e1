"""GPU parity of the segmented (batched) scans: many sequences of uneven
length laid end to end, each checked against the FP64 oracle on its own."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    from paper_1905_13002_gb300 import _build
    _build.build()
    import paper_1905_13002_gb300 as ks
    return ks


def make_batch(dim, lengths, seed):
    rng = np.random.default_rng(seed)
    seqs = []
    for T in lengths:
        m = workloads.wiener_velocity(dim, dt=0.1, q=float(rng.uniform(0.5, 2)), r=float(rng.uniform(0.1, 1)))
        _, y = workloads.simulate(m, int(T), rng)
        seqs.append(workloads.Sequence(m, y))
    return seqs


def run_and_check(ks, seqs):
    batch = ks.ModelBatch.create([s.model for s in seqs], [s.T for s in seqs])
    y = torch.as_tensor(np.concatenate([s.y for s in seqs]), dtype=torch.float32, device="cuda")
    ws = torch.empty(ks.workspace_bytes_batch(batch.nx, batch.ny, batch.B, y.shape[0]), dtype=torch.uint8,
                     device="cuda")
    assert ks.lib().ks_workspace_init(ks._p(ws), ws.numel(), ks._stream(None)) == 0
    out = [t.cpu().numpy() for t in ks.smooth_batch(batch, y, ws)]
    assert ks.status(ws) == ks.KS_OK
    worst = 0.0
    o = 0
    for s in seqs:
        ref = oracle.kf_rts(s.model, s.y)
        e = parity.check_all([x[o:o + s.T] for x in out], ref)
        e = {k: e[k] for k in ("fmean", "fcov", "smean", "scov")}
        worst = max(worst, max(e.values()))
        o += s.T
    assert worst < parity.TOL, worst
    return worst


# Lengths put boundaries inside thread blocks (32 steps) and tiles (4096),
# include one-step sequences, and sequences shorter than a block.
EDGE = [1, 2, 31, 32, 33, 1, 127, 128, 129, 5000, 1, 4096, 4097, 3, 8191, 64]


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_edge_lengths(ks, dim):
    run_and_check(ks, make_batch(dim, EDGE, 10 + dim))


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_log_uniform_lengths(ks, dim):
    rng = np.random.default_rng(20 + dim)
    lengths = workloads.batch_lengths(120, rng, 256, 16384)
    run_and_check(ks, make_batch(dim, lengths, 30 + dim))



# Batches are dispatched by their total length like single sequences (4, 8,
# 16 or 32 steps per thread below 96 Ki, 192 Ki, 640 Ki steps, and above):
# one batch per band, the edge lengths mixed in.
@pytest.mark.parametrize("dim,B,band", [(2, 30, (98304, 196608)), (2, 90, (196608, 655360)),
                                        (2, 200, (655360, 1 << 30)), (3, 90, (196608, 655360)),
                                        (1, 200, (655360, 1 << 30))])
def test_chunk_variant_batches(ks, dim, B, band):
    rng = np.random.default_rng(50 + B + dim)
    lengths = np.concatenate([EDGE, workloads.batch_lengths(B, rng, 256, 16384)])
    rng.shuffle(lengths)
    assert band[0] <= lengths.sum() < band[1], lengths.sum()
    run_and_check(ks, make_batch(dim, lengths, 60 + B + dim))

def test_single_sequence_batch_equals_plain_call(ks):
    seqs = make_batch(2, [20000], 7)
    run_and_check(ks, seqs)


def test_batched_config_sample(ks):
    """The batched workload's own generator (mixed nx), one call per nx group."""
    seqs = workloads.config_batched(B=96)
    for nx in (2, 4, 6):
        group = [s for s in seqs if s.model.nx == nx]
        if group:
            run_and_check(ks, group)


def test_bad_offsets_reported(ks):
    seqs = make_batch(2, [100, 200], 9)
    batch = ks.ModelBatch.create([s.model for s in seqs], [s.T for s in seqs])
    y = torch.as_tensor(np.concatenate([s.y for s in seqs]), dtype=torch.float32, device="cuda")
    ws = torch.zeros(ks.workspace_bytes_batch(4, 2, 2, 300), dtype=torch.uint8, device="cuda")
    # The second sequence is made empty (offsets 0, 300, 300): every offset
    # stays within [0, T], so all accesses are in bounds, and the device check
    # flags the table as inconsistent.
    batch.offsets[1] = 300
    ks.smooth_batch(batch, y, ws)
    assert ks.status(ws) == ks.KS_EINVAL


def test_random_stable_nx8_batch(ks):
    rng = np.random.default_rng(77)
    seqs = []
    for T in [1, 5, 31, 32, 33, 127, 128, 129, 3000, 1, 700]:
        m = workloads.random_stable(8, 4, rng)
        _, y = workloads.simulate(m, T, rng)
        seqs.append(workloads.Sequence(m, y))
    run_and_check(ks, seqs)


def test_random_stable_nx32_batch(ks):
    """nx = 32 batches run on the CUDA-core group kernels."""
    rng = np.random.default_rng(78)
    seqs = []
    for T in [1, 5, 63, 64, 65, 200, 1]:
        m = workloads.random_stable(32, 8, rng)
        _, y = workloads.simulate(m, T, rng)
        seqs.append(workloads.Sequence(m, y))
    run_and_check(ks, seqs)


def run_mixed_and_check(ks, seqs):
    """All sequences through ks_smooth_batched (one group per state size, one
    launch per scan); every sequence against its own oracle run."""
    groups, members = [], []
    for nx in (6, 4, 2):
        grp = [s for s in seqs if s.model.nx == nx]
        if not grp:
            continue
        batch = ks.ModelBatch.create([s.model for s in grp], [s.T for s in grp])
        y = torch.as_tensor(np.concatenate([s.y for s in grp]), dtype=torch.float32, device="cuda")
        groups.append((batch, y))
        members.append(grp)
    sizes = [(b.nx, b.ny, b.B, int(y.shape[0])) for b, y in groups]
    ws = torch.empty(ks.workspace_bytes_batched(sizes), dtype=torch.uint8, device="cuda")
    assert ks.lib().ks_workspace_init(ks._p(ws), ws.numel(), ks._stream(None)) == 0
    outs = ks.smooth_batched(groups, ws)
    assert ks.status(ws) == ks.KS_OK
    worst = {}
    for grp, out in zip(members, outs):
        out = [t.cpu().numpy() for t in out]
        w, o = 0.0, 0
        for s in grp:
            e = parity.check_all([x[o:o + s.T] for x in out], oracle.kf_rts(s.model, s.y))
            w = max(w, e["fmean"], e["fcov"], e["smean"], e["scov"])
            o += s.T
        worst[grp[0].model.nx] = w
    return worst


def test_batched_workload_full_size(ks):
    """The whole batched workload in one ks_smooth_batched call (one launch
    per scan over all three state sizes): 4096 sequences, log-uniform lengths
    in [256, 16384] (15.9 M steps), nx in {2, 4, 6}, every sequence checked
    against its own FP64 oracle run."""
    seqs = workloads.config_batched()
    assert len(seqs) == 4096
    worst = run_mixed_and_check(ks, seqs)
    print("batched workload (one launch per scan), worst relative error per nx", worst)


# Mixed-size batches: the three sizes with the edge lengths, two sizes only,
# one size only, and totals in each steps-per-thread band.
@pytest.mark.parametrize("dims,extra", [((1, 2, 3), 0), ((1, 3), 0), ((2,), 0), ((1, 2, 3), 60),
                                        ((2, 3), 250), ((1, 2, 3), 400)])
def test_mixed_state_sizes(ks, dims, extra):
    rng = np.random.default_rng(70 + extra + len(dims))
    seqs = []
    for dim in dims:
        lengths = np.concatenate([EDGE, workloads.batch_lengths(extra, rng, 256, 16384)]) if extra else EDGE
        seqs += make_batch(dim, lengths, 80 + dim + extra)
    rng.shuffle(seqs)
    worst = run_mixed_and_check(ks, seqs)
    print("mixed", dims, sum(s.T for s in seqs), worst)


@pytest.mark.parametrize("steps", [8, 32])
def test_mixed_batch_with_block_fold(ks, steps):
    """The mixed-size launch with the linear block fold forced on (per-sequence
    coefficients, segment-relative tables): every sequence against its oracle."""
    from paper_1905_13002_gb300 import tune
    rng = np.random.default_rng(90 + steps)
    seqs = []
    for dim in (1, 2, 3):
        lengths = np.concatenate([EDGE, workloads.batch_lengths(30, rng, 256, 16384)])
        seqs += make_batch(dim, lengths, 95 + dim + steps)
    rng.shuffle(seqs)
    ks.set_chunk_rules(0, [(tune.T_NEVER, steps, 1)])
    try:
        assert ks.chunk_fold(0, 1 << 20) == 1
        run_mixed_and_check(ks, seqs)
    finally:
        ks.set_chunk_rules(0, [])
        tune.load_default()


def test_mixed_batch_rejects_unsupported_groups(ks):
    seqs = make_batch(2, [100, 50], 5)
    batch = ks.ModelBatch.create([s.model for s in seqs], [s.T for s in seqs])
    y = torch.as_tensor(np.concatenate([s.y for s in seqs]), dtype=torch.float32, device="cuda")
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(ks.KsError) as ei:            # two groups of one size
        ks.smooth_batched([(batch, y), (batch, y)], ws)
    assert ei.value.code == ks.KS_EINVAL
    rng = np.random.default_rng(6)
    m8 = workloads.random_stable(8, 4, rng)
    b8 = ks.ModelBatch.create([m8], [10])
    y8 = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ks.KsError) as ei:            # nx = 8 runs on the lane-group kernels
        ks.smooth_batched([(b8, y8)], ws)
    assert ei.value.code == ks.KS_EUNSUPPORTED
