"""The time-sharding protocol (paper_1905_13002_gb300.shard) on the CPU: the
oracle's lemma folds stand in for the device steps; ranks exchange their
aggregates in one process (every shard count) and over gloo in 2 and 3
processes.  The concatenated shards must equal the oracle on the whole
sequence (the protocol is exact in FP64)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads
from shard_ops import NumpyOps
from paper_1905_13002_gb300 import shard


def model_and_data(seed, T, dim=2):
    rng = np.random.default_rng(seed)
    m = workloads.wiener_velocity(dim, dt=0.1, q=float(rng.uniform(0.5, 2)), r=float(rng.uniform(0.1, 1)))
    m = workloads.make_model(m.F, m.Q, m.H, m.R, rng.standard_normal(2 * dim), np.eye(2 * dim) * 2.0,
                             u=0.01 * rng.standard_normal(2 * dim), d=0.1 * rng.standard_normal(dim))
    _, y = workloads.simulate(m, T, rng)
    return m, y


def run_local(m, y, world):
    """All ranks in one process: each phase for every rank, then the exchange."""
    n = m.F.shape[0]
    parts = [shard.ShardSmoother(NumpyOps(), m, y[s:e], r, world, n)
             for r, (s, e) in enumerate(shard.shard_bounds(y.shape[0], world))]
    aggs = [p.filter_aggregate() for p in parts]
    for p in parts:
        p.forward(aggs)
    saggs = [p.smoother_aggregate() for p in parts]
    outs = [p.reverse(saggs) for p in parts]
    return [np.concatenate([o[i].numpy() for o in outs]) for i in range(4)]


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_local_shards_equal_the_whole_sequence(world):
    m, y = model_and_data(11 + world, 61)
    got = run_local(m, y, world)
    ref = oracle.kf_rts(m, y)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=1e-9, atol=1e-9)


def test_shard_bounds_cover_the_sequence():
    for T, w in [(10, 3), (7, 7), (1000, 8)]:
        b = shard.shard_bounds(T, w)
        assert b[0][0] == 0 and b[-1][1] == T
        assert all(a[1] == c[0] for a, c in zip(b, b[1:]))
        assert max(e - s for s, e in b) - min(e - s for s, e in b) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(2, 3)


def test_wrong_aggregate_count_is_rejected():
    m, y = model_and_data(5, 20)
    p = shard.ShardSmoother(NumpyOps(), m, y, 0, 2, 4)
    with pytest.raises(ValueError):
        p.forward([p.filter_aggregate()])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, T, seed, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, y = model_and_data(seed, T)
        s, e = shard.shard_bounds(T, world)[rank]
        out = shard.smooth_sharded(NumpyOps(), m, y[s:e], rank, world, m.F.shape[0], shard.dist_all_gather)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), *[o.numpy() for o in out])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_whole_sequence(world, tmp_path):
    import torch.multiprocessing as mp
    T, seed = 47, 77 + world
    mp.start_processes(_worker, args=(world, _free_port(), T, seed, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    parts = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    got = [np.concatenate([p[f"arr_{i}"] for p in parts]) for i in range(4)]
    m, y = model_and_data(seed, T)
    ref = oracle.kf_rts(m, y)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=1e-9, atol=1e-9)
