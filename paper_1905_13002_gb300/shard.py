"""One sequence smoothed across devices, split along time (the paper's
block-level elements, Section III-C, with one block per device).

Rank r of R owns the consecutive steps of shard r.  Each scan needs one
exchange of one element per shard:

1. every rank folds its shard's filtering elements into one aggregate
   (Lemma 4; rank 0's first element is Lemma 3's k = 1 element) and the
   aggregates are all-gathered;
2. rank r combines aggregates 0..r-1 in order: the result has A = 0 (it
   starts with the k = 1 element) and its (b, C) is the filtered posterior at
   the step before the shard, so the shard's forward scan is the plain
   forward scan with that posterior as its prior (Lemma 3's k = 1 element is
   "posterior (x) measurement element");
3. every rank folds its shard's smoothing elements into one aggregate
   (Lemma 6; the last rank's last element is Lemma 5's k = n element) and the
   aggregates are all-gathered;
4. rank r combines aggregates r+1..R-1 in order: the result has E = 0 (it
   ends with the k = n element) and its (g, L) is the smoothed posterior at
   the step after the shard; appended to the shard's filtered moments as one
   extra step, Lemma 5's last-step element (E = 0, g, L) makes it the suffix
   entering the shard, so the shard's reverse scan is the plain reverse scan
   over one step more.

The device work goes through an ``ops`` object (``DeviceOps``: libks) and
the exchange through an ``all_gather(tensor) -> list`` callable
(``dist_all_gather``: torch.distributed, NCCL or gloo), so the protocol runs
unchanged with any of them.
"""
from __future__ import annotations

import dataclasses

import torch

from . import Model, filter_aggregate, filter_combine_batch, smooth, smooth_scan, smoother_aggregate, \
    smoother_combine_batch


def unpack_filter(x: torch.Tensor, n: int):
    """(b, C) of a packed filtering element A[n*n] b[n] C[n*n] eta[n] J[n*n]."""
    return x[n * n:n * n + n], x[n * n + n:2 * n * n + n].reshape(n, n)


def unpack_smoother(x: torch.Tensor, n: int):
    """(g, L) of a packed smoothing element E[n*n] g[n] L[n*n]."""
    return x[n * n:n * n + n], x[n * n + n:2 * n * n + n].reshape(n, n)


def _aligned(t: torch.Tensor) -> torch.Tensor:
    """A 16-byte aligned contiguous copy when the view is not (libks reads its
    inputs with vector loads)."""
    t = t.contiguous()
    return t if t.data_ptr() % 16 == 0 else t.clone()


class DeviceOps:
    """The four device steps of a shard on libks (nx <= 6)."""

    def filter_aggregate(self, model: Model, y: torch.Tensor, first: bool) -> torch.Tensor:
        return filter_aggregate(model, _aligned(y), first)[0]

    def filter_combine(self, left: torch.Tensor, right: torch.Tensor, n: int) -> torch.Tensor:
        return filter_combine_batch(n, left[None], right[None])[0][0]

    def forward(self, model: Model, y: torch.Tensor, prior):
        """Filtered moments of the shard from the posterior entering it
        (None: the model's own prior)."""
        if prior is not None:
            b, C = prior
            model = dataclasses.replace(model, m0=b.to(torch.float64).contiguous(),
                                        P0=(0.5 * (C + C.T)).to(torch.float64).contiguous())
        fm, fc, _, _ = smooth(model, _aligned(y), filter_only=True)
        return fm, fc

    def smoother_aggregate(self, model: Model, fm: torch.Tensor, fc: torch.Tensor, last: bool) -> torch.Tensor:
        return smoother_aggregate(model, fm, fc, last)[0]

    def smoother_combine(self, left: torch.Tensor, right: torch.Tensor, n: int) -> torch.Tensor:
        return smoother_combine_batch(n, left[None], right[None])[0][0]

    def reverse(self, model: Model, fm: torch.Tensor, fc: torch.Tensor, boundary):
        """Smoothed moments of the shard; ``boundary`` = (g, L) of the smoothed
        posterior at the step after the shard (None on the last shard)."""
        if boundary is None:
            return smooth_scan(model, fm, fc)
        g, L = boundary
        fm1 = torch.cat([fm, g[None].to(fm.dtype)]).contiguous()
        fc1 = torch.cat([fc, (0.5 * (L + L.T))[None].to(fc.dtype)]).contiguous()
        sm, sc = smooth_scan(model, fm1, fc1)
        return sm[:-1], sc[:-1]


class ShardSmoother:
    """The protocol for one rank; the steps run in order
    filter_aggregate -> forward(aggregates) -> smoother_aggregate -> reverse(aggregates)."""

    def __init__(self, ops, model, y, rank: int, world: int, nx: int):
        if not 0 <= rank < world:
            raise ValueError("rank out of range")
        self.ops, self.model, self.y = ops, model, y
        self.rank, self.world, self.n = rank, world, nx
        self.fm = self.fc = None

    def filter_aggregate(self):
        return self.ops.filter_aggregate(self.model, self.y, self.rank == 0)

    def forward(self, aggs: list):
        if len(aggs) != self.world:
            raise ValueError("one filtering aggregate per rank expected")
        prior = None
        if self.rank > 0:
            x = aggs[0]
            for i in range(1, self.rank):                # earlier shard on the left (Lemma 4)
                x = self.ops.filter_combine(x, aggs[i], self.n)
            prior = unpack_filter(x, self.n)
        self.fm, self.fc = self.ops.forward(self.model, self.y, prior)
        return self.fm, self.fc

    def smoother_aggregate(self):
        return self.ops.smoother_aggregate(self.model, self.fm, self.fc, self.rank == self.world - 1)

    def reverse(self, saggs: list):
        if len(saggs) != self.world:
            raise ValueError("one smoothing aggregate per rank expected")
        boundary = None
        if self.rank < self.world - 1:
            x = saggs[self.world - 1]
            for i in range(self.world - 2, self.rank, -1):   # earlier shard on the left (Lemma 6)
                x = self.ops.smoother_combine(saggs[i], x, self.n)
            boundary = unpack_smoother(x, self.n)
        sm, sc = self.ops.reverse(self.model, self.fm, self.fc, boundary)
        return self.fm, self.fc, sm, sc


def smooth_sharded(ops, model, y, rank: int, world: int, nx: int, all_gather):
    """Rank ``rank``'s part of the time-sharded smoother: returns its shard's
    (fmean, fcov, smean, scov)."""
    s = ShardSmoother(ops, model, y, rank, world, nx)
    s.forward(all_gather(s.filter_aggregate()))
    return s.reverse(all_gather(s.smoother_aggregate()))


def dist_all_gather(x: torch.Tensor) -> list:
    """all_gather over the default torch.distributed process group."""
    import torch.distributed as dist
    out = [torch.empty_like(x) for _ in range(dist.get_world_size())]
    dist.all_gather(out, x.contiguous())
    return out


def shard_bounds(T: int, world: int) -> list:
    """Steps [start, end) of each of `world` near-equal consecutive shards."""
    if world < 1 or T < world:
        raise ValueError("need at least one step per shard")
    base, extra = divmod(T, world)
    out, s = [], 0
    for r in range(world):
        e = s + base + (1 if r < extra else 0)
        out.append((s, e))
        s = e
    return out
