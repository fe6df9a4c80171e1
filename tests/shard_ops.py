"""A CPU stand-in for the device steps of the time-sharded smoother (test
infrastructure): the oracle's Lemma 3-6 folds (numpy FP64) and its
sequential filter/smoother, in the packed element layout of the operator
batches, over torch CPU float64 tensors (so gloo can all-gather them)."""
import dataclasses

import numpy as np
import torch

import oracle
from oracle import lemmas as L


def pack_f(e):
    return torch.from_numpy(np.concatenate([e.A.ravel(), e.b, e.C.ravel(), e.eta, e.J.ravel()]))


def unpack_f(x, n):
    x = x.numpy()
    o = [0]

    def take(k):
        v = x[o[0]:o[0] + k]
        o[0] += k
        return v
    return L.FElem(take(n * n).reshape(n, n), take(n), take(n * n).reshape(n, n), take(n), take(n * n).reshape(n, n))


def pack_s(e):
    return torch.from_numpy(np.concatenate([e.E.ravel(), e.g, e.L.ravel()]))


def unpack_s(x, n):
    x = x.numpy()
    return L.SElem(x[:n * n].reshape(n, n), x[n * n:n * n + n], x[n * n + n:].reshape(n, n))


def _params(m):
    return [np.asarray(getattr(m, k), dtype=np.float64) for k in ("F", "u", "Q", "H", "d", "R")]


class NumpyOps:
    def filter_aggregate(self, model, y, first):
        F, u, Q, H, d, R = _params(model)
        y = np.asarray(y, dtype=np.float64)
        acc = (L.filter_element_first(F, u, Q, H, d, R, y[0], model.m0, model.P0) if first
               else L.filter_element(F, u, Q, H, d, R, y[0]))
        for k in range(1, y.shape[0]):
            acc = L.filter_combine(acc, L.filter_element(F, u, Q, H, d, R, y[k]))
        return pack_f(acc)

    def filter_combine(self, left, right, n):
        return pack_f(L.filter_combine(unpack_f(left, n), unpack_f(right, n)))

    def forward(self, model, y, prior):
        if prior is not None:
            b, C = (np.asarray(t, dtype=np.float64) for t in prior)
            model = dataclasses.replace(model, m0=b.copy(), P0=0.5 * (C + C.T))
        fm, fc = oracle.kf(model, np.asarray(y, dtype=np.float64))
        return torch.from_numpy(fm), torch.from_numpy(fc)

    def smoother_aggregate(self, model, fm, fc, last):
        F, u, Q = (np.asarray(getattr(model, k), dtype=np.float64) for k in ("F", "u", "Q"))
        fm, fc = fm.numpy(), fc.numpy()
        T = fm.shape[0]

        def el(k):
            if last and k == T - 1:
                return L.smoother_element_last(fm[k], fc[k])
            return L.smoother_element(F, u, Q, fm[k], fc[k])
        acc = el(0)
        for k in range(1, T):
            acc = L.smoother_combine(acc, el(k))
        return pack_s(acc)

    def smoother_combine(self, left, right, n):
        return pack_s(L.smoother_combine(unpack_s(left, n), unpack_s(right, n)))

    def reverse(self, model, fm, fc, boundary):
        fm, fc = fm.numpy(), fc.numpy()
        if boundary is not None:
            g, Lb = (np.asarray(t, dtype=np.float64) for t in boundary)
            fm = np.concatenate([fm, g[None]])
            fc = np.concatenate([fc, 0.5 * (Lb + Lb.T)[None]])
        sm, sc = oracle.rts(model, fm, fc)
        if boundary is not None:
            sm, sc = sm[:-1], sc[:-1]
        return torch.from_numpy(np.ascontiguousarray(sm)), torch.from_numpy(np.ascontiguousarray(sc))
