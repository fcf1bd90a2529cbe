"""K-partitioned MPPI iteration: the host side of the two exchanges (no arithmetic of the method).

Eq. (11) sums over the samples, so one iteration splits into K-slices (one per context, normally
one per GPU) with two exchanges: the minimum cost over the slices (with its global index and the
number of finite costs), then the sum over the slices of each slice's softmin normaliser eta and
its weighted noise sums du[T][2].  Every slice then runs the same update from the totals
(mppi_slice_finalize), so every slice holds the same warm start afterwards.

``combine_minima`` / ``combine_sums`` do the exchanges in one process (slices in a list, summed
in slice order); ``allreduce_minima`` / ``allreduce_sums`` do them across the ranks of a
``torch.distributed`` process group (one slice per rank).  ``plan_partitioned`` drives one
iteration over several contexts in one process.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np


def combine_minima(records: Sequence[Tuple[float, int, int]]) -> Tuple[float, int, int]:
    """(s_min, global argmin, n_finite) per slice -> the global record (ties: lowest index)."""
    best, arg, n = math.inf, -1, 0
    for s, a, nf in records:
        n += int(nf)
        if nf > 0 and (s < best or (s == best and (arg < 0 or a < arg))):
            best, arg = float(s), int(a)
    return best, arg, n


def combine_sums(parts: Sequence[Tuple[float, np.ndarray]]) -> Tuple[float, np.ndarray]:
    """(eta, du[T][2]) per slice -> totals, added in slice order in binary64."""
    eta = 0.0
    du = np.zeros_like(np.asarray(parts[0][1], dtype=np.float64))
    for e, d in parts:
        eta += float(e)
        du += np.asarray(d, dtype=np.float64)
    return eta, du


def allreduce_minima(s_min: float, argmin: int, n_finite: int, group=None) -> Tuple[float, int, int]:
    """The global (s_min, argmin, n_finite) over the ranks of a process group."""
    import torch
    import torch.distributed as dist
    s = torch.tensor([s_min if n_finite > 0 else math.inf], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.MIN, group=group)
    big = 2 ** 62
    idx = torch.tensor([argmin if (n_finite > 0 and s_min == s.item()) else big], dtype=torch.int64)
    dist.all_reduce(idx, op=dist.ReduceOp.MIN, group=group)
    n = torch.tensor([int(n_finite)], dtype=torch.int64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM, group=group)
    a = int(idx.item())
    return float(s.item()), (a if a != big else -1), int(n.item())


def allreduce_sums(eta: float, du, group=None) -> Tuple[float, np.ndarray]:
    """The totals of (eta, du[T][2]) over the ranks of a process group, in binary64."""
    import torch
    import torch.distributed as dist
    d = np.asarray(du, dtype=np.float64)
    t = torch.tensor(np.concatenate([[eta], d.ravel()]), dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.numpy()
    return float(v[0]), v[1:].reshape(d.shape).copy()


def slice_offsets(sizes: Sequence[int]) -> List[int]:
    """Global index of the first sample of each slice."""
    out, k = [], 0
    for s in sizes:
        out.append(k)
        k += int(s)
    return out


def plan_partitioned(planners, offsets, x0, ref, circles=None, centres=None):
    """One iteration over several slice contexts in this process: costs, the minimum exchange,
    sums, the sum exchange, then the same update on every slice.  Returns the outputs of every
    slice [(u*, x*, info)], the global minimum record and the per-slice costs records."""
    mins = [pl.slice_costs(k0, x0, ref, circles, centres) for pl, k0 in zip(planners, offsets)]
    s_min, arg, n_fin = combine_minima(mins)
    parts = [pl.slice_sums(s_min) for pl in planners]
    eta, du = combine_sums(parts)
    outs = [pl.slice_finalize(eta, du, n_fin, s_min, arg) for pl in planners]
    return outs, (s_min, arg, n_fin), mins
