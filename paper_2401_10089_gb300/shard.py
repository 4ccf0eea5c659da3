"""Spreading a batch of independent matrices over ranks (one process per GPU).

Every matrix's logarithm is independent, so the data path has no collective:
each rank runs its own share, and the only communication is a max-reduce of
the step time (and, when a caller wants every result on one rank, a gather).

* ``cost_key``      -- n^3 (1 + log2(1 + ||A - I||_1 / Theta)), the same
                       work estimate the device queue orders by: the number
                       of square roots grows with log(||A - I|| / Theta).
* ``partition``     -- greedy longest-first assignment of matrices to ranks
                       (each matrix to the rank with the least assigned cost).
* ``max_over_ranks``, ``gather_to_root`` -- the two collectives.
"""
from __future__ import annotations

import math

import numpy as np

THETA_5 = 0.246  # Theta_{m_5} of Table Table_theta (the loop's threshold with k_max = 5)


def cost_key(n: int, norm_a_minus_i: float, theta: float = THETA_5) -> float:
    return float(n) ** 3 * (1.0 + math.log2(1.0 + norm_a_minus_i / theta))


def batch_costs(mats) -> np.ndarray:
    """Cost keys of a list (or array) of square numpy matrices."""
    out = np.empty(len(mats))
    for i, a in enumerate(mats):
        n = a.shape[0]
        b = a - np.eye(n)
        out[i] = cost_key(n, float(np.abs(b).sum(axis=0).max()))
    return out


def partition(costs, world: int) -> list[list[int]]:
    """Indices per rank, longest first, each matrix to the least-loaded rank
    (ties to the lowest rank); every index lands on exactly one rank."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the step time the whole job took)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_root(obj, root: int = 0):
    """The list of every rank's ``obj`` on ``root`` (None elsewhere)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == root else None
    dist.gather_object(obj, out, dst=root)
    return out
