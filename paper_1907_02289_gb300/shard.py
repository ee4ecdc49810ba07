"""Assignment of independent patches to GPUs (host logic).

A set of independent patches (the batched configuration: annular sectors
that never interact) is split across ranks with no data-path collective.
Each patch goes whole to one rank, chosen by the longest-processing-time
rule on an estimated cost: patches in decreasing cost order, each to the
rank with the smallest assigned cost so far (ties: lowest rank).  This is
the cost-ordered balance of Sec. 4.6 applied one level up, to GPUs instead
of cores.

Cost of a patch of n particles: n log2(n), the growth of the tree walk and
of the force work per particle with the tree depth at fixed surface density.
"""
from __future__ import annotations

import math


def patch_cost(n: int) -> float:
    """Estimated cost of a patch of n particles."""
    return float(n) * math.log2(max(n, 2))


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Patch indices per rank (each list ascending), by the LPT rule.

    Deterministic: every rank computes the same assignment from the same
    costs.  Raises ValueError for world < 1."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [float(c) for c in costs]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def imbalance(costs, assignment) -> float:
    """Largest rank load over the mean rank load (1.0 = perfect)."""
    loads = [sum(float(costs[i]) for i in part) for part in assignment]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0
