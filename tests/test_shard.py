"""LPT assignment of independent patches to ranks (host logic, no GPU),
pinned to brute force: on small instances its largest load is within
Graham's bound (4/3 - 1/(3m)) of the optimal makespan found by trying every
assignment, every patch goes to exactly one rank, and the rule is the
textbook one (decreasing cost, least-loaded rank, lowest rank on ties)."""
import itertools
import math

import numpy as np
import pytest

from paper_1907_02289_gb300 import shard, synth


def _makespan(costs, parts):
    return max(sum(costs[i] for i in p) for p in parts)


@pytest.mark.parametrize("seed", range(12))
def test_lpt_within_graham_bound_of_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(2, 9)), int(rng.integers(2, 4))
    costs = [float(c) for c in rng.integers(1, 50, n)]
    parts = shard.lpt_assign(costs, m)
    assert sorted(i for p in parts for i in p) == list(range(n))
    best = min(max(sum(costs[i] for i in range(n) if a[i] == r) for r in range(m))
               for a in itertools.product(range(m), repeat=n))
    assert _makespan(costs, parts) <= (4 / 3 - 1 / (3 * m)) * best + 1e-9


def test_lpt_rule_by_hand():
    # costs 7, 5, 4, 3, 1 in decreasing order onto 2 ranks: 7 -> rank 0;
    # 5 -> 1; 4 -> 1 (load 5 < 7); 3 -> 0 (7 < 9); 1 -> 1 (9 < 10)
    parts = shard.lpt_assign([3, 7, 1, 5, 4], 2)
    assert parts == [[0, 1], [2, 3, 4]]
    # ties go to the lowest rank; equal costs keep index order
    assert shard.lpt_assign([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert shard.lpt_assign([2.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.lpt_assign([1.0], 0)


def test_patch_cost_and_imbalance():
    assert shard.patch_cost(1024) == 1024 * 10
    assert shard.patch_cost(1) == 1.0  # log2 floored at 1
    costs = [4.0, 4.0, 4.0, 4.0]
    assert shard.imbalance(costs, [[0, 1], [2, 3]]) == 1.0
    assert math.isclose(shard.imbalance(costs, [[0, 1, 2], [3]]), 1.5)


def test_batched_patches_split_evenly():
    """The 64 patches of the batched configuration over 2-8 ranks: estimated
    loads within a few percent of each other."""
    sizes = synth.patch_sizes(64, 3)
    costs = [shard.patch_cost(int(s)) for s in sizes]
    for m in (2, 4, 8):
        parts = shard.lpt_assign(costs, m)
        assert sorted(i for p in parts for i in p) == list(range(64))
        assert shard.imbalance(costs, parts) < 1.05
