"""List builds from one tree walk into per-group slots (sized from the
previous build's longest lists) give exactly the lists of the count-and-fill
walks: the first build (no slot sizes yet), a one-walk rebuild, a rebuild
whose lists outgrow the slots (larger n_g: falls back to count and fill) and
one whose slots would take too much memory (much smaller n_g: more groups) all
give the oracle's lists bit for bit, and rebuilding the same particles gives
the same forces."""
import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import accel_of, orc_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _lists_equal_oracle(ctx, D, prm):
    """The library's lists (mapped through its group/node numbering, which
    the parity tests pin to the oracle's) against the oracle's on the same
    sorted particles."""
    out = D.numpy()
    ref = orc.rebuild(out, orc_params(prm))
    L = ctx.bh_get_lists()
    for f in ("pp_off", "P", "pc_off", "C"):
        assert np.array_equal(L[f], ref.lists[f]), f
    return L


@pytest.mark.parametrize("prec", [0, 1])
def test_one_walk_builds_equal_count_and_fill(prec):
    from paper_1907_02289_gb300 import bh
    P = synth.ring(30011, 41)
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"])
    prm.update(n_g=64, precision=prec)
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    forces, builds = [], []
    for rebuild in range(3):
        ctx.bh_build_tree(D)
        ctx.bh_make_lists()
        ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
        ctx.bh_sync()
        builds.append(ctx.bh_get_counters()["n_one_walk_builds"])
        _lists_equal_oracle(ctx, D, prm)
        forces.append(accel_of(D))
    assert builds == [0, 1, 2]  # the first build has no slot sizes yet
    assert np.array_equal(forces[0], forces[1]) and np.array_equal(forces[0], forces[2])


def test_outgrown_and_oversized_slots_fall_back():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(30011, 42)
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"])
    prm.update(n_g=16)
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_sync()
    lp16 = np.diff(ctx.bh_get_lists()["pp_off"]).max()
    # larger groups: longer particle lists than the slots sized at n_g 16 hold
    ctx.bh_set_tuning(n_g=256)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_sync()
    L = _lists_equal_oracle(ctx, D, dict(prm, n_g=256))
    assert np.diff(L["pp_off"]).max() > lp16 + lp16 // 4 + 4
    assert ctx.bh_get_counters()["n_one_walk_builds"] == 0
    # the next build at n_g 256 fits its slots
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_sync()
    _lists_equal_oracle(ctx, D, dict(prm, n_g=256))
    assert ctx.bh_get_counters()["n_one_walk_builds"] == 1
    # down to n_g 8: many more groups, slots of the n_g 256 sizes would take
    # more than 4x the lists' storage, so count and fill again
    ctx.bh_set_tuning(n_g=8)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_sync()
    _lists_equal_oracle(ctx, D, dict(prm, n_g=8))
    assert ctx.bh_get_counters()["n_one_walk_builds"] == 1
