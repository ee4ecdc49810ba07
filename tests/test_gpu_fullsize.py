"""The ring configurations at their full sizes, in the launch configuration the
benchmark times: 2^20 (FP64 path, 10 steps with list reuse), 2^24 (FP32 vs FP64
on a 65,536-particle sample) and 2^26 (FP32 on a sample of whole groups).
Integer structures are compared bit for bit (the whole key array and tree,
the lists of the sampled groups); forces at the sampled particles against the
oracle, which builds the full tree but walks and sums only the sampled groups."""
import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import accel_of, assert_force_close, force_errors, orc_params

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _gpu(P, prm, precision):
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(**dict(prm, precision=precision))
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    return ctx, D


def _groups_of(particles):
    """group_subset for the oracle: the groups holding the given sorted-order
    particle indices."""
    def pick(grp, tree):
        b = tree["begin"][grp].astype(np.int64)
        return np.unique(np.searchsorted(b, particles, side="right") - 1)
    return pick


def _check_structures(ctx, n, S):
    k, perm = ctx.bh_get_keys(n)
    assert np.array_equal(k, S.skeys) and np.array_equal(perm, S.perm)
    t = ctx.bh_get_tree()
    for f in ("level", "begin", "end", "parent", "first_child", "nchild"):
        assert np.array_equal(t[f], S.tree[f]), f
    assert np.array_equal(t["qlo"], S.qlo) and np.array_equal(t["qhi"], S.qhi)


def _check_lists(ctx, S):
    """Lists of the oracle's (sampled) groups against the GPU's lists."""
    g_all = ctx.bh_get_groups()
    L = ctx.bh_get_lists()
    pos = np.full(int(max(g_all.max(), S.groups.max())) + 1, -1, np.int64)
    pos[g_all] = np.arange(len(g_all))
    where = pos[S.groups]
    assert (where >= 0).all()
    for q, k in enumerate(where):
        assert np.array_equal(L["P"][L["pp_off"][k]:L["pp_off"][k + 1]],
                              S.lists["P"][S.lists["pp_off"][q]:S.lists["pp_off"][q + 1]])
        assert np.array_equal(L["C"][L["pc_off"][k]:L["pc_off"][k + 1]],
                              S.lists["C"][S.lists["pc_off"][q]:S.lists["pc_off"][q + 1]])


def _sampled_rows(S):
    t = S.tree
    return np.concatenate([np.arange(t["begin"][g], t["end"][g]) for g in S.groups])


def test_ring_2p20_fp64_forces_and_ten_steps():
    """2^20 ring, FP64 path: every particle's force of the first evaluation
    within 1e-12 of the oracle; then 10 steps with list reuse, structures at
    the rebuilds of evaluations 4 and 8 bit for bit, and positions/velocities
    after 10 steps within the force tolerance propagated through the steps
    (the accelerations after 10 steps are not compared: positions differing
    in the last bit move contact forces, of stiffness kappa, by more than the
    force tolerance)."""
    from paper_1907_02289_gb300 import bh
    P, prm = synth.make("ring1m_fp64")
    op = orc_params(prm)
    ctx0, D0 = _gpu(P, prm, 0)
    S0 = orc.rebuild(P, op)
    _check_structures(ctx0, len(P["x"]), S0)
    assert_force_close(accel_of(D0), orc.tree_forces(S0, op), 1e-12, "2^20 first evaluation")
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_step(D, 4)
    ctx.bh_sync()
    S4, _, _ = orc.step(P, op, 4)
    _check_structures(ctx, len(P["x"]), S4)
    ctx.bh_step(D, 6)
    ctx.bh_sync()
    S10, aref, _ = orc.step(P, op, 10)
    _check_structures(ctx, len(P["x"]), S10)
    g = ctx.bh_get_groups()
    assert np.array_equal(g, S10.groups)
    out = D.numpy()
    assert np.array_equal(out["id"], S10.P["id"])
    a_tree = np.linalg.norm(aref - orc.central(S10.P["x"], S10.P["y"], S10.P["z"], 1.0, 1.0), axis=1).max()
    dx = max(np.abs(out[f] - S10.P[f]).max() for f in ("x", "y", "z"))
    dv = max(np.abs(out[f] - S10.P[f]).max() for f in ("vx", "vy", "vz"))
    assert dv <= 20 * prm["dt"] * 1e-12 * a_tree + 1e-14
    assert dx <= 200 * prm["dt"] ** 2 * 1e-12 * a_tree + 1e-14


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_ring_2p20_list_reusing_evaluation(precision, tol):
    """2^20 ring: after two leapfrog steps on the lists of the first build
    (evaluations 1 and 2 reuse them), one more list-reusing evaluation on the
    GPU's own state (positions and velocities as the steps left them) against
    the oracle's list-reusing evaluation (Sec. 4.2: moments refreshed, the
    first build's order, groups and lists kept) on that same state."""
    from paper_1907_02289_gb300 import bh
    P, prm = synth.make("ring1m_fp64")
    op = orc_params(prm)
    ctx = bh.Context(**dict(prm, precision=precision))
    D = bh.Particles(P)
    ctx.bh_step(D, 2)
    ctx.bh_sync()
    assert ctx.bh_get_counters()["n_rebuilds"] == 1
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    S = orc.rebuild(P, op)
    now = D.numpy()
    assert np.array_equal(now["id"], S.P["id"])
    L = ctx.bh_get_lists()
    assert np.array_equal(L["P"], S.lists["P"]) and np.array_equal(L["C"], S.lists["C"])
    S.P = {f: np.ascontiguousarray(now[f]) for f in orc.FIELDS}
    orc.refresh(S, op)
    assert_force_close(accel_of(D), orc.tree_forces(S, op), tol, f"2^20 list-reusing evaluation, precision {precision}")


def test_ring_2p24_fp32_vs_fp64_sample(capsys):
    """2^24 ring, theta 0.5: FP64 and FP32 forces on a 65,536-particle sample
    (rng(2)) against the oracle on the same lists."""
    P, prm = synth.make("ring16m_fp32")
    n = len(P["x"])
    sample = np.sort(np.random.default_rng(2).choice(n, 65536, replace=False))
    ctx64, D64 = _gpu(P, prm, 0)
    ctx32, D32 = _gpu(P, prm, 1)
    S = orc.rebuild(P, orc_params(prm), group_subset=_groups_of(sample))
    _check_structures(ctx64, n, S)
    _check_lists(ctx32, S)
    a_ref = orc.tree_forces(S, orc_params(prm))[sample]
    a64 = accel_of(D64)[sample]
    a32 = accel_of(D32)[sample]
    assert_force_close(a64, a_ref, 1e-12, "FP64 2^24")
    rel, rmsn, r = force_errors(a32, a_ref)
    with capsys.disabled():
        print(f"\n2^24 FP32 sample of 65536: max {rel.max():.3e} p99.9 {np.percentile(rel, 99.9):.3e} "
              f"median {np.median(rel):.3e} rms-normalised max {rmsn.max():.3e}")
    assert_force_close(a32, a_ref, 1e-5, "FP32 2^24")


def test_ring_2p26_fp32_sampled_groups(capsys):
    """2^26 ring, theta 0.4 (the benchmark workload): keys and tree bit for
    bit, the lists of 256 seeded groups, and FP32 forces of their particles."""
    P, prm = synth.make("ring64m_fp32")
    n = len(P["x"])
    ctx, D = _gpu(P, prm, 1)
    g_all = ctx.bh_get_groups()
    pick_idx = np.sort(np.random.default_rng(5).choice(len(g_all), 256, replace=False))
    S = orc.rebuild(P, orc_params(prm), group_subset=lambda grp, tree: pick_idx)
    _check_structures(ctx, n, S)
    _check_lists(ctx, S)
    rows = _sampled_rows(S)
    a_ref = orc.tree_forces(S, orc_params(prm))[rows]
    a32 = accel_of(D)[rows]
    rel, rmsn, r = force_errors(a32, a_ref)
    with capsys.disabled():
        print(f"\n2^26 FP32, {len(rows)} particles of 256 groups: max {rel.max():.3e} "
              f"p99.9 {np.percentile(rel, 99.9):.3e} median {np.median(rel):.3e} rms-normalised max {rmsn.max():.3e}")
    assert_force_close(a32, a_ref, 1e-5, "FP32 2^26")
