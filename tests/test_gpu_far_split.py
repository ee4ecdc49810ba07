"""The FP32 path's near/far split of the list particles (the expansion puts
"far" leaves after the near ones; the kernel gives far particles a single
FP32 separation and no contact test).

Pinned here, from the tree boxes and lists (themselves bit-exact with the
oracle in the parity tests):
* the count of far interactions the library reports equals the one
  recomputed on the host from the stated rule: a leaf is far for a group
  when its squared whole-cell gap d2 to the group box exceeds the widened
  contact reach ((a (1 + 1e-5) + 2)^2, a the contact reach in cells) and
  64 d2 >= (largest group side in cells)^2;
* no pair closer than r_coll ever has its j in a leaf that is far for i's
  group (brute force over all close pairs), also across the phi seam of a
  whole ring in the cylindrical frame;
* forces stay within the FP32 gate against the oracle (the other parity
  tests run the same split).
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import accel_of, assert_force_close, orc_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _prm(**kw):
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"])
    prm.update(n_g=64)
    prm.update(kw)
    return prm


def _build(P, prm):
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    return ctx, D


def _thresholds(prm, lo, L):
    """(widened contact reach rfar, phi period) on the key grid, by the
    stated rule."""
    S = 2097152.0 / L
    if prm.get("key_frame", 0) == 1:
        a = (prm["r_coll"] / lo[1] + 4e-6) * S
        period = int(math.floor(2 * math.pi * S))
    else:
        a = prm["r_coll"] * S
        period = 0
    w = a * (1.0 + 1e-5) + 2.0 if prm["r_coll"] > 0 else 0.0
    return int(math.floor(w * w)), period


def _gap2(qlo, qhi, glo, ghi, period):
    """Squared whole-cell gaps of boxes [qlo, qhi] (rows) to [glo, ghi]."""
    t1 = qlo[:, 0] - ghi[0] - 1
    t2 = glo[0] - qhi[:, 0] - 1
    d0 = np.maximum(0, np.maximum(t1, t2))
    if period > 0:
        wrap = np.where(t1 > 0, glo[0] + period - qhi[:, 0] - 1, qlo[:, 0] + period - ghi[0] - 1)
        d0 = np.where(d0 > 0, np.minimum(d0, np.maximum(0, wrap)), d0)
    d1 = np.maximum(0, np.maximum(qlo[:, 1] - ghi[1] - 1, glo[1] - qhi[:, 1] - 1))
    d2 = np.maximum(0, np.maximum(qlo[:, 2] - ghi[2] - 1, glo[2] - qhi[:, 2] - 1))
    return d0 * d0 + d1 * d1 + d2 * d2


def _far_leaves(ctx, prm):
    """Per group: (non-own leaves of its list, far flags); and the far
    interaction count n_i x (far particles) summed over groups."""
    t = ctx.bh_get_tree()
    grp = ctx.bh_get_groups()
    lst = ctx.bh_get_lists()
    lo, L = ctx.bh_get_root()
    rfar, period = _thresholds(prm, lo, L)
    qlo, qhi = t["qlo"].astype(np.int64), t["qhi"].astype(np.int64)
    b, e = t["begin"].astype(np.int64), t["end"].astype(np.int64)
    out, n_far = [], 0
    for k, g in enumerate(grp):
        lv = lst["P"][lst["pp_off"][k]:lst["pp_off"][k + 1]]
        lv = lv[~((b[lv] >= b[g]) & (b[lv] < e[g]))]
        ext = int((qhi[g] - qlo[g]).max()) + 1
        d2 = _gap2(qlo[lv], qhi[lv], qlo[g], qhi[g], period)
        far = (d2 > rfar) & (64 * d2 >= ext * ext)
        n_far += int(e[g] - b[g]) * int((e[lv[far]] - b[lv[far]]).sum())
        out.append((lv, far))
    return t, grp, out, n_far


def _check_no_close_pair_is_far(D, prm, t, grp, leaves):
    """Every pair (i, j) with |x_i - x_j| <= r_coll (1 + 1e-3): j's leaf is
    never far for i's group."""
    from scipy.spatial import cKDTree
    P = D.numpy()
    X = np.stack([P["x"], P["y"], P["z"]], 1)
    pairs = cKDTree(X).query_pairs(prm["r_coll"] * (1 + 1e-3), output_type="ndarray")
    assert len(pairs) > 0, "workload has no close pairs"
    pairs = np.concatenate([pairs, pairs[:, ::-1]])
    b, e = t["begin"].astype(np.int64), t["end"].astype(np.int64)
    leaf = np.nonzero(t["nchild"] == 0)[0]
    leaf_of = np.empty(len(X), np.int64)
    for q in leaf:
        leaf_of[b[q]:e[q]] = q
    gb = b[grp]
    order = np.argsort(gb)
    grp_of = order[np.searchsorted(gb[order], pairs[:, 0], side="right") - 1]
    far_set = {}
    for k, (lv, far) in enumerate(leaves):
        far_set[k] = set(lv[far].tolist())
    bad = [(i, j) for (i, j), k in zip(pairs, grp_of) if leaf_of[j] in far_set[k]]
    assert not bad, f"{len(bad)} close pairs in far leaves, e.g. {bad[:3]}"
    return len(pairs) // 2


@pytest.mark.parametrize("frame", [0, 1], ids=["cartesian", "cylindrical"])
def test_far_count_and_close_pairs(frame):
    if frame == 0:  # dense sector: ~4 contacts per particle
        P = synth.ring(20000, 31, r_in=0.99995, r_out=1.00005, phi_max=0.033, sigma_z=1e-5)
    else:  # whole thin ring: contacts across the phi seam too
        P = synth.ring(200000, 32, r_in=0.99999, r_out=1.00001, sigma_z=1e-6)
    prm = _prm(key_frame=frame)
    ctx, D = _build(P, prm)
    t, grp, leaves, n_far = _far_leaves(ctx, prm)
    c = ctx.bh_get_counters()
    assert c["n_pp_far"] == n_far
    # groups of the thin whole ring are long in phi, so few leaves clear an
    # eighth of their largest side; the sector has many far leaves
    assert (0.2 if frame == 0 else 0.0) * c["n_pp"] < n_far < c["n_pp"]
    _check_no_close_pair_is_far(D, prm, t, grp, leaves)


def test_fp64_path_has_no_split():
    P = synth.ring(20000, 33)
    ctx, _ = _build(P, _prm(precision=0))
    assert ctx.bh_get_counters()["n_pp_far"] == 0


@pytest.mark.parametrize("frame", [0, 1], ids=["cartesian", "cylindrical"])
def test_split_forces_meet_gate(frame):
    """Sector at the 2^26 ring's density with groups of up to 192: most list
    particles are far; the forces stay within the FP32 gate."""
    n = 1 << 17
    P = synth.ring(n, 34, phi_max=2 * math.pi * n / (1 << 26))
    prm = _prm(key_frame=frame, n_g=192, theta=0.4)
    ctx, D = _build(P, prm)
    c = ctx.bh_get_counters()
    assert c["n_pp_far"] > 0.3 * c["n_pp"]
    ref = orc.rebuild(P, orc_params(prm))
    a_ref = orc.tree_forces(ref, orc_params(prm))
    assert_force_close(accel_of(D), a_ref, 1e-5, f"frame {frame}")
