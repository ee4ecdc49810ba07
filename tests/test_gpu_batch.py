"""Independent patches in one context (bh_batch_create): every patch must come
out exactly as when it is run alone -- keys, order, tree, boxes, moments,
groups and lists bit for bit (node ids mapped), forces equal -- and its FP64
forces must match the oracle run on that patch alone."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import accel_of, assert_force_close, orc_params

pytestmark = pytest.mark.gpu

# uneven patches: one below n_g, ragged sizes, several sort tiles
SIZES = [3000, 20011, 517, 40961, 9000]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _params(**kw):
    prm = dict(synth.PRESETS["patches64"]["params"])
    prm.update(n_g=64, precision=0)
    prm.update(kw)
    return prm


def _patches():
    out = []
    for q, n in enumerate(SIZES):
        out.append(synth.ring(n, 500 + q, phi_max=2 * math.pi * n / (1 << 20), id0=sum(SIZES[:q])))
    return out


def _concat(parts):
    return {f: np.concatenate([p[f] for p in parts]) for f in synth.FIELDS}


def _run(P, prm, offsets=None, forces=True):
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(offsets=offsets, **prm)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    if forces:
        ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    return ctx, D


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "fp32"])
def runs(request):
    prm = _params(precision=request.param)
    parts = _patches()
    off = np.concatenate([[0], np.cumsum(SIZES)]).astype(np.int64)
    batch = _run(_concat(parts), prm, offsets=off)
    singles = [_run(p, prm) for p in parts]
    return prm, parts, off, batch, singles


def _patch_nodes(tree, off, q):
    """Batch node ids of patch q in id order (BFS: level-major, like the
    patch's own numbering)."""
    b = tree["begin"].astype(np.int64)
    return np.nonzero((b >= off[q]) & (b < off[q + 1]))[0]


def test_keys_order_root_per_patch(runs):
    prm, parts, off, (bc, bD), singles = runs
    n = int(off[-1])
    kb, pb = bc.bh_get_keys(n)
    lo, L = bc.bh_get_root()
    out = bD.numpy()
    for q, (sc, sD) in enumerate(singles):
        nq = SIZES[q]
        ks, ps = sc.bh_get_keys(nq)
        assert np.array_equal(kb[off[q]:off[q + 1]], ks)
        assert np.array_equal(pb[off[q]:off[q + 1]].astype(np.int64) - off[q], ps.astype(np.int64))
        los, Ls = sc.bh_get_root()
        assert np.array_equal(lo[q], los) and L[q] == Ls
        so = sD.numpy()
        for f in ("x", "y", "z", "vx", "vy", "vz", "m", "id"):
            assert np.array_equal(out[f][off[q]:off[q + 1]], so[f]), f


def test_tree_groups_lists_per_patch(runs):
    prm, parts, off, (bc, bD), singles = runs
    tb = bc.bh_get_tree()
    mb = bc.bh_get_moments()
    gb = bc.bh_get_groups()
    Lb = bc.bh_get_lists()
    assert np.array_equal(tb["level"][:len(SIZES)], np.zeros(len(SIZES)))  # roots 0..P-1
    for q, (sc, sD) in enumerate(singles):
        ids = _patch_nodes(tb, off, q)
        ts = sc.bh_get_tree()
        assert len(ids) == len(ts["level"])
        local = np.full(len(tb["level"]), -1, np.int64)
        local[ids] = np.arange(len(ids))
        assert np.array_equal(tb["level"][ids], ts["level"])
        assert np.array_equal(tb["begin"][ids].astype(np.int64) - off[q], ts["begin"])
        assert np.array_equal(tb["end"][ids].astype(np.int64) - off[q], ts["end"])
        par = tb["parent"][ids]
        assert np.array_equal(np.where(par >= 0, local[np.maximum(par, 0)], -1), ts["parent"])
        fc = tb["first_child"][ids]
        assert np.array_equal(np.where(fc >= 0, local[np.maximum(fc, 0)], -1), ts["first_child"])
        assert np.array_equal(tb["nchild"][ids], ts["nchild"])
        assert np.array_equal(tb["qlo"][ids], ts["qlo"]) and np.array_equal(tb["qhi"][ids], ts["qhi"])
        if prm["precision"] == 0:
            ms = sc.bh_get_moments()
            for f in ("M", "cx", "cy", "cz", "Q"):
                assert np.array_equal(mb[f][ids], ms[f]), f
        # groups of the patch, in order, and their lists
        gs = sc.bh_get_groups()
        sel = np.nonzero(local[gb] >= 0)[0]
        assert np.array_equal(local[gb[sel]], gs)
        Ls = sc.bh_get_lists()
        for k_local, k in enumerate(sel):
            pb = Lb["P"][Lb["pp_off"][k]:Lb["pp_off"][k + 1]]
            cb = Lb["C"][Lb["pc_off"][k]:Lb["pc_off"][k + 1]]
            ps = Ls["P"][Ls["pp_off"][k_local]:Ls["pp_off"][k_local + 1]]
            cs = Ls["C"][Ls["pc_off"][k_local]:Ls["pc_off"][k_local + 1]]
            assert np.array_equal(local[pb], ps) and np.array_equal(local[cb], cs)


def test_forces_equal_single_and_oracle(runs):
    prm, parts, off, (bc, bD), singles = runs
    ab = accel_of(bD)
    for q, (sc, sD) in enumerate(singles):
        a_s = accel_of(sD)
        np.testing.assert_allclose(ab[off[q]:off[q + 1]], a_s, rtol=1e-13, atol=0)
        ref = orc.rebuild(parts[q], orc_params(prm))
        aref = orc.tree_forces(ref, orc_params(prm))
        assert_force_close(a_s if prm["precision"] else ab[off[q]:off[q + 1]], aref,
                           1e-12 if prm["precision"] == 0 else 1e-5, f"patch {q}")


def test_steps_match_single_runs():
    from paper_1907_02289_gb300 import bh
    prm = _params(precision=1)
    parts = _patches()
    off = np.concatenate([[0], np.cumsum(SIZES)]).astype(np.int64)
    ctx = bh.Context(offsets=off, **prm)
    D = bh.Particles(_concat(parts))
    ctx.bh_step(D, 6)
    ctx.bh_sync()
    out = D.numpy()
    for q, p in enumerate(parts):
        cs = bh.Context(**prm)
        Ds = bh.Particles(p)
        cs.bh_step(Ds, 6)
        cs.bh_sync()
        so = Ds.numpy()
        for f in ("x", "y", "z", "vx", "vy", "vz"):
            np.testing.assert_allclose(out[f][off[q]:off[q + 1]], so[f], rtol=1e-13, atol=1e-18)
        assert np.array_equal(out["id"][off[q]:off[q + 1]], so["id"])


def test_bad_offsets_rejected():
    from paper_1907_02289_gb300 import bh
    prm = _params()
    for off in ([1, 10, 20], [0, 10, 10], [0, 20, 10]):
        with pytest.raises(bh.BHError):
            bh.Context(offsets=np.array(off), **prm)
    ctx = bh.Context(offsets=np.array([0, 100, 300]), **prm)
    D = bh.Particles(synth.ring(301, 3))
    with pytest.raises(bh.BHError) as e:
        ctx.bh_build_tree(D)
    assert e.value.code == bh.BH_E_INVAL


@pytest.mark.parametrize("prec", [0, 1])
def test_tiny_and_uneven_patches(prec):
    """Patches of 1, 2 and 3 particles beside a large one: the forest, the
    segmented sort and the per-patch walk still give each patch its own
    result (a lone particle feels nothing from the tree)."""
    from paper_1907_02289_gb300 import bh
    sizes = [1, 5000, 2, 3, 4097]
    parts = [synth.ring(n, 800 + q, phi_max=2 * math.pi * max(n, 64) / (1 << 20), id0=sum(sizes[:q]))
             for q, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    prm = _params(precision=prec)
    ctx, D = _run(_concat(parts), prm, offsets=off)
    a = accel_of(D)
    out = D.numpy()
    assert np.all(a[0] == 0.0)
    for q, p in enumerate(parts):
        sc, sD = _run(p, prm)
        so = sD.numpy()
        assert np.array_equal(out["id"][off[q]:off[q + 1]], so["id"])
        np.testing.assert_allclose(a[off[q]:off[q + 1]], accel_of(sD), rtol=1e-13, atol=0)
