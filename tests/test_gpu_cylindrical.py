"""Cylindrical key frame (Sec. 4.3): keys, tree and opening test in
(phi, r, z), forces Cartesian.  GPU against the oracle: structures and lists
bit for bit, forces within the stated tolerances, across the phi seam too."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import accel_of, assert_force_close, gpu_build, orc_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _prm(**kw):
    prm = dict(synth.PRESETS["ring1m_fp64"]["params"])
    prm.update(n_g=64, key_frame=1)
    prm.update(kw)
    return prm


def _seam_ring(n=8000, seed=44):
    """A dense arc on both sides of phi = 0 (contacts across the seam)."""
    rng = np.random.default_rng(seed)
    phi = np.concatenate([rng.uniform(0, 2e-3, n // 2), rng.uniform(2 * np.pi - 2e-3, 2 * np.pi, n - n // 2)])
    r = rng.uniform(0.9998, 1.0002, n)
    return {"x": r * np.cos(phi), "y": r * np.sin(phi), "z": rng.normal(0, 5e-6, n),
            "vx": -np.sin(phi) / np.sqrt(r) + rng.normal(0, 1e-4, n), "vy": np.cos(phi) / np.sqrt(r),
            "vz": np.zeros(n), "m": np.full(n, 1e-12), "id": np.arange(n, dtype=np.int64)}


CASES = {"ring30k": lambda: synth.ring(30011, 45), "seam": _seam_ring}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_structures_lists_forces_match_oracle(name, prec):
    P = CASES[name]()
    prm = _prm(precision=prec)
    ref = orc.rebuild(P, orc_params(prm))
    ctx, D = gpu_build(P, prm)
    k, perm = ctx.bh_get_keys(len(P["x"]))
    assert np.array_equal(k, ref.skeys) and np.array_equal(perm, ref.perm)
    lo, L = ctx.bh_get_root()
    assert np.array_equal(lo, ref.lo) and L == ref.L
    t = ctx.bh_get_tree()
    for f in ("level", "begin", "end", "parent", "first_child", "nchild"):
        assert np.array_equal(t[f], ref.tree[f]), f
    assert np.array_equal(t["qlo"], ref.qlo) and np.array_equal(t["qhi"], ref.qhi)
    assert np.array_equal(ctx.bh_get_groups(), ref.groups)
    Lg = ctx.bh_get_lists()
    for f in ("pp_off", "P", "pc_off", "C"):
        assert np.array_equal(Lg[f], ref.lists[f]), f
    a_ref = orc.tree_forces(ref, orc_params(prm))
    assert_force_close(accel_of(D), a_ref, 1e-12 if prec == 0 else 1e-5, f"{name} prec {prec}")


def test_cylindrical_lists_shorter_or_equal_and_accurate_against_direct():
    """Reported comparison of the two frames on one ring, with the theta error
    of each against the direct sum on a sample."""
    P = synth.ring(20000, 46)
    out = {}
    for frame in (0, 1):
        prm = _prm(key_frame=frame, theta=0.5)
        S = orc.rebuild(P, orc_params(prm))
        a = orc.tree_forces(S, orc_params(prm))
        d = orc.direct(S.P, orc_params(prm))
        rel = np.linalg.norm(a - d, axis=1) / np.linalg.norm(d, axis=1)
        out[frame] = (len(S.lists["C"]) + len(S.lists["P"]), float(np.median(rel)), float(np.percentile(rel, 99)))
    print(f"\nentries / median / p99 theta error: cartesian {out[0]}, cylindrical {out[1]}")
    assert out[1][2] < 1e-2 and out[0][2] < 1e-2


def test_batch_patches_in_cylindrical_frame():
    from paper_1907_02289_gb300 import bh
    sizes = [5000, 12000, 3000]
    parts = [synth.ring(n, 700 + q, phi_max=2 * math.pi * n / (1 << 18), id0=sum(sizes[:q]))
             for q, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    prm = _prm(precision=1)
    ctx = bh.Context(offsets=off, **prm)
    D = bh.Particles({f: np.concatenate([p[f] for p in parts]) for f in synth.FIELDS})
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    a = accel_of(D)
    out = D.numpy()
    for q, p in enumerate(parts):
        ref = orc.rebuild(p, orc_params(prm))
        assert np.array_equal(out["id"][off[q]:off[q + 1]], ref.P["id"])
        assert_force_close(a[off[q]:off[q + 1]], orc.tree_forces(ref, orc_params(prm)), 1e-5, f"patch {q}")


def test_particle_on_axis_rejected():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(1000, 47)
    P["x"][5] = 0.0
    P["y"][5] = 0.0
    ctx = bh.Context(**_prm())
    D = bh.Particles(P)
    with pytest.raises(bh.BHError) as e:
        ctx.bh_build_tree(D)
    assert e.value.code == bh.BH_E_INVAL
