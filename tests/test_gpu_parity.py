"""GPU path vs the CPU oracle on the same seeded inputs (sizes the oracle
finishes in seconds; several tiles and ragged tails).  Integer structures are
compared bit for bit, forces within the stated tolerances."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import accel_of, assert_force_close, gpu_build, orc_params

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
# The uniform cube is an FP64 configuration; there a group spans ~1/4 of the
# box, so FP32 group-relative coordinates carry absolute errors of
# ~2^-24 x 0.5 against nearest separations ~1e-2 (eps = 1e-3): the FP32 form is
# held to 1e-4 there.  The 1e-5 gate is the ring configurations'.
TOL32_CUBE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def ring_prm(**kw):
    P, prm = synth.make("ring1m_fp64", 16)
    prm = dict(prm)
    prm.update(kw)
    return prm


CASES = {
    "cube4096": (lambda: synth.uniform_cube(4096, 0), dict(synth.PRESETS["cube4k"]["params"])),
    "ring20k": (lambda: synth.ring(20000, 7), ring_prm(n_g=64)),
    "ring_ragged_65537": (lambda: synth.ring(65537, 8), ring_prm()),
    "dense_contacts": (lambda: synth.ring(6000, 9, r_in=0.99995, r_out=1.00005, phi_max=4e-4, sigma_z=5e-6),
                       ring_prm(n_g=32, theta=0.6)),
}


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, (gen, prm) in CASES.items():
        P = gen()
        ref = orc.rebuild(P, orc_params(prm))
        out[name] = (P, prm, ref)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_keys_and_sort_bitexact(built, name):
    P, prm, ref = built[name]
    ctx, D = gpu_build(P, prm, forces=False)
    k, perm = ctx.bh_get_keys(len(P["x"]))
    assert np.array_equal(k, ref.skeys)
    assert np.array_equal(perm, ref.perm)
    lo, L = ctx.bh_get_root()
    assert np.array_equal(lo, ref.lo) and L == ref.L
    out = D.numpy()
    for f in ("x", "y", "z", "vx", "vy", "vz", "m", "id"):
        assert np.array_equal(out[f], ref.P[f]), f


@pytest.mark.parametrize("name", list(CASES))
def test_tree_boxes_moments_groups_bitexact(built, name):
    P, prm, ref = built[name]
    ctx, D = gpu_build(P, prm, forces=False)
    t = ctx.bh_get_tree()
    for f in ("level", "begin", "end", "parent", "first_child", "nchild"):
        assert np.array_equal(t[f], ref.tree[f]), f
    assert np.array_equal(t["qlo"], ref.qlo) and np.array_equal(t["qhi"], ref.qhi)
    mo = ctx.bh_get_moments()
    for f in ("M", "cx", "cy", "cz", "Q"):
        assert np.array_equal(mo[f], ref.mom[f]), f
    assert np.array_equal(ctx.bh_get_groups(), ref.groups)


@pytest.mark.parametrize("name", list(CASES))
def test_lists_bitexact(built, name):
    P, prm, ref = built[name]
    ctx, D = gpu_build(P, prm, forces=False)
    L = ctx.bh_get_lists()
    for f in ("pp_off", "P", "pc_off", "C"):
        assert np.array_equal(L[f], ref.lists[f]), f
    c = ctx.bh_get_counters()
    t = ref.tree
    ni = (t["end"][ref.groups].astype(np.int64) - t["begin"][ref.groups])
    leafn = (t["end"].astype(np.int64) - t["begin"])
    nj = np.array([leafn[ref.lists["P"][a:b]].sum() for a, b in zip(ref.lists["pp_off"][:-1], ref.lists["pp_off"][1:])])
    assert c["n_pp"] == int((ni * nj).sum())
    assert c["n_pc"] == int((ni * np.diff(ref.lists["pc_off"])).sum())


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_forces_vs_oracle(built, name, prec, tol):
    P, prm, ref = built[name]
    if name.startswith("cube") and prec == 1:
        tol = TOL32_CUBE
    aref = orc.tree_forces(ref, orc_params(prm))
    ctx, D = gpu_build(P, prm, precision=prec)
    a = accel_of(D)
    assert np.all(np.isfinite(a))
    assert_force_close(a, aref, tol, f"{name} prec={prec}")


@pytest.mark.parametrize("prec", [0, 1])
def test_central_term_added(built, prec):
    """Without BH_FORCE_TREE_ONLY the kernel adds -G M_c x / |x|^3 (FP64): the
    difference of the two outputs is the central term to FP64 rounding."""
    P, prm, ref = built["ring20k"]
    ac = orc.central(ref.P["x"], ref.P["y"], ref.P["z"], 1.0, 1.0)
    ctx, D = gpu_build(P, prm, precision=prec, flags=0)
    ctx2, D2 = gpu_build(P, prm, precision=prec)
    d = accel_of(D) - accel_of(D2)
    rel = np.linalg.norm(d - ac, axis=1) / np.linalg.norm(ac, axis=1)
    assert rel.max() <= 1e-13, rel.max()


def test_cube_vs_direct_reported(built):
    """Config 1: the tree error of theta = 0.5, monopole, against the direct
    sum (reported; the paper prints no accuracy) and the GPU against the CPU
    tree (gated)."""
    P, prm, ref = built["cube4096"]
    ad = orc.direct(ref.P, orc_params(prm))
    at = orc.tree_forces(ref, orc_params(prm))
    ctx, D = gpu_build(P, prm, precision=0)
    assert_force_close(accel_of(D), at, TOL64)
    err = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert np.median(err) < 1e-2


def test_theta_zero_gpu_equals_direct():
    P = synth.ring(3000, 2, r_in=0.999, r_out=1.001, phi_max=0.01)
    prm = ring_prm(theta=0.0, n_g=32, n_leaf=4)
    ref = orc.rebuild(P, orc_params(prm))
    ad = orc.direct(ref.P, orc_params(prm))
    ctx, D = gpu_build(P, prm, precision=0)
    assert ctx.bh_get_sizes()["n_pc"] == 0
    assert_force_close(accel_of(D), ad, TOL64)


# ---------------------------------------------------------------- edges ----
@pytest.mark.parametrize("n", [1, 2, 3, 9, 4097])
def test_small_and_ragged_n(n):
    P = synth.uniform_cube(n, 3)
    prm = dict(synth.PRESETS["cube4k"]["params"])
    ref = orc.rebuild(P, orc_params(prm))
    for prec, tol in ((0, TOL64), (1, TOL32_CUBE)):
        ctx, D = gpu_build(P, prm, precision=prec)
        L = ctx.bh_get_lists()
        assert np.array_equal(L["P"], ref.lists["P"]) and np.array_equal(L["C"], ref.lists["C"])
        aref = orc.tree_forces(ref, orc_params(prm))
        a = accel_of(D)
        if n == 1:
            assert np.all(a == 0)
        else:
            assert_force_close(a, aref, tol)


def test_coincident_particles_deep_leaf():
    """Many particles on one point: duplicate keys down to level 21, a leaf
    holding more than n_leaf and n_g particles; coincident pairs add nothing."""
    P = synth.uniform_cube(300, 4)
    for f in ("x", "y", "z"):
        P[f][:200] = 0.5
    prm = dict(synth.PRESETS["cube4k"]["params"], n_g=16)
    ref = orc.rebuild(P, orc_params(prm))
    assert ref.tree["level"].max() == 21
    for prec, tol in ((0, TOL64), (1, TOL32_CUBE)):
        ctx, D = gpu_build(P, prm, precision=prec)
        t = ctx.bh_get_tree()
        assert np.array_equal(t["begin"], ref.tree["begin"]) and np.array_equal(t["level"], ref.tree["level"])
        L = ctx.bh_get_lists()
        assert np.array_equal(L["P"], ref.lists["P"]) and np.array_equal(L["C"], ref.lists["C"])
        assert_force_close(accel_of(D), orc.tree_forces(ref, orc_params(prm)), tol)


def test_flat_ring_z_zero():
    P = synth.ring(5000, 5, sigma_z=0.0)
    prm = ring_prm(n_g=64)
    ref = orc.rebuild(P, orc_params(prm))
    for prec, tol in ((0, TOL64), (1, TOL32)):
        ctx, D = gpu_build(P, prm, precision=prec)
        L = ctx.bh_get_lists()
        assert np.array_equal(L["P"], ref.lists["P"]) and np.array_equal(L["C"], ref.lists["C"])
        assert_force_close(accel_of(D), orc.tree_forces(ref, orc_params(prm)), tol)


def test_errors_are_reported_not_trapped():
    from paper_1907_02289_gb300 import bh
    P = synth.uniform_cube(100, 1)
    P["x"][17] = np.nan
    ctx = bh.Context(**synth.PRESETS["cube4k"]["params"])
    D = bh.Particles(P)
    with pytest.raises(bh.BHError) as e:
        ctx.bh_build_tree(D)
    assert e.value.code == bh.BH_E_INVAL
    with pytest.raises(bh.BHError) as e:
        ctx.bh_compute_forces(D)
    assert e.value.code == bh.BH_E_STATE
    with pytest.raises(bh.BHError) as e:
        ctx.bh_make_lists()
    assert e.value.code == bh.BH_E_STATE
    for bad in (dict(theta=-1.0), dict(n_g=0), dict(n_leaf=100, n_g=64), dict(order=3), dict(precision=7)):
        with pytest.raises(bh.BHError):
            bh.Context(**dict(synth.PRESETS["cube4k"]["params"], **bad))
    # the context still works after the errors
    Q = synth.uniform_cube(100, 1)
    D = bh.Particles(Q)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D)
    ctx.bh_sync()


# ----------------------------------------------------------------- step ----
@pytest.mark.parametrize("prec", [0, 1])
def test_step_with_list_reuse_matches_oracle(prec):
    """10 KDK steps, lists rebuilt at force evaluations 0, 4, 8, vs the
    oracle's step.  Positions/velocities differ only through the force
    tolerance (times dt^2, summed over steps)."""
    n = 30000
    P = synth.ring(n, 12, r_in=0.999, r_out=1.001, phi_max=0.05)
    prm = ring_prm(n_g=64)
    S, aref, k = orc.step(P, orc_params(prm), 10)
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(**dict(prm, precision=prec))
    D = bh.Particles(P)
    ctx.bh_step(D, 10)
    ctx.bh_sync()
    c = ctx.bh_get_counters()
    assert c["n_rebuilds"] == 3 and c["n_evals"] == 3  # evaluations 8, 9, 10 since the last build
    out = D.numpy()
    assert np.array_equal(out["id"], S.P["id"])  # same sort order at the last rebuild
    dx = max(np.abs(out[f] - S.P[f]).max() for f in ("x", "y", "z"))
    dv = max(np.abs(out[f] - S.P[f]).max() for f in ("vx", "vy", "vz"))
    a_tree = np.linalg.norm(aref - orc.central(S.P["x"], S.P["y"], S.P["z"], 1.0, 1.0), axis=1).max()
    tol = TOL64 if prec == 0 else TOL32
    assert dv <= 20 * prm["dt"] * tol * a_tree + 1e-14
    assert dx <= 200 * prm["dt"] ** 2 * tol * a_tree + 1e-14


def test_step_host_buffers_equal_device_path():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(20000, 13, r_in=0.999, r_out=1.001, phi_max=0.05)
    prm = ring_prm(n_g=64, precision=1)
    c1 = bh.Context(**prm)
    D = bh.Particles(P)
    c1.bh_step(D, 3)
    c1.bh_step(D, 2)
    c1.bh_sync()
    c2 = bh.Context(**prm)
    H = bh.HostParticles(P)
    c2.bh_step_host(H, 3)
    c2.bh_step_host(H, 2)
    out = D.numpy()
    for f in ("x", "y", "z", "vx", "vy", "vz", "id", "ax"):
        assert np.array_equal(out[f], H.a[f]), f


@pytest.mark.parametrize("name", ["ring20k", "ring_ragged_65537", "cube4096"])
def test_fp32_moments_close(built, name):
    """The FP32 path's node records (FP32 mass and quadrupole, hi/lo centre)
    against the oracle's FP64 moments of the same tree."""
    P, prm, ref = built[name]
    ctx, D = gpu_build(P, prm, precision=1, forces=False)
    mo = ctx.bh_get_moments()
    t = ref.tree
    s = ref.L * 2.0 ** -t["level"].astype(float)  # node side
    M = ref.mom["M"]
    assert np.allclose(mo["M"], M, rtol=2e-6, atol=0)
    for f in ("cx", "cy", "cz"):
        assert np.all(np.abs(mo[f] - ref.mom[f]) <= 2e-6 * s + 1e-15)
    scale = (M * s * s)[:, None]
    assert np.all(np.abs(mo["Q"] - ref.mom["Q"]) <= 1e-5 * scale)


@pytest.mark.parametrize("n_g,chunk", [(16, 96), (40, 96), (100, 96), (200, 96), (300, 96), (100, 32), (200, 64),
                                       (300, 32)])
def test_fp32_every_group_size_class(n_g, chunk):
    """Groups from a few particles to several i-chunks (every slot/tail
    variant of the FP32 kernel and multi-chunk groups, at each i-chunk)."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(30000, 21, r_in=0.999, r_out=1.001, phi_max=0.05)
    prm = ring_prm(n_g=n_g, n_leaf=min(8, n_g))
    ref = orc.rebuild(P, orc_params(prm))
    sizes = ref.tree["end"][ref.groups].astype(int) - ref.tree["begin"][ref.groups]
    assert sizes.max() > min(n_g, chunk) // 2
    aref = orc.tree_forces(ref, orc_params(prm))
    ctx = bh.Context(**dict(prm, precision=1))
    ctx.bh_set_tuning(chunk=chunk)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    assert_force_close(accel_of(D), aref, TOL32, f"n_g={n_g} chunk={chunk}")
