"""Pins for the CPU oracle: every function is checked against something other
than itself -- hand-derived values, closed forms, conservation laws, special
cases that reduce to direct summation, and brute force on tiny inputs.

These run on the CPU (not marked gpu)."""
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- keys ----
def test_keys_hand_derived():
    """Golden keys worked out by hand from the key definition."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_keys.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for r in rows:
        lo = np.array([float(v) for v in r[0:3]])
        L = float(r[3])
        x, y, z = (np.array([float(r[4 + a])]) for a in range(3))
        k = orc.keys(x, y, z, lo, L)
        assert int(k[0]) == int(r[7], 16), r


def test_root_box_and_degenerate():
    x = np.array([0.5, -0.25, 0.75])
    y = np.array([1.0, 2.0, 1.5])
    z = np.array([0.0, 0.0, 0.0])
    lo, L = orc.root_box(x, y, z)
    assert list(lo) == [-0.25, 1.0, 0.0] and L == 1.0
    # one particle: extent 0 -> L = 1
    lo, L = orc.root_box(np.array([3.0]), np.array([4.0]), np.array([5.0]))
    assert L == 1.0 and list(lo) == [3.0, 4.0, 5.0]
    with pytest.raises(ValueError):
        orc.root_box(np.array([np.nan]), np.array([0.0]), np.array([0.0]))


def test_key_coords_roundtrip_and_order():
    rng = np.random.default_rng(5)
    q = rng.integers(0, 1 << 21, (1000, 3))
    # encode with integer arithmetic on a unit box: x = (q + 0.5) / 2^21
    x, y, z = ((q[:, a] + 0.5) / 2 ** 21 for a in range(3))
    k = orc.keys(x, y, z, np.zeros(3), 1.0)
    assert np.array_equal(orc.key_coords(k).astype(np.int64), q)
    # Morton property: the top digit is the octant of the unit cube
    oct_ = ((q[:, 0] >= 2 ** 20) * 4 + (q[:, 1] >= 2 ** 20) * 2 + (q[:, 2] >= 2 ** 20) * 1)
    assert np.array_equal((k >> np.uint64(60)).astype(np.int64), oct_)


# ----------------------------------------------------------------- sort ----
def test_sort_is_stable_permutation():
    rng = np.random.default_rng(1)
    k = rng.integers(0, 50, 5000).astype(np.uint64)  # many ties
    p = orc.sort_perm(k).astype(np.int64)
    assert np.array_equal(p, orc.sort_perm_c(k))
    assert np.array_equal(np.sort(p), np.arange(len(k)))
    sk = k[p]
    assert np.all(sk[1:] >= sk[:-1])
    ties = sk[1:] == sk[:-1]
    assert np.all(p[1:][ties] > p[:-1][ties])  # ties keep input order
    assert np.array_equal(p, np.argsort(k, kind="stable"))


# ----------------------------------------------------------------- tree ----
def _digit(k, level):
    return (int(k) >> (3 * (21 - level))) & 7


def _brute_tree(sk, n_leaf):
    """Recursive definition, then numbered level by level in key order."""
    def rec(b, e, lev):
        node = {"b": b, "e": e, "lev": lev, "kids": []}
        if e - b > n_leaf and lev < 21:
            for o in range(8):
                idx = [i for i in range(b, e) if _digit(sk[i], lev + 1) == o]
                if idx:
                    assert idx == list(range(idx[0], idx[-1] + 1))
                    node["kids"].append(rec(idx[0], idx[-1] + 1, lev + 1))
        return node
    root = rec(0, len(sk), 0)
    order, frontier = [], [root]
    while frontier:
        order.extend(frontier)
        frontier = [c for nd in frontier for c in nd["kids"]]
    return order


@pytest.mark.parametrize("seed,n,n_leaf", [(0, 1, 8), (1, 2, 1), (2, 9, 8), (3, 64, 8), (4, 64, 1), (5, 40, 3)])
def test_tree_matches_brute_force(seed, n, n_leaf):
    P = synth.uniform_cube(n, seed)
    lo, L = orc.root_box(P["x"], P["y"], P["z"])
    k = orc.keys(P["x"], P["y"], P["z"], lo, L)
    sk = np.ascontiguousarray(k[orc.sort_perm(k)])
    t = orc.build_tree(sk, n_leaf)
    ref = _brute_tree(sk, n_leaf)
    assert len(ref) == len(t["level"])
    ids = {id(nd): i for i, nd in enumerate(ref)}
    for i, nd in enumerate(ref):
        assert (t["begin"][i], t["end"][i], t["level"][i]) == (nd["b"], nd["e"], nd["lev"])
        assert t["nchild"][i] == len(nd["kids"])
        if nd["kids"]:
            assert t["first_child"][i] == ids[id(nd["kids"][0])]
            assert [ids[id(c)] for c in nd["kids"]] == list(range(t["first_child"][i], t["first_child"][i] + len(nd["kids"])))
            for c in nd["kids"]:
                assert t["parent"][ids[id(c)]] == i


def _ring_state(n, seed=7, **kw):
    P = synth.ring(n, seed)
    prm = orc.Params(**{**dict(theta=0.5, n_g=64, n_leaf=8, order=2, r_coll=2e-5), **kw})
    return P, prm, orc.rebuild(P, prm)


def test_tree_invariants_ring():
    P, prm, S = _ring_state(20000)
    t = S.tree
    nn = len(t["level"])
    leaf = t["nchild"] == 0
    cnt = t["end"].astype(np.int64) - t["begin"]
    assert np.all(cnt > 0)
    assert np.all(cnt[leaf] <= prm.n_leaf) or np.all(t["level"][leaf & (cnt > prm.n_leaf)] == 21)
    # leaves partition [0, n)
    lb = np.sort(t["begin"][leaf]); le = np.sort(t["end"][leaf])
    assert lb[0] == 0 and le[-1] == 20000 and np.array_equal(lb[1:], le[:-1])
    # children partition their parent, levels increase by one, BFS numbering
    for k in np.nonzero(~leaf)[0]:
        f, c = t["first_child"][k], t["nchild"][k]
        assert t["begin"][f] == t["begin"][k] and t["end"][f + c - 1] == t["end"][k]
        assert np.array_equal(t["begin"][f + 1:f + c], t["end"][f:f + c - 1])
        assert np.all(t["level"][f:f + c] == t["level"][k] + 1) and f > k
    assert np.all(np.diff(t["level"].astype(int)) >= 0)
    # every particle of a node shares the node's key prefix
    sk = S.skeys
    for k in range(0, nn, 97):
        lev = int(t["level"][k]); b, e = t["begin"][k], t["end"][k]
        sh = np.uint64(3 * (21 - lev))
        pre = sk[b:e] >> sh if lev < 21 else sk[b:e]
        assert np.all(pre == pre[0])


def test_qboxes_brute_force():
    P, prm, S = _ring_state(3000)
    q = orc.key_coords(S.skeys).astype(np.int64)
    t = S.tree
    for k in range(len(t["level"])):
        b, e = t["begin"][k], t["end"][k]
        assert np.array_equal(S.qlo[k], q[b:e].min(0)) and np.array_equal(S.qhi[k], q[b:e].max(0))


# -------------------------------------------------------------- moments ----
def test_moments_two_masses_closed_form():
    """Two masses m at (+-a,0,0): M = 2m, c = 0, Qxx = 4 m a^2, Qyy = Qzz = -2 m a^2."""
    t = {"begin": np.array([0], np.uint32), "end": np.array([2], np.uint32),
         "first_child": np.array([-1], np.int32), "nchild": np.array([0], np.uint8), "level": np.array([0], np.uint8)}
    a, m = 0.25, 3.0
    mo = orc.moments(t, np.array([-a, a]), np.zeros(2), np.zeros(2), np.array([m, m]), 2)
    assert mo["M"][0] == 2 * m and mo["cx"][0] == 0.0
    assert np.allclose(mo["Q"][0], [4 * m * a * a, -2 * m * a * a, -2 * m * a * a, 0, 0, 0], rtol=0, atol=1e-15)


def test_moments_hierarchy_equals_direct():
    """Bottom-up moments (parallel-axis shifts) equal the direct sums over
    every node's particles."""
    P, prm, S = _ring_state(5000)
    t, mo, Q = S.tree, S.mom, S.P
    x = np.stack([Q["x"], Q["y"], Q["z"]], 1); m = Q["m"]
    for k in list(range(0, len(t["level"]), 53)) + [0]:
        b, e = t["begin"][k], t["end"][k]
        Mk = m[b:e].sum(); c = (m[b:e, None] * x[b:e]).sum(0) / Mk
        assert math.isclose(mo["M"][k], Mk, rel_tol=1e-13)
        assert np.allclose([mo["cx"][k], mo["cy"][k], mo["cz"][k]], c, rtol=0, atol=1e-14)
        d = x[b:e] - c; d2 = (d * d).sum(1)
        Qd = [(m[b:e] * (3 * d[:, 0] ** 2 - d2)).sum(), (m[b:e] * (3 * d[:, 1] ** 2 - d2)).sum(),
              (m[b:e] * (3 * d[:, 2] ** 2 - d2)).sum(), (3 * m[b:e] * d[:, 0] * d[:, 1]).sum(),
              (3 * m[b:e] * d[:, 0] * d[:, 2]).sum(), (3 * m[b:e] * d[:, 1] * d[:, 2]).sum()]
        scale = Mk * (d2.max() + 1e-300)
        assert np.allclose(mo["Q"][k], Qd, rtol=0, atol=1e-10 * scale)
        assert abs(mo["Q"][k][0] + mo["Q"][k][1] + mo["Q"][k][2]) <= 1e-10 * scale  # traceless


# --------------------------------------------------------------- groups ----
def test_groups_partition_and_maximal():
    P, prm, S = _ring_state(20000, n_g=64)
    t, g = S.tree, S.groups
    b, e = t["begin"][g].astype(np.int64), t["end"][g].astype(np.int64)
    assert b[0] == 0 and e[-1] == 20000 and np.array_equal(b[1:], e[:-1])  # partition, ordered by begin
    cnt = e - b
    assert np.all((cnt <= prm.n_g) | (t["nchild"][g] == 0))
    par = t["parent"][g]
    assert np.all((g == 0) | (t["end"][par].astype(np.int64) - t["begin"][par] > prm.n_g))


# ---------------------------------------------------------------- lists ----
def _ranges(S, k):
    t, L = S.tree, S.lists
    ent = [(int(t["begin"][c]), int(t["end"][c]), "P", c) for c in L["P"][L["pp_off"][k]:L["pp_off"][k + 1]]]
    ent += [(int(t["begin"][c]), int(t["end"][c]), "C", c) for c in L["C"][L["pc_off"][k]:L["pc_off"][k + 1]]]
    return ent


def test_lists_partition_and_order():
    P, prm, S = _ring_state(20000)
    n = 20000
    for k in range(0, len(S.groups), 7):
        ent = _ranges(S, k)
        ent_sorted = sorted(ent)
        assert ent_sorted[0][0] == 0 and ent_sorted[-1][1] == n
        assert all(ent_sorted[i][1] == ent_sorted[i + 1][0] for i in range(len(ent) - 1))
        for kind in "PC":  # each list is in ascending first particle
            bs = [r[0] for r in ent if r[2] == kind]
            assert bs == sorted(bs)
        assert all(S.tree["nchild"][r[3]] == 0 for r in ent if r[2] == "P")
        # the group's own particles are always particles of its list
        gb, ge = S.tree["begin"][S.groups[k]], S.tree["end"][S.groups[k]]
        assert all(r[2] == "P" for r in ent if r[0] < ge and r[1] > gb)


def test_lists_theta_zero_all_leaves():
    P, prm, S = _ring_state(3000, theta=0.0)
    leaves = np.nonzero(S.tree["nchild"] == 0)[0]
    leaves = leaves[np.argsort(S.tree["begin"][leaves])]
    L = S.lists
    assert len(L["C"]) == 0
    for k in range(len(S.groups)):
        assert np.array_equal(L["P"][L["pp_off"][k]:L["pp_off"][k + 1]], leaves)


def test_lists_accepted_cells_are_far_and_contacts_are_particles():
    """An accepted cell satisfies the opening angle against the true particle
    positions (quantised boxes only make the test more conservative), and
    every particle within r_coll of a group particle is in the P-list."""
    n = 4000
    P = synth.ring(n, 11, r_in=0.999, r_out=1.001, phi_max=0.01, sigma_z=1e-5)
    prm = orc.Params(theta=0.6, n_g=32, n_leaf=4, order=2, r_coll=3e-5)
    S = orc.rebuild(P, prm)
    X = np.stack([S.P["x"], S.P["y"], S.P["z"]], 1)
    t = S.tree
    side = S.L * 2.0 ** -t["level"].astype(float)
    for k in range(0, len(S.groups), 3):
        g = S.groups[k]; gb, ge = t["begin"][g], t["end"][g]
        Xi = X[gb:ge]
        inP = np.zeros(n, bool)
        for b, e, kind, c in _ranges(S, k):
            if kind == "P":
                inP[b:e] = True
            else:
                d = np.sqrt(((Xi[:, None, :] - X[None, b:e, :]) ** 2).sum(-1)).min()
                assert side[c] <= prm.theta * d * (1 + 1e-12) + 1e-15
                assert d > prm.r_coll
        d_all = np.sqrt(((Xi[:, None, :] - X[None, :, :]) ** 2).sum(-1)).min(0)
        assert np.all(inP[d_all <= prm.r_coll])


def test_lists_brute_force_ancestor_definition():
    """C(g) = accepted nodes all of whose proper ancestors are opened;
    P(g) = opened leaves all of whose ancestors are opened.  The opening
    decisions are read back from a traversal-free evaluation per node."""
    P, prm, S = _ring_state(64, n_g=8, n_leaf=2, theta=0.7)
    t = S.tree
    nn = len(t["level"])
    S2 = 2097152.0 / S.L * prm.r_coll
    rcq2 = S2 * S2

    def opened(g, c):  # definition of the opening test, on integer boxes
        d2 = 0
        for a in range(3):
            delta = max(0, int(S.qlo[c][a]) - int(S.qhi[g][a]) - 1, int(S.qlo[g][a]) - int(S.qhi[c][a]) - 1)
            d2 += delta * delta
        s = 2.0 ** (21 - int(t["level"][c]))
        return prm.theta * prm.theta * float(d2) < s * s or float(d2) <= rcq2

    for k, g in enumerate(S.groups):
        Pset, Cset = [], []
        for c in range(nn):
            anc, a = [], t["parent"][c]
            while a >= 0:
                anc.append(a); a = t["parent"][a]
            if not all(opened(g, a) for a in anc):
                continue
            if opened(g, c):
                if t["nchild"][c] == 0:
                    Pset.append(c)
            else:
                Cset.append(c)
        L = S.lists
        key = lambda c: t["begin"][c]
        assert list(L["P"][L["pp_off"][k]:L["pp_off"][k + 1]]) == sorted(Pset, key=key)
        assert list(L["C"][L["pc_off"][k]:L["pc_off"][k + 1]]) == sorted(Cset, key=key)


# ---------------------------------------------------------- pair (Eq. 1) ----
def test_pair_two_body_closed_form():
    prm = orc.Params(G=1.0)
    a = orc.pair_accel(prm, [0, 0, 0], [0, 0, 0], 1.0, [3, 4, 0], [0, 0, 0], 2.0)
    assert np.allclose(a, [2 * 3 / 125, 2 * 4 / 125, 0], rtol=1e-15, atol=0)
    prm = orc.Params(G=2.0, eps=1.0)  # softened: G m r / (r^2+eps^2)^1.5 = 2*1*(1,0,0)/2^1.5
    a = orc.pair_accel(prm, [0, 0, 0], [0, 0, 0], 1.0, [1, 0, 0], [0, 0, 0], 1.0)
    assert math.isclose(a[0], 2.0 / 2 ** 1.5, rel_tol=1e-15)
    assert np.all(orc.pair_accel(prm, [1, 2, 3], [0, 0, 0], 1.0, [1, 2, 3], [1, 0, 0], 1.0) == 0)


def test_pair_gravity_continuous_at_rcoll_and_contact_terms():
    kappa, eta = 100.0, 3.0
    prm = orc.Params(G=1.0, r_coll=0.1, kappa=kappa, eta=eta)
    out = orc.pair_accel(prm, [0, 0, 0], [0, 0, 0], 1.0, [0.1 * (1 + 1e-12), 0, 0], [0, 0, 0], 1.0)
    ins = orc.pair_accel(prm, [0, 0, 0], [0, 0, 0], 1.0, [0.1, 0, 0], [0, 0, 0], 1.0)
    assert math.isclose(out[0], ins[0], rel_tol=1e-9)  # kappa term vanishes at r = r_coll
    # overlap 0.05 at rest: a_x = [G m_j/rc^3 + m_j/(m_i+m_j) kappa (r - rc)/r] r
    r = 0.05
    a = orc.pair_accel(prm, [0, 0, 0], [0, 0, 0], 1.0, [r, 0, 0], [0, 0, 0], 3.0)
    assert math.isclose(a[0], (3.0 / 0.1 ** 3 + 0.75 * kappa * (r - 0.1) / r) * r, rel_tol=1e-14)
    # approaching at speed 2: dashpot adds m_j/(m_i+m_j) eta (r.v)/r^2 * r
    a2 = orc.pair_accel(prm, [0, 0, 0], [0, 0, 0], 1.0, [r, 0, 0], [-2.0, 0, 0], 3.0)
    assert math.isclose(a2[0] - a[0], 0.75 * eta * (r * -2.0) / r ** 2 * r, rel_tol=1e-12)


def test_contact_restitution_half():
    """Head-on pair, gravity off: the outgoing/incoming relative speed is the
    restitution coefficient exp(-eta t_c / 2) = 0.5 (the paper's choice)."""
    dt = 1e-3
    kappa, eta = synth.contact_params(dt)
    prm = orc.Params(G=0.0, r_coll=2e-5, kappa=kappa, eta=eta)
    h = 8 * dt / 4000  # fine substeps of the leapfrog
    x = np.array([[0.0, 0, 0], [2.2e-5, 0, 0]]); v = np.array([[0.0, 0, 0], [-1e-3, 0, 0]])
    m = [1.0, 1.0]
    acc = lambda x, v: np.array([orc.pair_accel(prm, x[0], v[0], m[0], x[1], v[1], m[1]),
                                 orc.pair_accel(prm, x[1], v[1], m[1], x[0], v[0], m[0])])
    vin = v[1, 0] - v[0, 0]
    a = acc(x, v)
    for _ in range(40000):
        v = v + 0.5 * h * a; x = x + h * v; a = acc(x, v); v = v + 0.5 * h * a
        if x[1, 0] - x[0, 0] > 2.2e-5 and v[1, 0] - v[0, 0] > 0:
            break
    e = (v[1, 0] - v[0, 0]) / -vin
    assert abs(e - 0.5) < 5e-3


# ---------------------------------------------------------------- cells ----
def test_cell_far_field_convergence_orders():
    """Monopole error ~ (s/d)^2 (dipole vanishes about the COM), quadrupole
    error ~ (s/d)^3, against direct summation over the cell's particles."""
    rng = np.random.default_rng(3)
    xs = rng.random((30, 3)) - 0.5; ms = rng.random(30) + 0.5
    t = {"begin": np.array([0], np.uint32), "end": np.array([30], np.uint32),
         "first_child": np.array([-1], np.int32), "nchild": np.array([0], np.uint8), "level": np.array([0], np.uint8)}
    mo = orc.moments(t, *(np.ascontiguousarray(xs[:, a]) for a in range(3)), ms, 2)
    c = [mo["cx"][0], mo["cy"][0], mo["cz"][0]]
    prm = orc.Params(G=1.0)
    u = np.array([0.48, 0.6, 0.64])
    err = {1: [], 2: []}
    for d in (8.0, 16.0, 32.0, 64.0):
        xi = d * u
        ref = sum(orc.pair_accel(prm, xi, [0, 0, 0], 1.0, xs[j], [0, 0, 0], ms[j]) for j in range(30))
        for order in (1, 2):
            a = orc.cell_accel(1.0, 0.0, order, xi, mo["M"][0], c, mo["Q"][0])
            err[order].append(np.linalg.norm(a - ref) / np.linalg.norm(ref))
    s1 = np.diff(np.log2(err[1])); s2 = np.diff(np.log2(err[2]))
    assert np.all(np.abs(s1 + 2) < 0.15), s1
    assert np.all(np.abs(s2 + 3) < 0.15), s2


def test_cell_two_masses_on_axis():
    """On the axis of two masses m at +-a: exact a_x = -Gm[1/(X-a)^2 + 1/(X+a)^2];
    the quadrupole expansion is -G(2m/X^2 + 6 m a^2 / X^4); the remainder is the
    next even term, relative size 5 u^4 (u = a/X) to leading order."""
    m, a0, X = 1.0, 0.1, 5.0
    Q = [4 * m * a0 * a0, -2 * m * a0 * a0, -2 * m * a0 * a0, 0, 0, 0]
    ac = orc.cell_accel(1.0, 0.0, 2, [X, 0, 0], 2 * m, [0, 0, 0], Q)
    assert math.isclose(ac[0], -(2 * m / X ** 2 + 6 * m * a0 ** 2 / X ** 4), rel_tol=1e-14)
    exact = -m * (1 / (X - a0) ** 2 + 1 / (X + a0) ** 2)
    u = a0 / X
    assert abs(abs(ac[0] - exact) / abs(exact) - 5 * u ** 4) < 0.02 * 5 * u ** 4


# ------------------------------------------------------- direct and tree ----
def test_direct_momentum_conservation():
    rng = np.random.default_rng(4)
    n = 300
    P = synth.ring(n, 9, r_in=0.9999, r_out=1.0001, phi_max=2e-4, sigma_z=1e-5)
    P["m"] = 1e-12 * (1 + rng.random(n))
    kappa, eta = synth.contact_params(1e-3)
    prm = orc.Params(G=1.0, r_coll=2e-5, kappa=kappa, eta=eta)
    a = orc.direct(P, prm)
    ma = (P["m"][:, None] * a).sum(0)
    scale = (P["m"][:, None] * np.abs(a)).sum(0)
    assert np.all(np.abs(ma) <= 1e-12 * scale)


def test_tree_theta_zero_equals_direct_bitwise():
    P = synth.ring(3000, 2, r_in=0.999, r_out=1.001, phi_max=0.01)
    kappa, eta = synth.contact_params(1e-3)
    prm = orc.Params(theta=0.0, n_g=32, n_leaf=4, order=2, r_coll=2e-5, kappa=kappa, eta=eta)
    S = orc.rebuild(P, prm)
    at = orc.tree_forces(S, prm)
    ad = orc.direct(S.P, prm)
    assert np.array_equal(at, ad)


def test_tree_error_decreases_with_theta_and_order():
    """Reported, not gated by the paper: the tree error at theta > 0 shrinks
    with theta and with the multipole order."""
    P = synth.uniform_cube(2000, 0)
    ad = None
    errs = {}
    for order in (1, 2):
        for th in (0.8, 0.4):
            prm = orc.Params(theta=th, n_g=32, n_leaf=8, order=order, eps=1e-3)
            S = orc.rebuild(P, prm)
            if ad is None:
                ad = orc.direct(S.P, prm)
            at = orc.tree_forces(S, prm)
            errs[(order, th)] = np.median(np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1))
    assert errs[(1, 0.4)] < errs[(1, 0.8)] and errs[(2, 0.4)] < errs[(2, 0.8)]
    assert errs[(2, 0.4)] < errs[(1, 0.4)] and errs[(2, 0.4)] < 1e-3


# ---------------------------------------------------- list reuse (refresh) ----
def test_refresh_keeps_lists_and_recomputes_moments_of_moved_particles():
    """The list-reusing evaluation (Sec. 4.2): after the particles move, the
    order, tree, groups and lists stay as built, and every node's moments are
    those of its (moved) particles, summed directly."""
    P, prm, S = _ring_state(5000)
    lists0 = {k: v.copy() for k, v in S.lists.items()}
    groups0, begin0 = S.groups.copy(), S.tree["begin"].copy()
    rng = np.random.default_rng(9)
    for c in "xyz":
        S.P[c] = S.P[c] + rng.normal(0.0, 3e-5, len(S.P[c]))
    orc.refresh(S, prm)
    assert all(np.array_equal(S.lists[k], lists0[k]) for k in lists0)
    assert np.array_equal(S.groups, groups0) and np.array_equal(S.tree["begin"], begin0)
    t, mo, Q = S.tree, S.mom, S.P
    x = np.stack([Q["x"], Q["y"], Q["z"]], 1); m = Q["m"]
    for k in list(range(0, len(t["level"]), 37)) + [0]:
        b, e = t["begin"][k], t["end"][k]
        Mk = m[b:e].sum(); c = (m[b:e, None] * x[b:e]).sum(0) / Mk
        assert math.isclose(mo["M"][k], Mk, rel_tol=1e-13)
        assert np.allclose([mo["cx"][k], mo["cy"][k], mo["cz"][k]], c, rtol=0, atol=1e-14)
        d = x[b:e] - c; d2 = (d * d).sum(1)
        assert math.isclose(mo["Q"][k][3], (3 * m[b:e] * d[:, 0] * d[:, 1]).sum(), rel_tol=1e-9,
                            abs_tol=1e-10 * Mk * (d2.max() + 1e-300))


def test_reused_lists_at_theta_zero_still_cover_every_pair():
    """At theta = 0 every list holds every leaf, so an evaluation on reused
    lists after the particles moved is still the direct sum in the current
    order (bit for bit), and a 4-step run with rebuilds every 4 evaluations
    stays within rounding of one that rebuilds at every evaluation."""
    P = synth.ring(1500, 12, r_in=0.999, r_out=1.001, phi_max=0.01)
    kappa, eta = synth.contact_params(1e-3)
    prm = orc.Params(theta=0.0, n_g=32, n_leaf=4, order=2, r_coll=2e-5, kappa=kappa, eta=eta, M_central=1.0,
                     dt=1e-3, rebuild_every=4)
    S = orc.rebuild(P, prm)
    for c in "xyz":
        S.P[c] = S.P[c] + 1e-3 * S.P["v" + c]
    orc.refresh(S, prm)
    assert np.array_equal(orc.tree_forces(S, prm), orc.direct(S.P, prm))
    S4, a4, _ = orc.step(P, prm, 3)
    S1, a1, _ = orc.step(P, orc.Params(**{**prm.__dict__, "rebuild_every": 1}), 3)
    o4, o1 = np.argsort(S4.P["id"]), np.argsort(S1.P["id"])
    assert np.allclose(a4[o4], a1[o1], rtol=1e-10, atol=0)
    assert np.max(np.abs(S4.P["x"][o4] - S1.P["x"][o1])) < 1e-15


# ----------------------------------------------------------------- step ----
def test_step_circular_orbit():
    """One particle about M_c = 1: KDK keeps a circular orbit's radius to
    O(dt^2) and returns near the start after one period 2 pi."""
    P = {"x": np.array([1.0]), "y": np.array([0.0]), "z": np.array([0.0]), "vx": np.array([0.0]),
         "vy": np.array([1.0]), "vz": np.array([0.0]), "m": np.array([1e-12]), "id": np.array([0], np.int64)}
    nst = 628
    prm = orc.Params(G=1.0, M_central=1.0, dt=2 * math.pi / nst, rebuild_every=4)
    S, a, k = orc.step(P, prm, nst)
    r = math.hypot(S.P["x"][0], S.P["y"][0])
    assert abs(r - 1.0) < 2 * prm.dt ** 2 and k == nst + 1
    assert math.hypot(S.P["x"][0] - 1.0, S.P["y"][0]) < 1e-3


def test_step_time_reversible_and_schedule():
    """KDK without contact is time-reversible: run n steps, flip v, run n
    steps, flip v -> back to the start (to rounding)."""
    P = synth.ring(200, 3, r_in=0.999, r_out=1.001, phi_max=0.002, mass=1e-9)
    prm = orc.Params(theta=0.5, n_g=16, n_leaf=4, order=2, G=1.0, M_central=1.0, dt=1e-3, rebuild_every=1)
    S, a, k = orc.step(P, prm, 6)
    assert k == 7
    Q = {f: S.P[f].copy() for f in S.P}
    for c in ("vx", "vy", "vz"):
        Q[c] = -Q[c]
    S2, _, _ = orc.step(Q, prm, 6)
    back = {f: S2.P[f][np.argsort(S2.P["id"])] for f in S2.P}
    x0 = np.stack([P["x"], P["y"], P["z"]], 1); x1 = np.stack([back["x"], back["y"], back["z"]], 1)
    assert np.max(np.abs(x1 - x0)) < 1e-12


# ---- self-gravity potential --------------------------------------------------
def test_pair_potential_closed_forms_and_its_gradient_is_the_gravity():
    """-G m / r outside r_coll (softened: -G m / sqrt(r^2 + eps^2)); inside,
    the potential of the held gravity, continuous at r_coll; its negative
    derivative equals the gravity of Eq. (1) on either side (central
    differences), and coincident pairs contribute nothing."""
    kappa, eta = synth.contact_params(1e-3)
    for eps in (0.0, 1e-3):
        prm = orc.Params(G=2.0, eps=eps, r_coll=2e-5, kappa=0.0, eta=0.0)
        xi = np.zeros(3)
        for r in (1e-5, 1.9e-5, 3e-5, 0.7):
            xj = np.array([r, 0.0, 0.0])
            phi = orc.pair_potential(prm, xi, xj, 3e-12)
            if r > 2e-5:
                assert math.isclose(phi, -2.0 * 3e-12 / math.sqrt(r * r + eps * eps), rel_tol=1e-15)
            h = 1e-4 * r
            dphi = (orc.pair_potential(prm, xi, xj + [h, 0, 0], 3e-12) -
                    orc.pair_potential(prm, xi, xj - [h, 0, 0], 3e-12)) / (2 * h)
            # a_i = -grad_{x_i} phi = +d phi / d x_j along the axis
            a = orc.pair_accel(prm, xi, np.zeros(3), 1.0, xj, np.zeros(3), 3e-12)
            assert math.isclose(a[0], dphi, rel_tol=1e-6)
        rc = 2e-5
        below = orc.pair_potential(prm, xi, np.array([rc * (1 - 1e-12), 0, 0]), 3e-12)
        above = orc.pair_potential(prm, xi, np.array([rc * (1 + 1e-12), 0, 0]), 3e-12)
        assert math.isclose(below, above, rel_tol=1e-10)
        assert orc.pair_potential(prm, xi, xi, 3e-12) == 0.0
    del kappa, eta


def test_cell_potential_far_field_orders_and_gradient():
    """A cell's potential against the direct sum over its particles: the
    monopole error falls as (s/d)^2 (the dipole vanishes about the centre of
    mass), the quadrupole's as (s/d)^3; its negative gradient is orc_cell."""
    rng = np.random.default_rng(4)
    xs = rng.uniform(-0.5, 0.5, (40, 3)); ms = rng.uniform(0.5, 1.5, 40)
    M = ms.sum(); c = (ms[:, None] * xs).sum(0) / M
    d = xs - c; d2 = (d * d).sum(1)
    Q = np.array([(ms * (3 * d[:, 0] ** 2 - d2)).sum(), (ms * (3 * d[:, 1] ** 2 - d2)).sum(),
                  (ms * (3 * d[:, 2] ** 2 - d2)).sum(), (3 * ms * d[:, 0] * d[:, 1]).sum(),
                  (3 * ms * d[:, 0] * d[:, 2]).sum(), (3 * ms * d[:, 1] * d[:, 2]).sum()])
    u = np.array([0.6, -0.3, 0.74]); u /= np.linalg.norm(u)
    errs = {1: [], 2: []}
    for D in (8.0, 16.0, 32.0, 64.0):
        x = c + D * u
        exact = -(ms / np.linalg.norm(x - xs, axis=1)).sum()
        for order in (1, 2):
            errs[order].append(abs(orc.cell_potential(1.0, 0.0, order, x, M, c, Q) - exact) / abs(exact))
    for order, slope in ((1, 2.0), (2, 3.0)):
        e = np.array(errs[order])
        k = np.log2(e[:-1] / e[1:])
        assert np.all(np.abs(k - slope) < 0.35), (order, k)
    x = c + 5.0 * u
    h = 1e-5
    g = [(orc.cell_potential(1.0, 1e-2, 2, x + h * np.eye(3)[a], M, c, Q) -
          orc.cell_potential(1.0, 1e-2, 2, x - h * np.eye(3)[a], M, c, Q)) / (2 * h) for a in range(3)]
    acc = orc.cell_accel(1.0, 1e-2, 2, x, M, c, Q)
    assert np.allclose(acc, -np.array(g), rtol=1e-7, atol=0)


def test_tree_potential_theta_zero_equals_direct_bitwise():
    P = synth.ring(3000, 2, r_in=0.999, r_out=1.001, phi_max=0.01)
    prm = orc.Params(theta=0.0, n_g=32, n_leaf=4, order=2, r_coll=2e-5)
    S = orc.rebuild(P, prm)
    assert np.array_equal(orc.tree_potential(S, prm), orc.direct_potential(S.P, prm))


def test_tree_potential_at_theta_half_close_to_direct_and_energy_symmetric():
    """theta 0.5, quadrupole: per-particle potentials within 1e-4 of the
    direct sum; W = 1/2 sum m phi equals the sum over unordered pairs."""
    P = synth.uniform_cube(1500, 3)
    prm = orc.Params(theta=0.5, n_g=32, n_leaf=8, order=2, eps=1e-3)
    S = orc.rebuild(P, prm)
    pt, pd = orc.tree_potential(S, prm), orc.direct_potential(S.P, prm)
    assert np.max(np.abs(pt - pd) / np.abs(pd)) < 1e-4
    x = np.stack([S.P["x"], S.P["y"], S.P["z"]], 1); m = S.P["m"]
    W = 0.0
    for i in range(len(m)):
        r = np.sqrt(((x[i + 1:] - x[i]) ** 2).sum(1) + 1e-6)
        W -= (m[i] * m[i + 1:] / r).sum()
    assert math.isclose(orc.self_energy(m, pd), W, rel_tol=1e-12)


def test_step_conserves_total_energy_without_contacts():
    """A softened self-gravitating cube starting at rest (no central mass, no
    contacts, theta 0 so the forces are the potential's exact gradient):
    kick-drift-kick conserves kinetic + self-gravity energy to O(dt^2), so
    the total moves by far less than the kinetic energy gained."""
    P = synth.uniform_cube(300, 6)
    prm = orc.Params(theta=0.0, n_g=16, n_leaf=4, order=2, eps=0.05, G=1.0, dt=1e-3, rebuild_every=4)

    def parts(Q):
        return orc.diagnostics(Q, 1.0, 0.0)["kinetic"], orc.self_energy(Q["m"], orc.direct_potential(Q, prm))

    k0, w0 = parts(P)
    S, _, _ = orc.step(P, prm, 200)
    k1, w1 = parts(S.P)
    assert k0 == 0.0 and k1 > 1e-2 * abs(w0)
    assert abs((k1 + w1) - (k0 + w0)) < 1e-4 * k1


# ---- rotating frame (Sec. 4.4) -----------------------------------------------
def _one(x, y, vx, vy, m=1e-12):
    return {"x": np.array([x]), "y": np.array([y]), "z": np.array([0.0]), "vx": np.array([vx]),
            "vy": np.array([vy]), "vz": np.array([0.0]), "m": np.array([m]), "id": np.array([0], np.int64)}


def test_rotating_frame_circular_orbit_stands_still():
    """A particle on the circular orbit r = 1 about M_c = 1 in a frame turning
    at its Kepler rate 1 stays at (1, 0) up to the integrator's O(dt^2)
    phase error, while in the inertial frame it goes round."""
    nst = 500
    prm = orc.Params(G=1.0, M_central=1.0, dt=1e-2, rebuild_every=4, omega=1.0)
    S, _, _ = orc.step(_one(1.0, 0.0, 0.0, 1.0), prm, nst)
    drift = math.hypot(S.P["x"][0] - 1.0, S.P["y"][0])
    assert drift < nst * prm.dt ** 3 and abs(math.hypot(S.P["x"][0], S.P["y"][0]) - 1.0) < 2 * prm.dt ** 2
    Si, _, _ = orc.step(_one(1.0, 0.0, 0.0, 1.0), orc.Params(**{**prm.__dict__, "omega": 0.0}), nst)
    assert math.hypot(Si.P["x"][0] - 1.0, Si.P["y"][0]) > 1.0


def test_rotating_frame_jacobi_integral_of_a_test_particle():
    """An eccentric test particle about M_c in the frame turning at Omega:
    the Jacobi integral C = 1/2 |v - Omega x r|^2 - 1/2 Omega^2 (x^2 + y^2)
    - G M_c / r (v the inertial velocity in the turning axes) is conserved to
    O(dt^2); it moves far less than the particle's speed relative to the
    frame does."""
    prm = orc.Params(G=1.0, M_central=1.0, dt=1e-3, rebuild_every=4, omega=1.0)

    def jacobi(Q):
        x, y, vx, vy = Q["x"][0], Q["y"][0], Q["vx"][0], Q["vy"][0]
        ux, uy = vx + prm.omega * y, vy - prm.omega * x  # velocity relative to the frame
        return 0.5 * (ux * ux + uy * uy + Q["vz"][0] ** 2) - 0.5 * prm.omega ** 2 * (x * x + y * y) - \
            1.0 / math.hypot(x, y)

    P = _one(1.1, 0.0, 0.0, 0.85)
    c0 = jacobi(P)
    S, _, _ = orc.step(P, prm, 3000)
    rel_speed = math.hypot(S.P["vx"][0] + S.P["y"][0], S.P["vy"][0] - S.P["x"][0])
    assert abs(jacobi(S.P) - c0) < 1e-5 and rel_speed > 1e-2


def test_rotating_frame_equals_inertial_run_mapped_back():
    """theta = 0 (tree forces = direct sums): a ring patch stepped in the
    turning frame, mapped back by the angle the frame turned, is the
    inertial run to rounding (the forces are rotation-invariant)."""
    P = synth.ring(800, 14, r_in=0.999, r_out=1.001, phi_max=0.01, mass=1e-9)
    kappa, eta = synth.contact_params(1e-3)
    prm = orc.Params(theta=0.0, n_g=16, n_leaf=4, order=2, G=1.0, M_central=1.0, dt=1e-3, rebuild_every=4,
                     r_coll=2e-5, kappa=kappa, eta=eta, omega=1.0)
    nst = 12
    Sr, _, _ = orc.step(P, prm, nst)
    Si, _, _ = orc.step(P, orc.Params(**{**prm.__dict__, "omega": 0.0}), nst)
    back = orc.to_inertial(Sr.P, prm.omega * prm.dt * nst)
    o_r, o_i = np.argsort(Sr.P["id"]), np.argsort(Si.P["id"])
    for f in ("x", "y", "z"):
        assert np.max(np.abs(back[f][o_r] - Si.P[f][o_i])) < 1e-13, f
    for f in ("vx", "vy", "vz"):
        assert np.max(np.abs(back[f][o_r] - Si.P[f][o_i])) < 1e-11, f
    # in the turning frame the ring centre barely moves
    x0 = np.stack([P["x"], P["y"]], 1)[np.argsort(P["id"])]
    xr = np.stack([Sr.P["x"], Sr.P["y"]], 1)[o_r]
    xi = np.stack([Si.P["x"], Si.P["y"]], 1)[o_i]
    assert np.max(np.linalg.norm(xr - x0, axis=1)) < 0.05 * np.max(np.linalg.norm(xi - x0, axis=1))


# ---- diagnostics ------------------------------------------------------------
def test_diagnostics_circular_orbit_closed_form():
    """One particle of mass m on a circular orbit of radius R about M_c:
    K = m v^2 / 2 = G M_c m / (2R), W = -G M_c m / R, L = m R v along z."""
    R, m, GM = 1.3, 2e-3, 1.0
    v = np.sqrt(GM / R)
    P = {"x": np.array([R]), "y": np.array([0.0]), "z": np.array([0.0]), "vx": np.array([0.0]),
         "vy": np.array([v]), "vz": np.array([0.0]), "m": np.array([m])}
    d = orc.diagnostics(P, 1.0, GM)
    assert d["mass"] == m
    assert np.isclose(d["kinetic"], GM * m / (2 * R), rtol=1e-15)
    assert np.isclose(d["potential_central"], -GM * m / R, rtol=1e-15)
    assert np.allclose(d["angular_momentum"], [0.0, 0.0, m * R * v], rtol=1e-15, atol=0)
    assert np.allclose(d["momentum"], [0.0, m * v, 0.0], rtol=1e-15, atol=0)


def test_diagnostics_opposite_pair_and_virial():
    """Two equal masses with opposite velocities: zero momentum; for circular
    Kepler orbits 2K + W = 0."""
    R, GM = 0.9, 1.0
    v = np.sqrt(GM / R)
    P = {"x": np.array([R, -R]), "y": np.array([0.0, 0.0]), "z": np.array([0.0, 0.0]), "vx": np.array([0.0, 0.0]),
         "vy": np.array([v, -v]), "vz": np.array([0.0, 0.0]), "m": np.array([1.0, 1.0])}
    d = orc.diagnostics(P, 1.0, GM)
    assert np.array_equal(d["momentum"], np.zeros(3))
    assert np.isclose(2 * d["kinetic"] + d["potential_central"], 0.0, atol=1e-15)


def test_contact_pairs_brute_force_small():
    P = {"x": np.array([0.0, 1.5e-5, 3.5e-5, 1.0]), "y": np.zeros(4), "z": np.zeros(4)}
    assert orc.contact_pairs(P, 2e-5) == 2  # (0,1) at 1.5e-5 and (1,2) at 2e-5 apart


# ------------------------------------------------- cylindrical frame (Sec. 4.3) ----
def test_cyl_angle_against_atan2_and_special_angles():
    rng = np.random.default_rng(41)
    x = rng.normal(size=20000)
    y = rng.normal(size=20000)
    phi, r = orc.cyl_coords(x, y)
    ref = np.mod(np.arctan2(y, x), 2 * np.pi)
    # FP32 coordinates: x, y rounded to FP32, a few FP32 roundings of a value
    # below 2 pi (ulp 4.8e-7) and the series' truncation (3e-9)
    assert np.abs(phi - ref).max() < 1e-6
    assert np.all((phi >= 0) & (phi <= 2 * np.pi))
    assert np.allclose(r, np.hypot(x, y), rtol=3e-7, atol=0)
    # r is the correctly rounded FP32 root of the FP32 sum of squares
    xf, yf = x.astype(np.float32), y.astype(np.float32)
    assert np.array_equal(r, np.sqrt(xf * xf + yf * yf).astype(np.float64))
    # axes and diagonals
    xs = np.array([1.0, 0.0, -1.0, 0.0, 1.0, -1.0, -1.0, 1.0, 0.0])
    ys = np.array([0.0, 1.0, 0.0, -1.0, 1.0, 1.0, -1.0, -1.0, 0.0])
    phi, _ = orc.cyl_coords(xs, ys)
    want = np.array([0, 0.5, 1, 1.5, 0.25, 0.75, 1.25, 1.75, 0]) * np.pi
    assert np.abs(phi - want).max() < 1e-6
    assert phi[0] == 0.0 and phi[8] == 0.0  # the positive x axis and the origin


def test_cyl_angle_monotone_around_the_circle():
    t = np.sort(np.random.default_rng(42).uniform(0, 2 * np.pi, 200000))
    phi, _ = orc.cyl_coords(np.cos(t), np.sin(t))
    assert np.all(np.diff(phi) >= 0)


def _cyl_state(n, seed=7, **kw):
    P = synth.ring(n, seed)
    prm = orc.Params(**{**dict(theta=0.5, n_g=64, n_leaf=8, order=2, r_coll=2e-5, key_frame=1), **kw})
    return P, prm, orc.rebuild(P, prm)


def test_cyl_lists_brute_force_periodic_definition():
    """Same ancestor definition as the Cartesian case, with the opening test
    written out independently: phi gap the shorter way round a period of
    floor(2 pi S) cells, contact clause ((r_coll / r_min + 4e-6) S)^2 with
    r_min the smallest FP32 radius."""
    P, prm, S = _cyl_state(64, n_g=8, n_leaf=2, theta=0.7)
    t = S.tree
    nn = len(t["level"])
    Sg = 2097152.0 / S.L
    period = int(np.floor(2 * np.pi * Sg))
    xf, yf = S.P["x"].astype(np.float32), S.P["y"].astype(np.float32)
    rmin = float(np.sqrt(xf * xf + yf * yf).min())
    rc = (prm.r_coll / rmin + 4e-6) * Sg
    rcq2 = rc * rc

    def gap(lo_c, hi_c, lo_g, hi_g, periodic):
        if lo_c > hi_g:
            d = lo_c - hi_g - 1
            w = lo_g + period - hi_c - 1
        elif lo_g > hi_c:
            d = lo_g - hi_c - 1
            w = lo_c + period - hi_g - 1
        else:
            return 0
        return max(0, min(d, w)) if periodic else max(0, d)

    def opened(g, c):
        d2 = sum(gap(int(S.qlo[c][a]), int(S.qhi[c][a]), int(S.qlo[g][a]), int(S.qhi[g][a]), a == 0) ** 2
                 for a in range(3))
        s = 2.0 ** (21 - int(t["level"][c]))
        return prm.theta * prm.theta * float(d2) < s * s or float(d2) <= rcq2

    for k, g in enumerate(S.groups):
        Pset, Cset = [], []
        for c in range(nn):
            anc, a = [], t["parent"][c]
            while a >= 0:
                anc.append(a); a = t["parent"][a]
            if not all(opened(g, a) for a in anc):
                continue
            if opened(g, c):
                if t["nchild"][c] == 0:
                    Pset.append(c)
            else:
                Cset.append(c)
        L = S.lists
        key = lambda c: t["begin"][c]
        assert list(L["P"][L["pp_off"][k]:L["pp_off"][k + 1]]) == sorted(Pset, key=key)
        assert list(L["C"][L["pc_off"][k]:L["pc_off"][k + 1]]) == sorted(Cset, key=key)


def test_cyl_contacts_always_particles_and_seam_neighbours_near():
    """Every particle within r_coll of a group particle is in the group's
    particle list, including pairs across the phi = 0 / 2 pi seam."""
    n = 3000
    rng = np.random.default_rng(43)
    phi = np.concatenate([rng.uniform(0, 3e-3, n // 2), rng.uniform(2 * np.pi - 3e-3, 2 * np.pi, n - n // 2)])
    r = rng.uniform(0.9995, 1.0005, n)
    P = {"x": r * np.cos(phi), "y": r * np.sin(phi), "z": rng.normal(0, 1e-5, n), "vx": np.zeros(n),
         "vy": np.zeros(n), "vz": np.zeros(n), "m": np.full(n, 1e-12), "id": np.arange(n)}
    prm = orc.Params(theta=0.6, n_g=32, n_leaf=4, order=2, r_coll=5e-5, key_frame=1)
    S = orc.rebuild(P, prm)
    X = np.stack([S.P["x"], S.P["y"], S.P["z"]], 1)
    t = S.tree
    across = 0
    for k in range(len(S.groups)):
        g = S.groups[k]; gb, ge = t["begin"][g], t["end"][g]
        inP = np.zeros(n, bool)
        for b, e, kind, c in _ranges(S, k):
            if kind == "P":
                inP[b:e] = True
        d = np.sqrt(((X[gb:ge, None, :] - X[None, :, :]) ** 2).sum(-1)).min(0)
        assert np.all(inP[d <= prm.r_coll])
        ph = np.mod(np.arctan2(X[:, 1], X[:, 0]), 2 * np.pi)
        if ph[gb:ge].max() < 1.0:
            across += int(np.sum((d <= prm.r_coll) & (ph > np.pi)))
    assert across > 0  # the case tested really has contact pairs across the seam


def test_cyl_theta_zero_tree_force_equals_direct_sum():
    P, prm, S = _cyl_state(600, theta=0.0, n_g=32, r_coll=0.0, order=1)
    a = orc.tree_forces(S, prm)
    d = orc.direct(S.P, prm)
    assert np.array_equal(a, d)
