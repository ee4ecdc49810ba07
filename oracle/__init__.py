"""CPU FP64 oracle for the group-shared Barnes-Hut force evaluation
(Iwasawa et al., arXiv:1907.02289).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg and reference arm may import this package.  It shares no code with the CUDA
library and never imports it; the only thing both sides use is the seeded input
generator, which holds none of the method's arithmetic.

The arithmetic lives in ``bh_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``).  This module compiles it, wraps each function with
numpy buffers and composes them into the build / list / force / step sequence
of Sec. 4.2 (list-constructing and list-reusing steps).

Parity unpinned: kappa and eta (the paper prints only the radial restitution
coefficient 0.5) and the tree-force accuracy at theta > 0 (the paper prints no
force error).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bh_oracle.c")
_LIB = os.path.join(_HERE, "libbh_oracle.so")
_lib = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile bh_oracle.c into libbh_oracle.so (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.orc_tree_count.restype = _i64
        _lib.orc_tree.restype = _i64
        _lib.orc_groups.restype = _i64
        _lib.orc_root_box.restype = _int
        _lib.orc_pair_potential.restype = _dbl
        _lib.orc_cell_potential.restype = _dbl
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_ptr)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
@dataclass
class Params:
    """Method parameters (symbols as in the paper where it has them)."""
    theta: float = 0.5
    n_g: int = 64
    n_leaf: int = 8
    eps: float = 0.0
    order: int = 1
    G: float = 1.0
    M_central: float = 0.0
    r_coll: float = 0.0
    kappa: float = 0.0
    eta: float = 0.0
    dt: float = 1e-3
    rebuild_every: int = 4
    key_frame: int = 0          # 0 Cartesian, 1 cylindrical (phi, r, z) tree (Sec. 4.3)
    omega: float = 0.0          # rotation rate of the coordinate frame (Sec. 4.4); 0 = inertial


# --------------------------------------------------------------------------
# Steps of the path, one function each
# --------------------------------------------------------------------------
def root_box(x, y, z):
    lo = np.zeros(3)
    L = np.zeros(1)
    rc = lib().orc_root_box(_i64(len(x)), _p(x), _p(y), _p(z), _p(lo), _p(L))
    if rc != 0:
        raise ValueError("non-finite particle coordinate")
    return lo, float(L[0])


def keys(x, y, z, lo, L):
    k = np.empty(len(x), dtype=np.uint64)
    lib().orc_keys(_i64(len(x)), _p(x), _p(y), _p(z), _p(np.ascontiguousarray(lo, dtype=np.float64)), _dbl(L), _p(k))
    return k


def key_coords(k):
    q = np.empty((len(k), 3), dtype=np.uint32)
    lib().orc_key_coords(_i64(len(k)), _p(k), _p(q))
    return q


def sort_perm(k):
    """Stable sort by key (ties keep input order).  numpy's stable argsort is
    used as the library primitive; orc_sort (qsort on (key, index)) is the
    plain-C statement of the same definition and is pinned equal to it."""
    return np.argsort(k, kind="stable").astype(np.uint32)


def sort_perm_c(k):
    perm = np.empty(len(k), dtype=np.uint32)
    lib().orc_sort(_i64(len(k)), _p(k), _p(perm))
    return perm


def build_tree(skeys, n_leaf):
    n = len(skeys)
    cnt = lib().orc_tree_count(_i64(n), _p(skeys), _int(n_leaf))
    t = {
        "level": np.empty(cnt, np.uint8),
        "begin": np.empty(cnt, np.uint32),
        "end": np.empty(cnt, np.uint32),
        "parent": np.empty(cnt, np.int32),
        "first_child": np.empty(cnt, np.int32),
        "nchild": np.empty(cnt, np.uint8),
    }
    got = lib().orc_tree(_i64(n), _p(skeys), _int(n_leaf), _i64(cnt), _p(t["level"]), _p(t["begin"]),
                         _p(t["end"]), _p(t["parent"]), _p(t["first_child"]), _p(t["nchild"]))
    assert got == cnt, (got, cnt)
    return t


def qboxes(tree, q):
    nn = len(tree["level"])
    qlo = np.empty((nn, 3), np.uint32)
    qhi = np.empty((nn, 3), np.uint32)
    lib().orc_qboxes(_i64(nn), _p(tree["begin"]), _p(tree["end"]), _p(tree["first_child"]),
                     _p(tree["nchild"]), _p(np.ascontiguousarray(q)), _p(qlo), _p(qhi))
    return qlo, qhi


def moments(tree, x, y, z, m, order):
    nn = len(tree["level"])
    M = np.empty(nn)
    cx, cy, cz = np.empty(nn), np.empty(nn), np.empty(nn)
    Q = np.empty((nn, 6))
    lib().orc_moments(_i64(nn), _p(tree["begin"]), _p(tree["end"]), _p(tree["first_child"]),
                      _p(tree["nchild"]), _p(x), _p(y), _p(z), _p(m), _int(order), _p(M), _p(cx),
                      _p(cy), _p(cz), _p(Q))
    return {"M": M, "cx": cx, "cy": cy, "cz": cz, "Q": Q}


def groups(tree, n_g):
    nn = len(tree["level"])
    g = np.empty(max(nn, 1), np.int32)
    ng = lib().orc_groups(_i64(nn), _p(tree["begin"]), _p(tree["end"]), _p(tree["parent"]),
                          _p(tree["nchild"]), _int(n_g), _p(g))
    return g[:ng].copy()


def lists(tree, qlo, qhi, grp, theta, r_coll, L):
    """Cartesian frame: contact threshold (r_coll S)^2 on the grid."""
    S = 2097152.0 / L
    rcq = r_coll * S
    return lists_ex(tree, qlo, qhi, grp, theta, rcq * rcq, 0)


def cyl_geometry(r_coll, r_min, L):
    """Cylindrical frame: (contact threshold on the grid, phi period in cells)."""
    rcq2 = np.zeros(1)
    period = np.zeros(1, np.int64)
    lib().orc_cyl_geometry(_dbl(r_coll), _dbl(r_min), _dbl(L), _p(rcq2), _p(period))
    return float(rcq2[0]), int(period[0])


def cyl_coords(x, y):
    """(phi, r) of every particle (Sec. 4.3 tree coordinates)."""
    n = len(x)
    phi = np.empty(n)
    r = np.empty(n)
    lib().orc_cyl(_i64(n), _p(np.ascontiguousarray(x, dtype=np.float64)),
                  _p(np.ascontiguousarray(y, dtype=np.float64)), _p(phi), _p(r))
    return phi, r


def lists_ex(tree, qlo, qhi, grp, theta, rcq2, period):
    ng = len(grp)
    pp_off = np.zeros(ng + 1, np.int64)
    pc_off = np.zeros(ng + 1, np.int64)
    args = [_i64(ng), _p(grp), _p(tree["level"]), _p(tree["first_child"]), _p(tree["nchild"]),
            _p(qlo), _p(qhi), _dbl(theta), _dbl(rcq2), _i64(period)]
    lib().orc_lists_ex(*args, _p(pp_off), None, _p(pc_off), None)
    P = np.empty(max(int(pp_off[-1]), 1), np.int32)
    C = np.empty(max(int(pc_off[-1]), 1), np.int32)
    lib().orc_lists_ex(*args, _p(pp_off), _p(P), _p(pc_off), _p(C))
    return {"pp_off": pp_off, "P": P[: pp_off[-1]].copy(), "pc_off": pc_off, "C": C[: pc_off[-1]].copy()}


def pair_accel(prm: Params, xi, vi, mi, xj, vj, mj):
    a = np.zeros(3)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    lib().orc_pair_accel(_dbl(prm.G), _dbl(prm.eps), _dbl(prm.r_coll), _dbl(prm.kappa), _dbl(prm.eta),
                         _p(f(xi)), _p(f(vi)), _dbl(mi), _p(f(xj)), _p(f(vj)), _dbl(mj), _p(a))
    return a


def cell_accel(G, eps, order, xi, M, c, Q):
    a = np.zeros(3)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    lib().orc_cell_accel(_dbl(G), _dbl(eps), _int(order), _p(f(xi)), _dbl(M), _p(f(c)), _p(f(Q)), _p(a))
    return a


def direct(P: dict, prm: Params):
    n = len(P["x"])
    ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
    lib().orc_direct(_i64(n), _p(P["x"]), _p(P["y"]), _p(P["z"]), _p(P["vx"]), _p(P["vy"]), _p(P["vz"]),
                     _p(P["m"]), _dbl(prm.G), _dbl(prm.eps), _dbl(prm.r_coll), _dbl(prm.kappa),
                     _dbl(prm.eta), _p(ax), _p(ay), _p(az))
    return np.stack([ax, ay, az], axis=1)


def central(x, y, z, G, Mc):
    n = len(x)
    ax, ay, az = np.empty(n), np.empty(n), np.empty(n)
    lib().orc_central(_i64(n), _p(x), _p(y), _p(z), _dbl(G), _dbl(Mc), _p(ax), _p(ay), _p(az))
    return np.stack([ax, ay, az], axis=1)


def pair_potential(prm: Params, xi, xj, mj) -> float:
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_pair_potential(_dbl(prm.G), _dbl(prm.eps), _dbl(prm.r_coll), _p(f(xi)), _p(f(xj)),
                                          _dbl(mj)))


def cell_potential(G, eps, order, xi, M, c, Q) -> float:
    f = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_cell_potential(_dbl(G), _dbl(eps), _int(order), _p(f(xi)), _dbl(M), _p(f(c)), _p(f(Q))))


def direct_potential(P: dict, prm: Params) -> np.ndarray:
    """phi_i = sum over j != i of the pair potential (direct summation)."""
    n = len(P["x"])
    phi = np.empty(n)
    lib().orc_direct_potential(_i64(n), _p(P["x"]), _p(P["y"]), _p(P["z"]), _p(P["m"]), _dbl(prm.G),
                               _dbl(prm.eps), _dbl(prm.r_coll), _p(phi))
    return phi


def tree_potential(S: "State", prm: Params) -> np.ndarray:
    """Per-particle self-gravity potential over the lists of S (the same
    leaves, cells and order as tree_forces)."""
    n = len(S.P["x"])
    phi = np.full(n, np.nan)
    t, L, mo, P = S.tree, S.lists, S.mom, S.P
    lib().orc_tree_potential(_i64(0), _i64(len(S.groups)), _p(S.groups), _p(t["begin"]), _p(t["end"]),
                             _p(L["pp_off"]), _p(L["P"] if len(L["P"]) else np.zeros(1, np.int32)), _p(L["pc_off"]),
                             _p(L["C"] if len(L["C"]) else np.zeros(1, np.int32)), _p(mo["M"]), _p(mo["cx"]),
                             _p(mo["cy"]), _p(mo["cz"]), _p(mo["Q"]), _int(prm.order), _p(P["x"]), _p(P["y"]),
                             _p(P["z"]), _p(P["m"]), _dbl(prm.G), _dbl(prm.eps), _dbl(prm.r_coll), _p(phi))
    return phi


def self_energy(m, phi) -> float:
    """Self-gravity potential energy W = 1/2 sum m_i phi_i."""
    return float(0.5 * np.sum(m * phi))


def tree_forces(S: "State", prm: Params, k0: int = 0, k1: int | None = None, out=None):
    """Tree acceleration (tree part only, no central mass) for groups [k0, k1).
    Entries of particles outside those groups are left as in ``out`` (NaN)."""
    ng = len(S.groups)
    k1 = ng if k1 is None else k1
    n = len(S.P["x"])
    if out is None:
        out = np.full((3, n), np.nan)
    ax, ay, az = out[0], out[1], out[2]
    t, L, mo, P = S.tree, S.lists, S.mom, S.P
    lib().orc_tree_forces(_i64(k0), _i64(k1), _p(S.groups), _p(t["begin"]), _p(t["end"]), _p(L["pp_off"]),
                          _p(L["P"] if len(L["P"]) else np.zeros(1, np.int32)), _p(L["pc_off"]),
                          _p(L["C"] if len(L["C"]) else np.zeros(1, np.int32)), _p(mo["M"]), _p(mo["cx"]),
                          _p(mo["cy"]), _p(mo["cz"]), _p(mo["Q"]), _int(prm.order), _p(P["x"]), _p(P["y"]),
                          _p(P["z"]), _p(P["vx"]), _p(P["vy"]), _p(P["vz"]), _p(P["m"]), _dbl(prm.G),
                          _dbl(prm.eps), _dbl(prm.r_coll), _dbl(prm.kappa), _dbl(prm.eta), _p(ax), _p(ay),
                          _p(az))
    return out.T


# --------------------------------------------------------------------------
# Composition: list-constructing step (keys .. lists) and list-reusing step
# --------------------------------------------------------------------------
FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "id")


@dataclass
class State:
    P: dict                     # particle arrays in current (sorted) order
    lo: np.ndarray = None
    L: float = 1.0
    skeys: np.ndarray = None    # sorted keys
    perm: np.ndarray = None     # sorted rank -> index before the sort
    tree: dict = None
    qlo: np.ndarray = None
    qhi: np.ndarray = None
    mom: dict = None
    groups: np.ndarray = None
    lists: dict = None
    extra: dict = field(default_factory=dict)


def rebuild(P: dict, prm: Params, group_subset=None) -> State:
    """List-constructing step (Sec. 4.2, steps 3a-3d): keys, sort, permute,
    octree, boxes, moments, groups and interaction lists.  group_subset
    (optional) maps the array of all groups to the indices of the groups to
    keep: lists (and tree forces) are then made for those groups only, for
    checking a sample of a workload too large to walk whole."""
    x, y, z = P["x"], P["y"], P["z"]
    if prm.key_frame == 1:  # Sec. 4.3: tree in (phi, r, z)
        x, y = cyl_coords(x, y)
    lo, L = root_box(x, y, z)
    k = keys(x, y, z, lo, L)
    perm = sort_perm(k)
    SP = {f: np.ascontiguousarray(P[f][perm]) for f in P}
    sk = np.ascontiguousarray(k[perm])
    tree = build_tree(sk, prm.n_leaf)
    qlo, qhi = qboxes(tree, key_coords(sk))
    mom = moments(tree, SP["x"], SP["y"], SP["z"], SP["m"], prm.order)
    grp = groups(tree, prm.n_g)
    if group_subset is not None:
        grp = np.ascontiguousarray(grp[group_subset(grp, tree)])
    if prm.key_frame == 1:
        if not lo[1] > 0.0:
            raise ValueError("the cylindrical key frame needs every particle off the axis (r > 0)")
        rcq2, period = cyl_geometry(prm.r_coll, lo[1], L)
        lst = lists_ex(tree, qlo, qhi, grp, prm.theta, rcq2, period)
    else:
        lst = lists(tree, qlo, qhi, grp, prm.theta, prm.r_coll, L)
    return State(P=SP, lo=lo, L=L, skeys=sk, perm=perm, tree=tree, qlo=qlo, qhi=qhi, mom=mom,
                 groups=grp, lists=lst)


def refresh(S: State, prm: Params) -> None:
    """List-reusing step (Sec. 4.2): same order, tree topology, groups and
    lists; only the node moments are recomputed from current positions."""
    P = S.P
    S.mom = moments(S.tree, P["x"], P["y"], P["z"], P["m"], prm.order)


def accel(S: State, prm: Params) -> np.ndarray:
    """Total acceleration: tree part plus the central mass."""
    a = tree_forces(S, prm)
    if prm.M_central != 0.0:
        a = a + central(S.P["x"], S.P["y"], S.P["z"], prm.G, prm.M_central)
    return a


def rotate_frame(Q: dict, omega_dt: float) -> None:
    """The coordinate frame turns by omega dt about the z axis (Sec. 4.4):
    positions and velocities, expressed in the frame, rotate by -omega dt."""
    c, s = math.cos(omega_dt), math.sin(omega_dt)
    x, y, vx, vy = Q["x"], Q["y"], Q["vx"], Q["vy"]
    Q["x"], Q["y"] = c * x + s * y, c * y - s * x
    Q["vx"], Q["vy"] = c * vx + s * vy, c * vy - s * vx


def to_inertial(Q: dict, angle: float) -> dict:
    """Arrays of a frame that has turned by angle, expressed in the inertial
    axes (the rotation undone)."""
    c, s = math.cos(angle), math.sin(angle)
    out = dict(Q)
    out["x"], out["y"] = c * Q["x"] - s * Q["y"], s * Q["x"] + c * Q["y"]
    out["vx"], out["vy"] = c * Q["vx"] - s * Q["vy"], s * Q["vx"] + c * Q["vy"]
    return out


def step(P: dict, prm: Params, nsteps: int):
    """Kick-drift-kick leapfrog with the persistent-list schedule of Sec. 4.2.
    Force evaluation k (k = 0 initial) rebuilds iff k % rebuild_every == 0,
    otherwise refreshes moments only.  The contact term at evaluation k+1 sees
    the half-step velocity.  With prm.omega != 0 the arrays live in a frame
    turning at omega (Sec. 4.4): after every drift the frame turns by
    omega dt.  Returns (final State, acceleration, #evaluations)."""
    dt = prm.dt
    S = rebuild({f: np.array(P[f]) for f in FIELDS}, prm)
    a = accel(S, prm)
    k = 1
    for _ in range(nsteps):
        Q = S.P
        for c in "xyz":
            Q["v" + c] = Q["v" + c] + (0.5 * dt) * a[:, "xyz".index(c)]
        for c in "xyz":
            Q[c] = Q[c] + dt * Q["v" + c]
        if prm.omega != 0.0:
            rotate_frame(Q, prm.omega * dt)
        if k % prm.rebuild_every == 0:
            S = rebuild(Q, prm)
        else:
            refresh(S, prm)
        a = accel(S, prm)
        Q = S.P
        for c in "xyz":
            Q["v" + c] = Q["v" + c] + (0.5 * dt) * a[:, "xyz".index(c)]
        k += 1
    return S, a, k

# --------------------------------------------------------------------------
# Diagnostics: the plain definitions of the conserved sums
# --------------------------------------------------------------------------
def diagnostics(P: dict, G: float, M_central: float) -> dict:
    """Mass, momentum sum m v, angular momentum sum m x cross v (about the
    origin), kinetic energy sum m |v|^2 / 2 and central-mass potential energy
    -sum G M_c m / |x|, in FP64 (numpy sums)."""
    m = P["m"]
    x = np.stack([P["x"], P["y"], P["z"]], 1)
    v = np.stack([P["vx"], P["vy"], P["vz"]], 1)
    r = np.linalg.norm(x, axis=1)
    return {"mass": float(m.sum()), "momentum": (m[:, None] * v).sum(0),
            "angular_momentum": (m[:, None] * np.cross(x, v)).sum(0),
            "kinetic": float(0.5 * (m * (v * v).sum(1)).sum()),
            "potential_central": float(np.where(r > 0, -G * M_central * m / np.where(r > 0, r, 1.0), 0.0).sum())}


def contact_pairs(P: dict, r_coll: float) -> int:
    """Unordered pairs with 0 < r <= r_coll, by brute force over all pairs."""
    x = np.stack([P["x"], P["y"], P["z"]], 1)
    n, cnt = len(x), 0
    for i0 in range(0, n, 1024):
        d = x[i0:i0 + 1024, None, :] - x[None, :, :]
        r2 = (d * d).sum(2)
        ii = np.arange(i0, min(n, i0 + 1024))[:, None]
        jj = np.arange(n)[None, :]
        cnt += int(((r2 > 0) & (r2 <= r_coll * r_coll) & (jj > ii)).sum())
    return cnt
