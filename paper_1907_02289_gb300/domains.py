"""Domain decomposition of one ring across ranks with the two-level tree of
domains (Sec. 4.5), in phi sectors (Sec. 4.3).

Every rank holds the particles of one contiguous range of tree nodes at a
split level l_d.  In the cylindrical key frame the first levels of the tree
divide phi only (the ring is 2 pi wide in phi, a few hundredths in r and
z), so the ranges are phi sectors.  The exchange reproduces the tree one rank
alone would build:

1. the root box is the exact all-reduced min/max, so every rank keys its
   particles on the same grid, and particles move to the rank owning their
   node at level l_d (ranges chosen from the all-reduced node counts);
2. each rank builds the subtrees below its level-l_d nodes, which are the
   single tree's own subtrees (a node splits on its own particles only);
3. all level-l_d nodes (box, count, moments) are all-gathered -- the
   paper's exchange of top-level centres of mass -- so every rank knows the
   top of the tree;
4. each rank walks its subtrees against every other rank's domain box with
   the group walk's own opening test and sends what the walk visited: the
   opened inner nodes (structure), the accepted nodes (moments) and the
   particles of the opened leaves (the halo that contact needs included).
   A group box lies inside its domain box, so a group opens at most what
   its domain opens: the receiver has every node any of its groups visits;
5. each rank assembles that view of the tree (nodes numbered breadth first,
   level by level in key order, like the single tree), computes the moments
   of the inner nodes from their children, and walks and evaluates its own
   groups on it.

The ranks exchange through torch.distributed (gloo on CPU ranks, NCCL on
GPUs).  The arithmetic of the path -- keys, trees, moments, walks, forces --
is the compute backend's, passed in (see ``Backend``); this module holds the
decomposition, the exchanges and the assembly of the view.
"""
from __future__ import annotations

import pickle
from dataclasses import dataclass

import numpy as np

LEVELS = 21
FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "id")


@dataclass
class Backend:
    """The path's arithmetic for one rank (the CUDA library's kernels on a GPU
    rank; the tests pass the CPU oracle's).

    tree_coords(P) -> (a0, a1, a2): coordinates of the key frame
    keys(a0, a1, a2, lo, L) -> uint64 keys on the grid of that root box
    key_coords(keys) -> [n, 3] uint32 grid coordinates
    build_tree(sorted_keys, n_leaf) -> tree dict (level, begin, end, parent,
        first_child, nchild) of a key-sorted set, breadth first
    moments(tree, x, y, z, m, order) -> dict M, cx, cy, cz, Q[n, 6]
    combine(tree, mom, frozen, V, order) -> moments of a view: leaves from
        the particles V, frozen nodes as given in mom, inner nodes from their
        children
    walk(tree, qlo, qhi, groups, theta, rcq2, period) -> lists dict
        (pp_off, P, pc_off, C): the group walk's lists
    contact_geometry(lo, L) -> (rcq2, period) of the opening test
    forces(tree, lists, groups, mom, V) -> [n, 3] tree accelerations of the
        groups' particles
    """
    tree_coords: object
    keys: object
    key_coords: object
    build_tree: object
    moments: object
    combine: object
    walk: object
    contact_geometry: object
    forces: object


# --------------------------------------------------------------------------
# collectives (torch.distributed; tensors on the device the backend wants)
# --------------------------------------------------------------------------
def _allreduce(v: np.ndarray, op: str):
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(v))
    dist.all_reduce(t, op={"min": dist.ReduceOp.MIN, "max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return t.numpy()


def _exchange(payloads: list) -> list:
    """payloads[r] goes to rank r; returns what every rank sent to this one
    (pickled, sizes exchanged first, paired non-blocking sends/receives)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(), dist.get_world_size()
    blobs = [np.frombuffer(pickle.dumps(p, protocol=4), dtype=np.uint8) for p in payloads]
    sizes = torch.tensor([len(b) for b in blobs], dtype=torch.int64)
    all_sizes = [torch.zeros(world, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_sizes, sizes)
    reqs, inbox = [], [None] * world
    for k in range(1, world):
        dst, src = (rank + k) % world, (rank - k) % world
        reqs.append(dist.isend(torch.from_numpy(blobs[dst].copy()), dst))
        buf = torch.empty(int(all_sizes[src][rank]), dtype=torch.uint8)
        reqs.append(dist.irecv(buf, src))
        inbox[src] = buf
    for q in reqs:
        q.wait()
    out = []
    for r in range(world):
        out.append(payloads[rank] if r == rank else pickle.loads(inbox[r].numpy().tobytes()))
    return out


def _allgather(obj) -> list:
    import torch.distributed as dist
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


# --------------------------------------------------------------------------
# decomposition
# --------------------------------------------------------------------------
def owner_ranges(counts: np.ndarray, world: int) -> np.ndarray:
    """Contiguous ranges of level-l_d nodes (in key order) with about equal
    particle counts: rank r owns prefixes [cut[r], cut[r+1])."""
    csum = np.concatenate([[0], np.cumsum(counts)])
    total = csum[-1]
    cut = np.searchsorted(csum, [total * r / world for r in range(world + 1)], side="left")
    cut[0], cut[-1] = 0, len(counts)
    return np.maximum.accumulate(cut)


def check_split_level(counts: np.ndarray, split_level: int, n_leaf: int, n_g: int) -> None:
    """The single tree has every level-l_d node of the decomposition only if
    each of their ancestors splits (more than n_leaf particles), and every
    group lies inside one rank's subtrees only if the level l_d - 1 nodes hold
    more than n_g particles."""
    c = counts.astype(np.int64)
    for lev in range(split_level - 1, -1, -1):
        c = c.reshape(-1, 8).sum(1)
        live = c[c > 0]
        if (live <= max(n_leaf, n_g)).any():
            raise ValueError(f"split level {split_level}: a level-{lev} node holds <= max(n_leaf, n_g) particles; "
                             "take a lower split level")


def _prefix(keys: np.ndarray, level: int) -> np.ndarray:
    return (keys >> np.uint64(3 * (LEVELS - level))).astype(np.uint64)


def _link(level: np.ndarray, prefix: np.ndarray):
    """parent / first_child / nchild of nodes sorted breadth first by
    (level, prefix); a node's parent is the present node of the nearest
    lower level whose prefix covers it (-1 for the first level present)."""
    n = len(level)
    parent = np.full(n, -1, np.int32)
    first_child = np.full(n, -1, np.int32)
    nchild = np.zeros(n, np.uint8)
    index = {(int(level[k]), int(prefix[k])): k for k in range(n)}
    levels = sorted(set(int(v) for v in level))
    for k in range(n):
        lv, p = int(level[k]), int(prefix[k])
        for up in reversed([v for v in levels if v < lv]):
            q = index.get((up, p >> (3 * (lv - up))))
            if q is not None:
                parent[k] = q
                break
    for k in range(n):
        q = parent[k]
        if q >= 0:
            if first_child[q] < 0:
                first_child[q] = k
            nchild[q] += 1
    return parent, first_child, nchild


def _ranges(sorted_keys: np.ndarray, level: np.ndarray, prefix: np.ndarray):
    """[begin, end) of each node's particles in a key-sorted array (empty
    where the node has none there)."""
    begin = np.empty(len(level), np.uint32)
    end = np.empty(len(level), np.uint32)
    for lv in np.unique(level):
        sel = np.nonzero(level == lv)[0]
        pk = _prefix(sorted_keys, int(lv))
        begin[sel] = np.searchsorted(pk, prefix[sel], side="left")
        end[sel] = np.searchsorted(pk, prefix[sel], side="right")
    return begin, end


def _subtrees(backend: Backend, sk: np.ndarray, split_level: int, n_leaf: int):
    """Nodes (level, prefix) of the single tree below the level-l_d nodes of
    the key-sorted set sk (all of whose particles are here)."""
    levels, prefixes = [], []
    pre = _prefix(sk, split_level)
    starts = np.concatenate([[0], np.nonzero(np.diff(pre))[0] + 1, [len(sk)]])
    for b, e in zip(starts[:-1], starts[1:]):
        if e - b <= n_leaf:  # a leaf of the single tree
            levels.append(np.array([split_level], np.uint8))
            prefixes.append(np.array([pre[b]], np.uint64))
            continue
        t = backend.build_tree(np.ascontiguousarray(sk[b:e]), n_leaf)
        keep = t["level"] >= split_level  # the chain above is the top of the tree
        lv = t["level"][keep]
        levels.append(lv)
        prefixes.append(np.array([int(sk[b + int(t["begin"][k])]) >> (3 * (LEVELS - int(t["level"][k])))
                                  for k in np.nonzero(keep)[0]], np.uint64))
    level = np.concatenate(levels) if levels else np.zeros(0, np.uint8)
    prefix = np.concatenate(prefixes) if prefixes else np.zeros(0, np.uint64)
    o = np.lexsort((prefix, level))
    return level[o], prefix[o]


def _boxes(qc: np.ndarray, begin: np.ndarray, end: np.ndarray):
    """Integer tight boxes of the nodes with particles here (min / max of the
    grid coordinates over [begin, end))."""
    qlo = np.zeros((len(begin), 3), np.uint32)
    qhi = np.zeros((len(begin), 3), np.uint32)
    for k in range(len(begin)):
        if end[k] > begin[k]:
            qlo[k] = qc[begin[k]:end[k]].min(0)
            qhi[k] = qc[begin[k]:end[k]].max(0)
    return qlo, qhi


def _tree(level, prefix, begin, end, fake_root: bool):
    """Tree arrays for the backend; with fake_root a node 0 whose children are
    the first level present and whose box covers everything (always opened)."""
    if fake_root:
        level = np.concatenate([[0], level]).astype(np.uint8)
        prefix = np.concatenate([[0], prefix]).astype(np.uint64)
        begin = np.concatenate([[begin.min() if len(begin) else 0], begin]).astype(np.uint32)
        end = np.concatenate([[end.max() if len(end) else 0], end]).astype(np.uint32)
        parent, first_child, nchild = _link(level[1:], prefix[1:])
        parent = np.where(parent >= 0, parent + 1, 0).astype(np.int32)
        first_child = np.where(first_child >= 0, first_child + 1, -1).astype(np.int32)
        roots = np.nonzero(parent == 0)[0] + 1
        parent = np.concatenate([[-1], parent]).astype(np.int32)
        first_child = np.concatenate([[roots.min() if len(roots) else -1], first_child]).astype(np.int32)
        nchild = np.concatenate([[len(roots)], nchild]).astype(np.uint8) if len(roots) < 256 else None
        if nchild is None:
            raise ValueError("more than 255 subtrees on one rank: take a lower split level")
    else:
        parent, first_child, nchild = _link(level, prefix)
    return {"level": np.asarray(level, np.uint8), "prefix": np.asarray(prefix, np.uint64),
            "begin": np.asarray(begin, np.uint32), "end": np.asarray(end, np.uint32), "parent": parent,
            "first_child": first_child, "nchild": nchild}


def decomposed_forces(P: dict, prm: dict, backend: Backend, split_level: int):
    """Tree accelerations (tree part) of the particles this rank owns after
    the decomposition, from the exchanged view of the single tree.

    P holds this rank's share of the particles (any share; together the
    ranks hold the set once, rank r's in the set's order after rank r-1's).
    Returns (owned particles in key order, their accelerations [n, 3], info).
    """
    import torch.distributed as dist
    rank, world = dist.get_rank(), dist.get_world_size()
    n_leaf, n_g, order = int(prm["n_leaf"]), int(prm["n_g"]), int(prm.get("order", 1))

    # 1. the common grid and the owners
    a = backend.tree_coords(P)
    have = len(P["x"]) > 0
    mn = _allreduce(np.array([c.min() if have else np.inf for c in a]), "min")
    mx = _allreduce(np.array([c.max() if have else -np.inf for c in a]), "max")
    lo = mn.astype(np.float64)
    ext = float((mx - mn).max())
    L = ext if ext > 0.0 else 1.0
    keys = backend.keys(*a, lo, L)
    nb = 8 ** split_level
    counts = _allreduce(np.bincount(_prefix(keys, split_level).astype(np.int64), minlength=nb).astype(np.int64),
                        "sum")
    check_split_level(counts, split_level, n_leaf, n_g)
    cut = owner_ranges(counts, world)
    owner = np.searchsorted(cut, _prefix(keys, split_level).astype(np.int64), side="right") - 1
    recv = _exchange([{f: P[f][owner == r] for f in FIELDS} for r in range(world)])
    Q = {f: np.concatenate([x[f] for x in recv]) for f in FIELDS}

    # 2. own particles in key order and the single tree's subtrees over them
    qa = backend.tree_coords(Q)
    k = backend.keys(*qa, lo, L)
    o = np.argsort(k, kind="stable")
    Q = {f: np.ascontiguousarray(Q[f][o]) for f in FIELDS}
    sk = np.ascontiguousarray(k[o])
    qc = backend.key_coords(sk)
    lv, pf = _subtrees(backend, sk, split_level, n_leaf)
    b, e = _ranges(sk, lv, pf)
    own = _tree(lv, pf, b, e, fake_root=True)
    own["qlo"], own["qhi"] = _boxes(qc, own["begin"], own["end"])
    mom = backend.moments(own, Q["x"], Q["y"], Q["z"], Q["m"], order)

    # 3. every level-l_d node, all-gathered (box, count and moments)
    top = np.nonzero(own["level"][1:] == split_level)[0] + 1
    mine = {"prefix": own["prefix"][top], "qlo": own["qlo"][top], "qhi": own["qhi"][top],
            "count": (own["end"][top] - own["begin"][top]).astype(np.int64),
            "M": mom["M"][top], "c": np.stack([mom["cx"][top], mom["cy"][top], mom["cz"][top]], 1), "Q": mom["Q"][top]}
    tops = _allgather(mine)
    dom_lo = [t["qlo"].min(0) if len(t["prefix"]) else None for t in tops]
    dom_hi = [t["qhi"].max(0) if len(t["prefix"]) else None for t in tops]

    # 4. the walk of the own subtrees against each other domain's box
    rcq2, period = backend.contact_geometry(lo, L)
    payloads = []
    for r in range(world):
        if r == rank or dom_lo[r] is None or len(own["level"]) <= 1:
            payloads.append(None)
            continue
        # a pseudo group node carrying the domain box, after the tree's nodes
        nn = len(own["level"])
        qlo = np.concatenate([own["qlo"], dom_lo[r][None].astype(np.uint32)])
        qhi = np.concatenate([own["qhi"], dom_hi[r][None].astype(np.uint32)])
        qlo[0], qhi[0] = 0, (1 << LEVELS) - 1  # the subtrees' common fake root: always opened
        walk_tree = {"level": np.concatenate([own["level"], [LEVELS]]).astype(np.uint8),
                     "first_child": np.concatenate([own["first_child"], [-1]]).astype(np.int32),
                     "nchild": np.concatenate([own["nchild"], [0]]).astype(np.uint8)}
        L_ = backend.walk(walk_tree, qlo, qhi, np.array([nn], np.int32), float(prm["theta"]), rcq2, period)
        acc, leaves = L_["C"], L_["P"]
        visited = set(int(v) for v in acc) | set(int(v) for v in leaves)
        for v in list(visited):  # the opened inner nodes: every ancestor below the fake root
            q = int(own["parent"][v])
            while q > 0 and q not in visited:
                visited.add(q)
                q = int(own["parent"][q])
        vis = np.array(sorted(visited), np.int64)
        frozen = np.isin(vis, acc)
        leafp = [np.arange(own["begin"][v], own["end"][v]) for v in leaves]
        pidx = np.concatenate(leafp) if leafp else np.zeros(0, np.int64)
        payloads.append({"level": own["level"][vis], "prefix": own["prefix"][vis], "qlo": own["qlo"][vis],
                         "qhi": own["qhi"][vis], "frozen": frozen,
                         "M": mom["M"][vis], "c": np.stack([mom["cx"][vis], mom["cy"][vis], mom["cz"][vis]], 1),
                         "Q": mom["Q"][vis], "particles": {f: Q[f][pidx] for f in FIELDS}})
    lets = _exchange(payloads)

    # 5. the view: top of the tree, own subtrees, all-gathered level-l_d
    #    nodes (frozen where nothing opened them) and the received walks
    nodes = {}  # (level, prefix) -> [frozen, qlo, qhi, M, c, Q]
    for t in tops:
        for j in range(len(t["prefix"])):
            nodes[(split_level, int(t["prefix"][j]))] = [True, t["qlo"][j], t["qhi"][j], t["M"][j], t["c"][j], t["Q"][j]]
    for p in lets:
        if p is None:
            continue
        for j in range(len(p["level"])):
            key = (int(p["level"][j]), int(p["prefix"][j]))
            nodes[key] = [bool(p["frozen"][j]), p["qlo"][j], p["qhi"][j], p["M"][j], p["c"][j], p["Q"][j]]
    for j in range(1, len(own["level"])):
        nodes[(int(own["level"][j]), int(own["prefix"][j]))] = [False, own["qlo"][j], own["qhi"][j], 0.0,
                                                                np.zeros(3), np.zeros(6)]
    for (lv_, p_) in [kk for kk in nodes if kk[0] == split_level]:  # the top of the tree
        for up in range(split_level - 1, -1, -1):
            kk = (up, p_ >> (3 * (split_level - up)))
            box = nodes[(lv_, p_)]
            if kk in nodes:
                cur = nodes[kk]
                cur[1] = np.minimum(cur[1], box[1])
                cur[2] = np.maximum(cur[2], box[2])
            else:
                nodes[kk] = [False, box[1].copy(), box[2].copy(), 0.0, np.zeros(3), np.zeros(6)]
    keys_sorted = sorted(nodes)
    vlevel = np.array([kk[0] for kk in keys_sorted], np.uint8)
    vprefix = np.array([kk[1] for kk in keys_sorted], np.uint64)
    vfrozen = np.array([nodes[kk][0] for kk in keys_sorted], bool)
    # particles of the view: own and received leaves, in key order
    recvp = [p["particles"] for p in lets if p is not None]
    V = {f: np.concatenate([Q[f]] + [x[f] for x in recvp]) for f in FIELDS}
    vk = backend.keys(*backend.tree_coords(V), lo, L)
    o = np.argsort(vk, kind="stable")
    V = {f: np.ascontiguousarray(V[f][o]) for f in FIELDS}
    vk = np.ascontiguousarray(vk[o])
    vb, ve = _ranges(vk, vlevel, vprefix)
    view = _tree(vlevel, vprefix, vb, ve, fake_root=False)
    view["nchild"] = np.where(vfrozen, 0, view["nchild"]).astype(np.uint8)  # frozen nodes end the walk
    view["qlo"] = np.stack([nodes[kk][1] for kk in keys_sorted]).astype(np.uint32)
    view["qhi"] = np.stack([nodes[kk][2] for kk in keys_sorted]).astype(np.uint32)
    vm = {"M": np.array([nodes[kk][3] for kk in keys_sorted], np.float64),
          "cx": np.array([nodes[kk][4][0] for kk in keys_sorted], np.float64),
          "cy": np.array([nodes[kk][4][1] for kk in keys_sorted], np.float64),
          "cz": np.array([nodes[kk][4][2] for kk in keys_sorted], np.float64),
          "Q": np.stack([nodes[kk][5] for kk in keys_sorted]).astype(np.float64)}
    vm = backend.combine(view, vm, vfrozen, V, order)

    # groups: maximal own nodes with at most n_g particles (the top of the
    # tree holds more than n_g per node: checked above), ordered by begin
    ownset = set((int(own["level"][j]), int(own["prefix"][j])) for j in range(1, len(own["level"])))
    cnt = (ve.astype(np.int64) - vb.astype(np.int64))
    grp = []
    for kq, kk in enumerate(keys_sorted):
        if kk not in ownset:
            continue
        small = cnt[kq] <= n_g or view["nchild"][kq] == 0
        par = view["parent"][kq]
        topok = kk[0] == split_level or cnt[par] > n_g
        if small and topok:
            grp.append(kq)
    grp = np.array(sorted(grp, key=lambda q: int(vb[q])), np.int32)
    lists = backend.walk(view, view["qlo"], view["qhi"], grp, float(prm["theta"]), rcq2, period)
    if len(lists["P"]) and (vfrozen[lists["P"]]).any():
        raise RuntimeError("a group opened a node its domain's walk accepted")
    acc_all = backend.forces(view, lists, grp, vm, V)
    ownmask = np.zeros(len(V["x"]), bool)
    for q in grp:
        ownmask[vb[q]:ve[q]] = True
    info = {"owned": int(ownmask.sum()), "view_particles": len(V["x"]), "view_nodes": len(vlevel),
            "let_nodes_received": int(sum(len(p["level"]) for p in lets if p is not None)),
            "let_particles_received": int(sum(len(p["particles"]["x"]) for p in lets if p is not None)),
            "frozen_nodes": int(vfrozen.sum()), "groups": len(grp), "cut": cut,
            "view": view, "lists": lists, "groups_nodes": grp, "view_keys": vk}
    return {f: V[f][ownmask] for f in FIELDS}, acc_all[ownmask], info
