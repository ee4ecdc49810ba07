"""phi-sector domains with the two-level exchange (Sec. 4.5), on 2 and 4 gloo
ranks on the CPU, each rank's arithmetic done by the oracle: every rank's
view of the tree gives its groups the single tree's lists (bit for bit, by
node level and key prefix) and forces equal to the single-domain oracle's
(FP64, 1e-12), across the phi seam of the cylindrical frame and in the
Cartesian frame, contacts included."""
import os
import socket
from types import SimpleNamespace

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_backend(prm):
    import oracle as orc
    from paper_1907_02289_gb300 import domains
    op = orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__})

    def tree_coords(P):
        if op.key_frame == 1:
            phi, r = orc.cyl_coords(P["x"], P["y"])
            return phi, r, np.ascontiguousarray(P["z"])
        return np.ascontiguousarray(P["x"]), np.ascontiguousarray(P["y"]), np.ascontiguousarray(P["z"])

    def keys(a0, a1, a2, lo, L):
        return orc.keys(np.ascontiguousarray(a0), np.ascontiguousarray(a1), np.ascontiguousarray(a2), lo, L)

    def contact_geometry(lo, L):
        if op.key_frame == 1:
            return orc.cyl_geometry(op.r_coll, lo[1], L)
        rcq = op.r_coll * (2097152.0 / L)
        return rcq * rcq, 0

    def moments(tree, x, y, z, m, order):
        return orc.moments(tree, x, y, z, m, order)

    def combine(tree, mom, frozen, V, order):
        """Leaves from their particles, frozen nodes as given, inner nodes
        from their children (parallel-axis shift), deepest level first."""
        out = orc.moments(tree, V["x"], V["y"], V["z"], V["m"], order)
        for f in ("M", "cx", "cy", "cz"):
            out[f][frozen] = mom[f][frozen]
        out["Q"][frozen] = mom["Q"][frozen]
        for lv in sorted(set(int(v) for v in tree["level"]), reverse=True):
            for k in np.nonzero((tree["level"] == lv) & (tree["nchild"] > 0) & ~frozen)[0]:
                ch = np.arange(tree["first_child"][k], tree["first_child"][k] + tree["nchild"][k])
                M = out["M"][ch].sum()
                c = np.array([(out["M"][ch] * out[f][ch]).sum() for f in ("cx", "cy", "cz")]) / M
                Q = out["Q"][ch].sum(0)
                if order >= 2:
                    d = np.stack([out["cx"][ch], out["cy"][ch], out["cz"][ch]], 1) - c
                    d2 = (d * d).sum(1)
                    mm = out["M"][ch]
                    Q = Q + np.array([(mm * (3 * d[:, 0] ** 2 - d2)).sum(), (mm * (3 * d[:, 1] ** 2 - d2)).sum(),
                                      (mm * (3 * d[:, 2] ** 2 - d2)).sum(), (3 * mm * d[:, 0] * d[:, 1]).sum(),
                                      (3 * mm * d[:, 0] * d[:, 2]).sum(), (3 * mm * d[:, 1] * d[:, 2]).sum()])
                out["M"][k], out["cx"][k], out["cy"][k], out["cz"][k] = M, c[0], c[1], c[2]
                out["Q"][k] = Q
        return out

    def walk(tree, qlo, qhi, groups, theta, rcq2, period):
        return orc.lists_ex(tree, np.ascontiguousarray(qlo), np.ascontiguousarray(qhi),
                            np.ascontiguousarray(groups, dtype=np.int32), theta, rcq2, period)

    def forces(tree, lists, groups, mom, V):
        S = SimpleNamespace(groups=np.ascontiguousarray(groups, dtype=np.int32), tree=tree, lists=lists, mom=mom, P=V)
        return np.nan_to_num(orc.tree_forces(S, op), nan=0.0)

    return domains.Backend(tree_coords=tree_coords, keys=keys, key_coords=orc.key_coords, build_tree=orc.build_tree,
                           moments=moments, combine=combine, walk=walk, contact_geometry=contact_geometry,
                           forces=forces)


def _case(frame):
    from paper_1907_02289_gb300 import synth
    kappa, eta = synth.contact_params(1e-3)
    prm = dict(theta=0.5, n_g=64, n_leaf=8, eps=0.0, order=2, G=1.0, M_central=1.0, r_coll=2e-5, kappa=kappa,
               eta=eta, dt=1e-3, rebuild_every=4, key_frame=frame)
    if frame == 1:  # a whole thin ring: sectors meet across the phi seam
        P = synth.ring(24000, 51, r_in=0.9995, r_out=1.0005, sigma_z=2e-6, mass=1e-12)
    else:
        P = synth.ring(24000, 52, r_in=0.999, r_out=1.001, phi_max=0.02)
    return P, prm


def _rank_main(rank, world, port, frame, split_level, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1907_02289_gb300 import domains
        P, prm = _case(frame)
        n = len(P["x"])
        share = slice(rank * n // world, (rank + 1) * n // world)
        mine = {f: P[f][share] for f in domains.FIELDS}
        Pown, acc, info = domains.decomposed_forces(mine, prm, _oracle_backend(prm), split_level)
        view, lists, grp, vk = info["view"], info["lists"], info["groups_nodes"], info["view_keys"]
        glists = []
        for q, g in enumerate(grp):
            P_ids = lists["P"][lists["pp_off"][q]:lists["pp_off"][q + 1]]
            C_ids = lists["C"][lists["pc_off"][q]:lists["pc_off"][q + 1]]
            key = lambda v: (int(view["level"][v]), int(view["prefix"][v]))
            glists.append((key(g), [key(v) for v in P_ids], [key(v) for v in C_ids]))
        out.put((rank, Pown["id"], acc, glists, {k: v for k, v in info.items()
                                                  if k in ("owned", "view_particles", "let_nodes_received",
                                                           "let_particles_received", "frozen_nodes", "groups")}))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,frame,split_level", [(2, 0, 3), (4, 1, 4), (2, 1, 3)])
def test_domains_reproduce_single_tree_lists_and_forces(world, frame, split_level):
    import multiprocessing as mp

    import oracle as orc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, frame, split_level, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    P, prm = _case(frame)
    op = orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__})
    S = orc.rebuild(P, op)
    a_ref = orc.tree_forces(S, op)
    t = S.tree
    key = lambda v: (int(t["level"][v]), int(S.skeys[t["begin"][v]]) >> (3 * (21 - int(t["level"][v]))))
    ref_lists = {}
    for k, g in enumerate(S.groups):
        ref_lists[key(g)] = ([key(v) for v in S.lists["P"][S.lists["pp_off"][k]:S.lists["pp_off"][k + 1]]],
                             [key(v) for v in S.lists["C"][S.lists["pc_off"][k]:S.lists["pc_off"][k + 1]]])
    pos = {int(i): j for j, i in enumerate(S.P["id"])}
    seen, ngroups = set(), 0
    for rank, ids, acc, glists, info in res:
        assert info["owned"] > 0 and info["let_nodes_received"] > 0
        assert info["view_particles"] < len(P["x"])  # a rank holds far less than the whole ring
        for gk, pl, cl in glists:
            assert ref_lists[gk] == (pl, cl), (rank, gk)
        ngroups += len(glists)
        rows = np.array([pos[int(i)] for i in ids])
        seen.update(int(i) for i in ids)
        err = np.linalg.norm(acc - a_ref[rows], axis=1) / np.linalg.norm(a_ref[rows], axis=1)
        assert err.max() <= 1e-12, (rank, err.max())
    assert ngroups == len(S.groups) and len(seen) == len(P["x"])  # every group and particle exactly once


def test_owner_ranges_balance_and_cover():
    from paper_1907_02289_gb300 import domains
    counts = np.random.default_rng(3).integers(0, 100, 512)
    for world in (1, 2, 3, 8):
        cut = domains.owner_ranges(counts, world)
        assert cut[0] == 0 and cut[-1] == 512 and np.all(np.diff(cut) >= 0)
        loads = [counts[cut[r]:cut[r + 1]].sum() for r in range(world)]
        assert max(loads) - min(loads) <= 2 * counts.max()


def test_split_level_too_deep_is_refused():
    from paper_1907_02289_gb300 import domains
    counts = np.zeros(8 ** 3, np.int64)
    counts[:10] = 5  # level-2 node 0 holds 40 <= n_g
    with pytest.raises(ValueError):
        domains.check_split_level(counts, 3, 8, 64)
