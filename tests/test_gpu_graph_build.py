"""List-constructing steps issued as one CUDA graph (tuning graph = 1): the
device-sized build (tree levels, group count and list sizes kept on the
device, buffers sized from the previous build) gives the bits of the eager
build, step after step; a build that outgrows those buffers stops after the
reordering and is finished eagerly, again with the same bits; graph = 2 keeps
list-constructing steps eager (Sec. 4.2: the list-constructing and the
list-reusing steps)."""
import math

import numpy as np
import pytest

from paper_1907_02289_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _ring_prm(**kw):
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"])
    prm.update(n_g=64)
    prm.update(kw)
    return prm


def _cube_prm(**kw):
    prm = dict(synth.PRESETS["cube4k"]["params"])
    prm.update(rebuild_every=4)
    prm.update(kw)
    return prm


def _run(P, prm, graph, steps, offsets=None, tune=None, between=None):
    """steps: list of step counts per bh_step call; between(k, D) may change
    the particles after call k (the same change for every run); tune
    "retune" changes the launch settings after every call."""
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(offsets=offsets, **prm) if offsets is not None else bh.Context(**prm)
    retune = tune == "retune"
    ctx.bh_set_tuning(graph=graph, sched=2, **({} if retune or not tune else tune))
    D = bh.Particles(P)
    for k, s in enumerate(steps):
        ctx.bh_step(D, s)
        ctx.bh_sync()
        if between:
            between(k, D)
        if retune:
            ctx.bh_set_tuning(warps=(2, 8, 4, 8)[k % 4], sched=(1, 2)[k % 2], chunk=(64, 96)[k % 2])
    return ctx, D


def _same_state(ca, Da, cb, Db, lists=True):
    a, b = Da.numpy(), Db.numpy()
    for f in a:
        assert np.array_equal(a[f], b[f]), f
    sa, sb = ca.bh_get_sizes(), cb.bh_get_sizes()
    assert sa == sb
    if lists:
        la, lb = ca.bh_get_lists(), cb.bh_get_lists()
        for f in la:
            assert np.array_equal(la[f], lb[f]), f
        ta, tb = ca.bh_get_tree(), cb.bh_get_tree()
        for f in ta:
            assert np.array_equal(ta[f], tb[f]), f


CASES = {
    # FP32, cylindrical key frame, contacts
    "ring_cyl_fp32": (lambda: synth.ring(30011, 31, r_in=0.999, r_out=1.001, phi_max=0.08),
                      lambda: _ring_prm(key_frame=1), None, None),
    # FP32, Cartesian, dense contacts (~4 per particle; its lists grow by half
    # from one build to the next, so the graph gets 100% of room)
    "ring_dense_fp32": (lambda: synth.ring(20000, 9, r_in=0.99995, r_out=1.00005, phi_max=0.033, sigma_z=1e-5),
                        lambda: _ring_prm(), None, dict(graph_room=100)),
    # FP64 path
    "ring_fp64": (lambda: synth.ring(20000, 32), lambda: _ring_prm(precision=0), None, None),
    # softened cube, FP64, monopole
    "cube_fp64": (lambda: synth.uniform_cube(6000, 33), lambda: _cube_prm(), None, None),
    # uneven patches (a forest of trees), FP32
    "patches": (None, lambda: _ring_prm(), [4000, 25000, 900, 12000], None),
    # frame rotating at the Kepler rate of r = 1 (Sec. 4.4), cylindrical keys
    "ring_rotating": (lambda: synth.ring(25013, 38, phi_max=0.1), lambda: _ring_prm(omega=1.0, key_frame=1), None,
                      None),
    # settings changed between steps: the step graphs are captured again
    "retuned": (lambda: synth.ring(20011, 39), lambda: _ring_prm(), None, "retune"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_graph_builds_equal_eager_builds(case):
    make, prm_of, sizes, tune = CASES[case]
    prm = prm_of()
    offsets = None
    if sizes:
        parts = [synth.ring(n, 700 + q, phi_max=2 * math.pi * n / (1 << 20), id0=sum(sizes[:q]))
                 for q, n in enumerate(sizes)]
        P = {f: np.concatenate([p[f] for p in parts]) for f in synth.FIELDS}
        offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    else:
        P = make()
    # evaluations 0..12: builds at 0 (eager: the first), 4, 8, 12
    steps = [3, 1, 4, 4]
    c0, D0 = _run(P, prm, 0, steps, offsets, tune="retune" if tune == "retune" else None)
    c1, D1 = _run(P, prm, 1, steps, offsets, tune=tune)
    _same_state(c0, D0, c1, D1)
    k0, k1 = c0.bh_get_counters(), c1.bh_get_counters()
    assert k0["n_rebuilds"] == k1["n_rebuilds"] == 4
    assert k0["n_graph_builds"] == 0
    assert k1["n_graph_builds"] == 3 and k1["n_graph_build_redos"] == 0
    for f in ("n_groups", "n_pp", "n_pc", "n_pp_far", "n_contacts", "n_refined"):
        assert k0[f] == k1[f], f


def test_graph_two_keeps_list_builds_eager():
    P = synth.ring(20000, 34)
    prm = _ring_prm()
    c2, D2 = _run(P, prm, 2, [9])
    c0, D0 = _run(P, prm, 0, [9])
    _same_state(c0, D0, c2, D2, lists=False)
    assert c2.bh_get_counters()["n_graph_builds"] == 0


def _cluster(k, D):
    """After the first call: 40 clusters of 12 coincident particles (a chain
    of single-child nodes down to the last level for each), so the next
    build needs more nodes than the previous one."""
    if k != 0:
        return
    import torch
    n = D.t["x"].numel()
    src = torch.arange(0, 40 * 997, 997, device=D.t["x"].device) % n
    for f in ("x", "y", "z"):
        t = D.t[f]
        for r in range(1, 12):
            t[(src + r * 13) % n] = t[src]
    torch.cuda.synchronize()


@pytest.mark.parametrize("what", ["nodes", "lists"])
def test_outgrown_graph_build_is_finished_eagerly(what):
    if what == "nodes":  # softened gravity, no contacts: coincident particles are harmless
        P = synth.uniform_cube(20000, 35)
        prm = _cube_prm(precision=1, order=2)
        between = _cluster
    else:  # a dense-contact ring whose lists grow by ~10% and then ~50% from one build to the next
        P = synth.ring(20000, 9, r_in=0.99995, r_out=1.00005, phi_max=0.033, sigma_z=1e-5)
        prm = _ring_prm()
        between = None
    steps = [3, 1, 4]  # builds at evaluations 0 (eager), 4 (graph, outgrown), 8 (graph)
    c0, D0 = _run(P, prm, 0, steps, between=between)
    c1, D1 = _run(P, prm, 1, steps, tune=dict(graph_room=0), between=between)
    _same_state(c0, D0, c1, D1)
    k1 = c1.bh_get_counters()
    assert k1["n_graph_builds"] == 2
    assert k1["n_graph_build_redos"] >= 1


@pytest.mark.parametrize("graph", [1, 2])
def test_force_kernel_timed_in_graph_steps(graph):
    """With timing on, every force launch is timed, those inside step
    graphs included (event-record nodes around the kernel, given fresh
    events at each launch); off again, the graphs record nothing."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(20000, 37)
    prm = _ring_prm()
    ctx = bh.Context(**prm)
    ctx.bh_set_tuning(graph=graph, sched=2)
    D = bh.Particles(P)
    ctx.bh_step(D, 3)  # evaluations 0..3 (graphs captured)
    ctx.bh_sync()
    ctx.bh_set_timing(True)
    ctx.bh_get_timing(reset=True)
    ctx.bh_step(D, 8)  # evaluations 4..11: two list builds, six reuses
    ctx.bh_sync()
    ms, launches = ctx.bh_get_timing(reset=True)
    assert launches == 8
    assert ms > 0.0
    ctx.bh_set_timing(False)
    ctx.bh_step(D, 2)
    ctx.bh_sync()
    ctx.bh_set_timing(True)
    ms, launches = ctx.bh_get_timing(reset=True)
    assert launches == 0
