"""Launch tuning, persistent schedules, CUDA-graph steps and the autotuner:
none of them may change what is computed.  Schedules and block sizes give the
same per-group arithmetic (equal up to the order of FP64 contact atomics);
the i-chunk size changes how a group's list is split between lanes, so those
results are held to the FP32 gate against the oracle."""
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


@pytest.fixture(scope="module")
def ring():
    P = synth.ring(30011, 21)
    prm = _prm()
    ref = orc.rebuild(P, orc_params(prm))
    a_ref = orc.tree_forces(ref, orc_params(prm))
    return P, prm, ref, a_ref


def _forces(P, prm, **tune):
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(**prm)
    if tune:
        ctx.bh_set_tuning(**tune)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    return ctx, D


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("warps", [1, 2, 4, 8])
def test_schedules_and_block_sizes_agree(ring, sched, warps):
    P, prm, ref, a_ref = ring
    _, D0 = _forces(P, prm)
    _, D1 = _forces(P, prm, sched=sched, warps=warps)
    np.testing.assert_allclose(accel_of(D1), accel_of(D0), rtol=1e-12, atol=1e-30)


@pytest.mark.parametrize("chunk", [32, 64, 96])
@pytest.mark.parametrize("by_cost", [0, 1])
def test_chunks_and_orders_meet_gate(ring, chunk, by_cost):
    P, prm, ref, a_ref = ring
    _, D = _forces(P, prm, chunk=chunk, order_by_cost=by_cost, sched=2)
    assert_force_close(accel_of(D), a_ref, 1e-5, f"chunk {chunk}")


@pytest.mark.parametrize("window", [64, 256, 100000])
def test_windowed_order_gives_same_forces(ring, window):
    """The processing order never changes a group's arithmetic."""
    P, prm, ref, a_ref = ring
    _, D0 = _forces(P, prm)
    _, D1 = _forces(P, prm, order_window=window)
    np.testing.assert_allclose(accel_of(D1), accel_of(D0), rtol=1e-12, atol=1e-30)


def test_tuning_validation(ring):
    from paper_1907_02289_gb300 import bh
    P, prm, _, _ = ring
    ctx = bh.Context(**prm)
    for kw in (dict(chunk=48), dict(warps=0), dict(warps=9), dict(sched=3), dict(n_g=4), dict(graph=3),
               dict(order_window=-1), dict(graph_contact_room=-1), dict(graph_room=-1), dict(graph_room=1001)):
        with pytest.raises(bh.BHError) as e:
            ctx.bh_set_tuning(**kw)
        assert e.value.code == bh.BH_E_INVAL
    t = ctx.bh_get_tuning()
    assert t == dict(n_g=64, chunk=96, warps=4, sched=2, order_by_cost=1, graph=0, order_window=0,
                     graph_contact_room=0, graph_room=25)


@pytest.mark.parametrize("precision,dense", [(0, False), (1, False), (1, True)])
def test_graph_steps_equal_eager_steps(precision, dense):
    """dense: ~9e4 contact candidates (4.4 contacts per particle), above the
    contact buffer's initial size of 65,536 pairs, so the graph steps rely on
    the room left before capture."""
    from paper_1907_02289_gb300 import bh
    if dense:
        P = synth.ring(20000, 9, r_in=0.99995, r_out=1.00005, phi_max=0.033, sigma_z=1e-5)
        prm = _prm(precision=precision)
    else:
        P = synth.ring(20000, 22)
        prm = _prm(precision=precision)
    outs = []
    for graph in (0, 1):
        ctx = bh.Context(**prm)
        ctx.bh_set_tuning(graph=graph, sched=2)
        D = bh.Particles(P)
        ctx.bh_step(D, 9)  # evaluations 0..9: rebuilds at 0, 4, 8; graphs at 1-3, 5-7, 9
        ctx.bh_sync()
        c = ctx.bh_get_counters()
        outs.append((D.numpy(), c))
    (a, ca), (b, cb) = outs
    assert np.array_equal(a["id"], b["id"])
    for f in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        np.testing.assert_allclose(b[f], a[f], rtol=1e-12, atol=1e-30, err_msg=f)
    assert ca["n_rebuilds"] == cb["n_rebuilds"] == 3
    assert cb["n_launches"] > 0


def test_balance_of_persistent_launch(ring):
    from paper_1907_02289_gb300 import bh
    P, prm, _, _ = ring
    ctx = bh.Context(**prm)
    ctx.bh_set_tuning(sched=2)
    ctx.bh_set_timing(True)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, 0)
    b = ctx.bh_get_balance()
    assert 0.0 < b <= 1.0


def test_autotune_then_step_matches_oracle():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(40000, 23)
    prm = _prm()
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ms = ctx.bh_autotune(D)
    assert ms > 0
    t = ctx.bh_get_tuning()
    assert t["n_g"] in (64, 96, 128, 192, 256) and t["chunk"] in (32, 64, 96) and t["warps"] in (2, 4, 8)
    # the accelerations left by the autotuner are the forces at the current positions
    out = D.numpy()
    tuned = dict(prm, n_g=t["n_g"])
    ref = orc.rebuild(out, orc_params(tuned))
    a_ref = orc.accel(ref, orc_params(tuned))
    inv = np.argsort(ref.perm)
    a = np.stack([out["ax"], out["ay"], out["az"]], 1)
    # total acceleration (central mass included): compare the tree part
    ac = orc.central(out["x"], out["y"], out["z"], tuned["G"], tuned["M_central"])
    assert_force_close(a - ac, a_ref[inv] - ac, 1e-5, "after autotune")
    ctx.bh_step(D, 2)
    ctx.bh_sync()


def test_batch_dynamic_graph_matches_single_patches():
    """Small version of the batched configuration: uneven patches, dynamic
    persistent schedule, graph-captured reuse steps."""
    from paper_1907_02289_gb300 import bh
    sizes = [4000, 25000, 900, 12000]
    parts = [synth.ring(n, 600 + q, phi_max=2 * math.pi * n / (1 << 20), id0=sum(sizes[:q]))
             for q, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    prm = _prm()
    ctx = bh.Context(offsets=off, **prm)
    ctx.bh_set_tuning(sched=2, graph=1)
    D = bh.Particles({f: np.concatenate([p[f] for p in parts]) for f in synth.FIELDS})
    ctx.bh_step(D, 6)
    ctx.bh_sync()
    out = D.numpy()
    for q, p in enumerate(parts):
        cs = bh.Context(**prm)
        Ds = bh.Particles(p)
        cs.bh_step(Ds, 6)
        cs.bh_sync()
        so = Ds.numpy()
        assert np.array_equal(out["id"][off[q]:off[q + 1]], so["id"])
        for f in ("x", "y", "z", "vx", "vy", "vz"):
            np.testing.assert_allclose(out[f][off[q]:off[q + 1]], so[f], rtol=1e-12, atol=1e-30, err_msg=f)


@pytest.mark.parametrize("graph", [0, 1])
def test_host_steps_equal_device_steps_cylindrical(graph):
    """bh_step_host (whose copy back of positions overlaps the last force
    kernel, or waits for the step when that step ran as a graph) gives the
    bits of bh_step, in the cylindrical frame with the autotuned kernel."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(30000, 24, r_in=0.999, r_out=1.001, phi_max=0.08)
    prm = _prm(key_frame=1)
    outs = []
    for host in (False, True):
        ctx = bh.Context(**prm)
        ctx.bh_set_tuning(graph=graph, sched=2)
        if host:
            H = bh.HostParticles(P, pinned=True)
            for _ in range(6):
                ctx.bh_step_host(H, 1)
            outs.append({f: H.a[f].copy() for f in bh.Particles.FIELDS})
        else:
            D = bh.Particles(P)
            for _ in range(6):
                ctx.bh_step(D, 1)
            ctx.bh_sync()
            outs.append(D.numpy())
    for f in bh.Particles.FIELDS:
        assert np.array_equal(outs[0][f], outs[1][f]), f


def test_host_steps_copy_ids_only_when_reordering():
    """bh_step_host copies ids (and masses back) only for calls with a
    list-constructing evaluation; the byte counters say so, and the host
    arrays end equal to the device path's."""
    from paper_1907_02289_gb300 import bh
    n = 20000
    P = synth.ring(n, 25)
    prm = _prm()  # lists rebuilt every 4 evaluations
    ctx = bh.Context(**prm)
    H = bh.HostParticles(P, pinned=True)
    deltas = []
    for _ in range(6):
        c0 = ctx.bh_get_counters()
        ctx.bh_step_host(H, 1)
        c1 = ctx.bh_get_counters()
        deltas.append((c1["n_h2d_bytes"] - c0["n_h2d_bytes"], c1["n_d2h_bytes"] - c0["n_d2h_bytes"]))
    full_in, full_out = 10 * 8 * n + 8 * n, 10 * 8 * n + 8 * n
    # evaluations: call 1 = initial (0) + 1, then 2, 3, 4 (list build), 5, 6
    assert deltas[0] == (7 * 8 * n + 8 * n, full_out)  # no accelerations to copy in yet
    assert deltas[1] == deltas[2] == deltas[4] == deltas[5] == (10 * 8 * n, 9 * 8 * n)
    assert deltas[3] == (full_in, full_out)
    D = bh.Particles(P)
    cd = bh.Context(**prm)
    cd.bh_step(D, 6)
    cd.bh_sync()
    out = D.numpy()
    for f in bh.Particles.FIELDS:
        assert np.array_equal(H.a[f], out[f]), f
