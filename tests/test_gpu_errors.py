"""Error paths made on the host (no device fault is provoked): a list
capacity too small for the lists, and a contact-candidate buffer too small
for a graph-captured step.  Each returns its error code with the sizes the
caller needs, and the context keeps working after it."""
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
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"], n_g=64)
    prm.update(kw)
    return prm


@pytest.mark.parametrize("precision", [0, 1])
def test_list_capacity_overflow_reports_needed_size(precision):
    from paper_1907_02289_gb300 import bh
    P = synth.ring(20000, 31)
    prm = _prm(precision=precision)
    ctx = bh.Context(**dict(prm, list_capacity=100))
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    with pytest.raises(bh.BHError) as e:
        ctx.bh_make_lists()
    assert e.value.code == bh.BH_E_LIST_OVERFLOW
    s = ctx.bh_get_sizes()
    need = s["n_pp"] + s["n_pc"] + s["n_jj"]
    assert need > 100 and s["n_pp"] > 0 and s["n_pc"] > 0 and s["n_jj"] >= s["n_pp"]
    with pytest.raises(bh.BHError) as e:
        ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    assert e.value.code == bh.BH_E_STATE
    ctx.bh_set_list_capacity(need - 1)
    with pytest.raises(bh.BHError) as e:
        ctx.bh_make_lists()
    assert e.value.code == bh.BH_E_LIST_OVERFLOW
    ctx.bh_set_list_capacity(need)  # exactly enough
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    ref = orc.rebuild(P, orc_params(prm))
    L = ctx.bh_get_lists()
    assert np.array_equal(L["P"], ref.lists["P"]) and np.array_equal(L["C"], ref.lists["C"])
    assert_force_close(accel_of(D), orc.tree_forces(ref, orc_params(prm)), 1e-12 if precision == 0 else 1e-5)
    with pytest.raises(bh.BHError):
        ctx.bh_set_list_capacity(-1)


def test_graph_step_contact_overflow_is_reported_and_recoverable():
    """~9e4 contact candidates per evaluation against a graph step allowed
    1000: the graph step drops the excess, the next synchronising call
    returns BH_E_LIST_OVERFLOW, and with the room restored the context steps
    on and gives forces that meet the gate."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(20000, 9, r_in=0.99995, r_out=1.00005, phi_max=0.033, sigma_z=1e-5)
    prm = _prm()
    ctx = bh.Context(**prm)
    ctx.bh_set_tuning(graph=1, sched=2, graph_contact_room=1000)
    D = bh.Particles(P)
    ctx.bh_step(D, 1)  # evaluation 0 (eager, list build) and 1 (the first graph step)
    with pytest.raises(bh.BHError) as e:
        ctx.bh_sync()
    assert e.value.code == bh.BH_E_LIST_OVERFLOW
    assert ctx.bh_get_counters()["n_contacts"] > 1000
    ctx.bh_set_tuning(graph_contact_room=0)
    ctx.bh_step(D, 2)  # evaluations 2 and 3: graph steps with room for the candidates
    ctx.bh_sync()
    ctx.bh_step(D, 1)  # evaluation 4: list build
    ctx.bh_sync()
    ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY)
    ctx.bh_sync()
    now = D.numpy()
    ref = orc.rebuild({f: now[f] for f in orc.FIELDS}, orc_params(prm))
    assert np.array_equal(ref.P["id"], now["id"])
    assert_force_close(accel_of(D), orc.tree_forces(ref, orc_params(prm)), 1e-5, "after recovery")
    with pytest.raises(bh.BHError):
        ctx.bh_set_tuning(graph_contact_room=-5)
