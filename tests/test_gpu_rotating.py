"""The rotating coordinate frame of Sec. 4.4 on the GPU: steps in a frame
turning at the Kepler rate of the ring centre against the oracle's steps in
the same frame, the graph-captured steps against eager ones, and the frame's
run mapped back against the inertial run."""
import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth
from _common import orc_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _prm(**kw):
    prm = dict(synth.PRESETS["ring16m_fp32"]["params"], n_g=64, omega=1.0)
    prm.update(kw)
    return prm


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_steps_in_rotating_frame_match_oracle(prec, tol):
    """10 KDK steps in the turning frame (lists rebuilt at evaluations 0, 4,
    8, in that frame) against the oracle's: same particle order at the last
    rebuild, positions and velocities within the force tolerance carried
    through the steps."""
    from paper_1907_02289_gb300 import bh
    n = 30000
    P = synth.ring(n, 41, r_in=0.999, r_out=1.001, phi_max=0.05)
    prm = _prm(precision=prec)
    S, aref, _ = orc.step(P, orc_params(prm), 10)
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_step(D, 10)
    ctx.bh_sync()
    out = D.numpy()
    assert np.array_equal(out["id"], S.P["id"])
    a_tree = np.linalg.norm(aref - orc.central(S.P["x"], S.P["y"], S.P["z"], 1.0, 1.0), axis=1).max()
    dx = max(np.abs(out[f] - S.P[f]).max() for f in ("x", "y", "z"))
    dv = max(np.abs(out[f] - S.P[f]).max() for f in ("vx", "vy", "vz"))
    assert dv <= 20 * prm["dt"] * tol * a_tree + 1e-14
    assert dx <= 200 * prm["dt"] ** 2 * tol * a_tree + 1e-14
    # the frame turned by 10 omega dt: the patch's centre barely moved in it
    assert abs(np.mean(out["y"]) - np.mean(P["y"])) < 2e-4


def test_rotating_graph_steps_equal_eager_steps():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(20000, 42)
    prm = _prm(precision=1)
    outs = []
    for graph in (0, 1):
        ctx = bh.Context(**prm)
        ctx.bh_set_tuning(graph=graph, sched=2)
        D = bh.Particles(P)
        ctx.bh_step(D, 7)
        ctx.bh_sync()
        outs.append(D.numpy())
    for f in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az"):
        np.testing.assert_allclose(outs[1][f], outs[0][f], rtol=1e-12, atol=1e-30, err_msg=f)


def test_rotating_run_mapped_back_equals_inertial_run():
    """theta = 0 (the lists cover every pair, so the forces do not depend on
    the frame's tree): the turning-frame run, rotated back by the angle the
    frame turned, is the inertial run to rounding."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(6000, 43, r_in=0.999, r_out=1.001, phi_max=0.01, mass=1e-9)
    prm = _prm(theta=0.0, precision=0)
    res = []
    for omega in (1.0, 0.0):
        ctx = bh.Context(**dict(prm, omega=omega))
        D = bh.Particles(P)
        ctx.bh_step(D, 8)
        ctx.bh_sync()
        res.append(D.numpy())
    back = orc.to_inertial(res[0], prm["dt"] * 8)
    o_r, o_i = np.argsort(res[0]["id"]), np.argsort(res[1]["id"])
    for f in ("x", "y", "z"):
        assert np.max(np.abs(back[f][o_r] - res[1][f][o_i])) < 1e-13, f
    for f in ("vx", "vy", "vz"):
        assert np.max(np.abs(back[f][o_r] - res[1][f][o_i])) < 1e-11, f
