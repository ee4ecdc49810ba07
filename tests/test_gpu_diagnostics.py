"""bh_get_diagnostics against the plain FP64 sums (oracle.diagnostics) and
the contact statistics against a brute-force count of pairs within r_coll."""
import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth

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


def test_sums_match_definition_and_repeat_bitwise():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(70001, 31)
    prm = _prm()
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    d1 = ctx.bh_get_diagnostics(D)
    d2 = ctx.bh_get_diagnostics(D)
    ref = orc.diagnostics(P, prm["G"], prm["M_central"])
    for k in ("mass", "kinetic", "potential_central"):
        assert d1[k] == d2[k]
        assert np.isclose(d1[k], ref[k], rtol=1e-13, atol=0), k
    for k in ("momentum", "angular_momentum"):
        assert np.array_equal(d1[k], d2[k])
        scale = np.abs(ref[k]).max()
        assert np.abs(d1[k] - ref[k]).max() <= 1e-13 * scale, k
    assert d1["contacts"] == -1  # no force evaluation yet


def test_energy_and_angular_momentum_nearly_conserved_by_steps():
    """Over 20 steps the total energy (kinetic + central + self-gravity
    potential) stays within O(dt^2) and L_z (the central force exerts no
    torque; self-gravity and contacts are internal) to rounding."""
    from paper_1907_02289_gb300 import bh
    P = synth.ring(30000, 32)
    prm = _prm()
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    d0 = ctx.bh_get_diagnostics(D)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    w0 = ctx.bh_compute_potential(D)
    ctx.bh_step(D, 20)
    d1 = ctx.bh_get_diagnostics(D)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    w1 = ctx.bh_compute_potential(D)
    assert w0 < 0.0 and w1 < 0.0
    e0 = d0["kinetic"] + d0["potential_central"] + w0
    e1 = d1["kinetic"] + d1["potential_central"] + w1
    assert abs(e1 - e0) <= 1e-6 * abs(e0)
    assert abs(d1["angular_momentum"][2] - d0["angular_momentum"][2]) <= 1e-9 * abs(d0["angular_momentum"][2])


@pytest.mark.parametrize("precision,frame", [(0, 0), (1, 0), (1, 1)])
def test_potential_matches_oracle(precision, frame):
    """Per-particle self-gravity potential over the GPU's lists against the
    oracle's tree potential on the same lists (FP64 either way: 1e-12), and
    W = 1/2 sum m phi against the oracle's, repeated bit for bit."""
    import torch
    from paper_1907_02289_gb300 import bh
    P = synth.ring(40000, 33, phi_max=0.05)
    prm = _prm(precision=precision, key_frame=frame)
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    phi = torch.empty(len(P["x"]), dtype=torch.float64, device="cuda")
    W1 = ctx.bh_compute_potential(D, phi)
    W2 = ctx.bh_compute_potential(D)
    assert W1 == W2
    ref = orc.rebuild(P, orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__}))
    pref = orc.tree_potential(ref, orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__}))
    got = phi.cpu().numpy()
    assert np.max(np.abs(got - pref) / np.abs(pref)) <= 1e-12
    assert np.isclose(W1, orc.self_energy(ref.P["m"], pref), rtol=1e-13, atol=0)


def test_potential_needs_lists():
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(**_prm())
    D = bh.Particles(synth.ring(1000, 34))
    with pytest.raises(bh.BHError) as e:
        ctx.bh_compute_potential(D)
    assert e.value.code == bh.BH_E_STATE


def test_contact_count_matches_brute_force():
    from paper_1907_02289_gb300 import bh
    P = synth.ring(6000, 9, r_in=0.99995, r_out=1.00005, phi_max=4e-4, sigma_z=5e-6)
    prm = _prm(n_g=32, theta=0.6)
    ctx = bh.Context(**prm)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    ctx.bh_compute_forces(D, 0)
    d = ctx.bh_get_diagnostics(D)
    n = orc.contact_pairs(D.numpy(), prm["r_coll"])
    assert n > 100
    assert d["contacts"] == n
    assert d["contact_candidates"] >= 2 * n
