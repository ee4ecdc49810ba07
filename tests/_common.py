"""Shared test helpers: parameter mapping, error metrics, GPU runs."""
import numpy as np

import oracle as orc

ORC_FIELDS = orc.Params.__dataclass_fields__


def orc_params(prm: dict) -> "orc.Params":
    return orc.Params(**{k: v for k, v in prm.items() if k in ORC_FIELDS})


def force_errors(a, ref):
    """Per-particle relative error |da|/|a_ref| and rms-normalised error
    |da|/rms(|a_ref|) of the tree acceleration."""
    d = np.linalg.norm(a - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    rel = d / np.where(r > 0, r, np.inf)
    rmsn = d / np.sqrt(np.mean(r * r))
    return rel, rmsn, r


# The FP64 path is held to its tolerance everywhere; the FP32 path's gate has
# the near-cancelling provision of the error metric (tree part only): every
# particle with |a_ref| >= NEAR_CANCEL x median|a_ref| must meet the relative
# tolerance, and the few below that cut (whose FP32 sums of terms far larger
# than the total carry a large relative error) meet it in the rms-normalised
# form |da_i| / rms|a_ref| instead.
NEAR_CANCEL = 1e-2
FP64_TOL_MAX = 1e-9  # tolerances at or below this are FP64 gates: no provision


def assert_force_close(a, ref, tol, what=""):
    """Gate of the force error.  FP64 tolerances (<= FP64_TOL_MAX): max
    relative error <= tol over every particle.  FP32 tolerances: max relative
    error <= tol over every particle with |a_ref| >= NEAR_CANCEL x median, and
    rms-normalised error <= tol for the particles below that cut.  Returns
    (the form used for the particles below the cut or "rel", max relative
    error over the gated particles)."""
    rel, rmsn, r = force_errors(a, ref)
    if tol <= FP64_TOL_MAX:
        i = int(np.argmax(rel))
        assert rel[i] <= tol, f"{what}: max rel err {rel[i]:.3e} > {tol} (particle {i})"
        return "rel", float(rel[i])
    med = np.median(r)
    ok = r >= NEAR_CANCEL * med
    worst = float(rel[ok].max()) if ok.any() else 0.0
    assert worst <= tol, (
        f"{what}: max rel err {worst:.3e} > {tol} over particles with |a| >= {NEAR_CANCEL} x median "
        f"({int((rel[ok] > tol).sum())} above)")
    if (~ok).any():
        assert rmsn[~ok].max() <= tol, f"{what}: rms-normalised err {rmsn[~ok].max():.3e} > {tol} (near-cancelling)"
        return "rms", worst
    return "rel", worst


def gpu_build(P, prm, precision=None, forces=True, flags=None):
    from paper_1907_02289_gb300 import bh
    p = dict(prm)
    if precision is not None:
        p["precision"] = precision
    ctx = bh.Context(**p)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    ctx.bh_make_lists()
    if forces:
        ctx.bh_compute_forces(D, bh.BH_FORCE_TREE_ONLY if flags is None else flags)
    ctx.bh_sync()
    return ctx, D


def accel_of(D):
    o = D.numpy()
    return np.stack([o["ax"], o["ay"], o["az"]], 1)
