"""Seeded synthetic inputs: a uniform cube and planetary-ring annuli.

This module draws particles and holds the workload presets; it contains none
of the method's arithmetic and is the only code shared by the CUDA path's
tests, the benchmark and the oracle's tests.

The ring recipe stands in for the paper's Saturn ring (Table 1: a narrow
ring around a central planet, equal-mass particles), scaled to ring radius 1
with G = M_central = 1:

* r ~ U[r_in, r_out] (uniform in radius), phi ~ U[0, 2 pi), z ~ N(0, sigma_z);
* circular Kepler velocity sqrt(G M_c / r) plus an isotropic Gaussian
  dispersion sigma_v per component;
* equal masses; contact distance r_coll = 2 x particle radius.

Draw order per call: r, phi, z, then the three velocity Gaussians.
"""
from __future__ import annotations

import math

import numpy as np

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "id")


def uniform_cube(n: int, seed: int = 0) -> dict:
    """n equal-mass particles (total mass 1) uniform in [0,1)^3, at rest."""
    rng = np.random.default_rng(seed)
    pos = rng.random((3, n))
    z0 = np.zeros(n)
    return {
        "x": np.ascontiguousarray(pos[0]), "y": np.ascontiguousarray(pos[1]),
        "z": np.ascontiguousarray(pos[2]), "vx": z0.copy(), "vy": z0.copy(), "vz": z0.copy(),
        "m": np.full(n, 1.0 / n), "id": np.arange(n, dtype=np.int64),
    }


def ring(n: int, seed: int, r_in: float = 0.98, r_out: float = 1.02, sigma_z: float = 1e-4,
         mass: float = 1e-12, sigma_v: float = 1e-4, GM: float = 1.0, phi_max: float = 2 * math.pi,
         id0: int = 0) -> dict:
    """Ring annulus (or the sector phi < phi_max of one)."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_in, r_out, n)
    phi = rng.uniform(0.0, phi_max, n)
    z = rng.normal(0.0, sigma_z, n)
    dv = rng.normal(0.0, sigma_v, (3, n))
    c, s = np.cos(phi), np.sin(phi)
    vk = np.sqrt(GM / r)
    return {
        "x": r * c, "y": r * s, "z": z,
        "vx": -vk * s + dv[0], "vy": vk * c + dv[1], "vz": dv[2],
        "m": np.full(n, mass), "id": np.arange(id0, id0 + n, dtype=np.int64),
    }


def contact_params(dt: float, restitution: float = 0.5, steps_per_contact: float = 8.0):
    """Spring/dashpot constants for Eq. (1)'s contact term.

    The paper fixes only the radial restitution coefficient (0.5).  With a
    contact lasting t_c = steps_per_contact * dt, the damped oscillator
    d'' + eta d' + kappa d = 0 gives e = exp(-eta t_c / 2), so
    eta = -2 ln(e) / t_c and kappa = (pi / t_c)^2 + eta^2 / 4.
    """
    tc = steps_per_contact * dt
    eta = -2.0 * math.log(restitution) / tc
    kappa = (math.pi / tc) ** 2 + 0.25 * eta * eta
    return kappa, eta


def patch_sizes(n_patches: int = 64, seed: int = 3, lo: float = 1e4, hi: float = 5e5):
    """Patch particle counts, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n_patches))).astype(np.int64)


def patches(n_patches: int = 64, seed: int = 3, surface_n: int = 1 << 20):
    """Independent annular sectors with the surface density of a
    surface_n-particle full ring; returns (list of particle dicts, sizes)."""
    sizes = patch_sizes(n_patches, seed)
    out, id0 = [], 0
    for p, n in enumerate(sizes):
        out.append(ring(int(n), seed=1000 * seed + p, phi_max=2 * math.pi * n / surface_n, id0=id0))
        id0 += int(n)
    return out, sizes


# --------------------------------------------------------------------------
# Workload presets: the five configurations the method is measured on.
# --------------------------------------------------------------------------
DT = 1e-3
PARTICLE_RADIUS = 1e-5


def _ring_params(theta, n_g, precision, steps, rebuild_every=4):
    kappa, eta = contact_params(DT)
    return dict(theta=theta, n_g=n_g, n_leaf=8, eps=0.0, order=2, G=1.0, M_central=1.0,
                r_coll=2 * PARTICLE_RADIUS, kappa=kappa, eta=eta, dt=DT, rebuild_every=rebuild_every,
                precision=precision, steps=steps)


PRESETS = {
    # uniform cube, FP64, one force evaluation
    "cube4k": dict(n=4096, seed=0, kind="cube",
                   params=dict(theta=0.5, n_g=64, n_leaf=8, eps=1e-3, order=1, G=1.0, M_central=0.0,
                               r_coll=0.0, kappa=0.0, eta=0.0, dt=DT, rebuild_every=1, precision=0,
                               steps=0)),
    # ring 2^20, plain FP64 path, 10 leapfrog steps, lists rebuilt every 4
    "ring1m_fp64": dict(n=1 << 20, seed=1, kind="ring", params=_ring_params(0.5, 128, 0, 10)),
    # ring 2^24, FP32 group-relative vs FP64 on the same lists
    "ring16m_fp32": dict(n=1 << 24, seed=2, kind="ring", params=_ring_params(0.5, 128, 1, 10)),
    # 64 independent patches, 20 steps
    "patches64": dict(n=None, seed=3, kind="patches", autotune=True, params=_ring_params(0.5, 128, 1, 20)),
    # ring 2^26, FP32 group-relative forces, theta 0.4, 10 steps; the paper's
    # cylindrical tree (Sec. 4.3) and an autotuned n_g
    "ring64m_fp32": dict(n=1 << 26, seed=4, kind="ring", autotune=True,
                         params=dict(_ring_params(0.4, 128, 1, 10), key_frame=1)),
}


def make(name: str, n: int | None = None):
    """Particles and parameters of a preset (n overrides the particle count)."""
    pr = PRESETS[name]
    n = pr["n"] if n is None else n
    if pr["kind"] == "cube":
        return uniform_cube(n, pr["seed"]), dict(pr["params"])
    if pr["kind"] == "ring":
        return ring(n, pr["seed"]), dict(pr["params"])
    raise ValueError(name)
