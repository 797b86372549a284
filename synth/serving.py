"""Seeded request traces for the serving benchmark (inputs only: scene
builders, transducers, arrival times and piston weights; no method
arithmetic).

The trace has Poisson arrivals (exponential gaps, mean rate `rate` per
second) of planning solves drawn uniformly from a pool of scenes whose sizes
span the stated ranges (spheres of 1k-5k triangles, rib scenes of 10k-40k,
kidney scenes of 20k-60k), each with a random number of random-phase piston
excitations.  The pool's frequencies are
chosen so that every mesh resolves about 6 elements per wavelength (k h ~ 1);
it spans spheres of 1k and 5k triangles, rib scenes of 10k and 20k and kidney
scenes of 20k and 40k.
Each scene carries the OSRC damping radius of the paper's corresponding
experiment, scaled to the same k R_eps (meta["r_eps"]).
"""
from __future__ import annotations

import math

import numpy as np

from . import meshes, scenes


def sphere_with_bowl(level: int, k0: float, k1: float, n_elem: int, seed: int) -> scenes.Scene:
    """Unit penetrable sphere (density ratio 1.1) with a small bowl of pistons
    facing it from +z (nondimensional units, omega rho0 = 2.6)."""
    v, t = meshes.icosphere(level, 1.0)
    s = scenes.Scene(name=f"sphere_L{level}", k0=complex(k0), rho0=1.0, plane_wave_dir=(0.0, 0.0, 1.0))
    s.domains.append(scenes.Domain("sphere", v, t, complex(k1), 1.1))
    s.transducer = scenes.bowl_transducer(seed=seed, n_elem=n_elem, R=4.0, aperture=4.0, piston_radius=0.2, gap=0.05)
    s.meta["omega_rho0"] = 2.6
    s.meta["r_eps"] = 0.1  # the paper's sphere value, 5e-4 m for a 5 mm radius, relative to the radius
    return s


def rib(h: float, tag: str) -> scenes.Scene:
    s = scenes.rib_scene(h=h, freq=1500.0 / (2 * math.pi * h))
    s.name = f"rib_fat_liver_{tag}"
    s.meta["omega_rho0"] = 2 * math.pi * s.freq * s.rho0
    s.meta["r_eps"] = 1e-4 * 1e6 / s.freq  # the paper's rib value (1e-4 m at 1 MHz) at the same k R_eps
    return s


def kidney(h: float, tag: str) -> scenes.Scene:
    s = scenes.kidney_scene(h=h, freq=1500.0 / (2 * math.pi * h))
    s.name = f"kidney_fat_{tag}"
    s.meta["omega_rho0"] = 2 * math.pi * s.freq * s.rho0
    s.meta["r_eps"] = 1e-3 * 1e6 / s.freq  # the paper's kidney value (1e-3 m at 1 MHz) at the same k R_eps
    return s


def rib_10k() -> scenes.Scene:
    return rib(5.3e-3, "10k")


def kidney_20k() -> scenes.Scene:
    return kidney(3.2e-3, "20k")


POOL = {
    "sphere_1k": lambda: sphere_with_bowl(3, 5.0, 5.25, 16, 11),
    "sphere_5k": lambda: sphere_with_bowl(4, 10.0, 10.5, 32, 12),
    "rib_10k": rib_10k,
    "rib_20k": lambda: rib(3.75e-3, "20k"),
    "kidney_20k": kidney_20k,
    "kidney_40k": lambda: kidney(2.26e-3, "40k"),
}
# the smallest scene of each kind (the pool of the short trace)
SMALL = ("sphere_1k", "sphere_5k", "rib_10k", "kidney_20k")


def trace(n_req: int, rate: float = 20.0, max_exc: int = 64, seed: int = 2, exc_seed: int = 3, pool=None):
    """[(arrival_s, scene_key, n_exc)], plus a function weights(i, n_elem)
    giving request i's excitation matrix (n_exc x n_elem, unit-modulus)."""
    keys = sorted(pool or POOL)
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_req)
    t = np.cumsum(gaps) - gaps[0]
    names = [keys[i] for i in rng.integers(0, len(keys), n_req)]
    ex = np.random.default_rng(exc_seed)
    n_exc = ex.integers(1, max_exc + 1, n_req)
    reqs = [(float(t[i]), names[i], int(n_exc[i])) for i in range(n_req)]

    def weights(i: int, n_elem: int) -> np.ndarray:
        r = np.random.default_rng([exc_seed, i])
        return np.exp(2j * np.pi * r.random((reqs[i][2], n_elem)))

    return reqs, weights
