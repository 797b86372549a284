"""Seeded synthetic scenes: domains (meshes + materials), the exterior medium,
and transducer layouts, shaped like the paper's model problems.

Input generation only.  The material-to-wavenumber rule is the problem
statement of Sec. 2.1 (real part 2*pi*f/c, imaginary part the power-law
attenuation alpha(f) = alpha_1MHz * (f / 1 MHz)^b, Table 1); the solver and
the oracle both receive the resulting complex wavenumbers as inputs.

The paper's CT-derived rib, fat, kidney and liver meshes are not available;
the scenes below are synthetic stand-ins with the stated sizes, proportions,
materials and triangle counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import meshes


@dataclass
class Domain:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    k: complex
    rho: float


@dataclass
class Scene:
    name: str
    k0: complex
    rho0: float
    domains: list = field(default_factory=list)
    freq: float = 0.0
    c0: float = 0.0
    plane_wave_dir: tuple | None = None
    transducer: dict | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_triangles(self) -> int:
        return int(sum(d.tris.shape[0] for d in self.domains))

    @property
    def n_vertices(self) -> int:
        return int(sum(d.verts.shape[0] for d in self.domains))

    @property
    def n_dofs(self) -> int:
        return 2 * self.n_vertices


def wavenumber(freq: float, c: float, alpha_1mhz: float = 0.0, b: float = 1.0) -> complex:
    """k = 2 pi f / c + i alpha(f), alpha(f) = alpha_1MHz (f/1MHz)^b (Sec. 2.1, Table 1)."""
    return complex(2.0 * math.pi * freq / c, alpha_1mhz * (freq / 1.0e6) ** b)


# ---------------------------------------------------------------- scenes


def sphere_scene(level: int = 3, k0: complex = 5.0, k1: complex = 5.25, rho_ratio: float = 1.1,
                 radius: float = 1.0) -> Scene:
    """One penetrable sphere (icosphere of the given level) in free space,
    plane wave along +z.  Level 3: 642 vertices, 1280 triangles."""
    v, t = meshes.icosphere(level, radius)
    s = Scene(name=f"sphere_L{level}", k0=complex(k0), rho0=1.0, plane_wave_dir=(0.0, 0.0, 1.0))
    s.domains.append(Domain("sphere", v, t, complex(k1), rho_ratio))
    s.meta["radius"] = radius
    return s


def two_sphere_scene(level: int = 2, k0=4.0, k1=4.5 + 0.2j, k2=3.6, rho1=1.3, rho2=0.8) -> Scene:
    """Two disjoint spheres of different materials (radius 1 at x=-1.3 and
    radius 0.8 at x=+1.2): the smallest multiple-domain case."""
    v1, t1 = meshes.icosphere(level, 1.0, (-1.3, 0.0, 0.0))
    v2, t2 = meshes.icosphere(level, 0.8, (1.2, 0.1, 0.0))
    s = Scene(name=f"two_spheres_L{level}", k0=complex(k0), rho0=1.0, plane_wave_dir=(0.0, 0.6, 0.8))
    s.domains.append(Domain("a", v1, t1, complex(k1), rho1))
    s.domains.append(Domain("b", v2, t2, complex(k2), rho2))
    return s


def shell_scene(level: int = 2, k0=3.0, k_core=3.4 + 0.1j, k_shell=2.7 + 0.05j) -> Scene:
    """A core sphere (radius 0.8) inside a hollow spherical shell (radii 1.0
    and 1.4) with a gap of exterior medium between them.  The shell domain's
    boundary has two components; its inner surface is oriented inward (out
    of the shell material), as for the perinephric fat layer."""
    vc, tc = meshes.icosphere(level, 0.8)
    vo, to = meshes.icosphere(level, 1.4)
    vi, ti = meshes.flip(*meshes.icosphere(level, 1.0))
    vs, ts = meshes.merge([(vo, to), (vi, ti)])
    s = Scene(name=f"shell_L{level}", k0=complex(k0), rho0=1.0, plane_wave_dir=(0.0, 0.0, 1.0))
    s.domains.append(Domain("core", vc, tc, complex(k_core), 1.2))
    s.domains.append(Domain("shell", vs, ts, complex(k_shell), 0.9))
    return s


# Materials: (c [m/s], rho [kg/m^3], alpha at 1 MHz [Np/m], b)
RIB_SCENE_MEDIA = {
    "water": (1500.0, 1000.0, 0.0, 2.0),
    "fat": (1478.0, 950.0, 0.0, 1.0),
    "liver": (1570.0, 1060.0, 0.0, 1.3),
    "bone": (2800.0, 1900.0, 47.0, 1.0),
}

KIDNEY_SCENE_MEDIA = {
    "water": (1500.0, 1000.0, 0.0, 2.0),
    "fat": (1478.0, 950.0, 0.0, 1.0),
    "kidney": (1560.0, 1050.0, 0.0, 1.0),
}


def _mat(media, name, freq):
    c, rho, a, b = media[name]
    return wavenumber(freq, c, a, b), rho


def rib_scene(h: float = 2.65e-3, freq: float = 0.5e6) -> Scene:
    """Five rounded-capsule ribs (100 x 12 x 8 mm, 18 mm pitch) between a
    rounded fat slab (150 x 150 x 20 mm) and an ellipsoidal liver (semi-axes
    60 x 50 x 40 mm), in water.  h = 2.65 mm gives about 40k triangles.
    Geometric focus at the origin (inside the liver, 30 mm behind the ribs);
    the bowl transducer faces it from +z."""
    fat_v, fat_t = meshes.rounded_box((75e-3, 75e-3, 10e-3), 6.0, h, center=(0.0, 0.0, 62e-3))
    ribs = []
    for i in range(5):
        y = (i - 2) * 18e-3
        ribs.append(meshes.capsule((50e-3, 6e-3, 4e-3), 2.0, h, center=(0.0, y, 40e-3)))
    rib_v, rib_t = meshes.merge(ribs)
    liv_v, liv_t = meshes.rounded_box((60e-3, 50e-3, 40e-3), 2.0, h, center=(0.0, 0.0, -12e-3))
    k0, rho0 = _mat(RIB_SCENE_MEDIA, "water", freq)
    s = Scene(name="rib_fat_liver", k0=k0, rho0=rho0, freq=freq, c0=1500.0)
    for name, (v, t), med in (("ribs", (rib_v, rib_t), "bone"), ("fat", (fat_v, fat_t), "fat"),
                              ("liver", (liv_v, liv_t), "liver")):
        k, rho = _mat(RIB_SCENE_MEDIA, med, freq)
        s.domains.append(Domain(name, v, t, k, rho))
    s.transducer = bowl_transducer(seed=0, focus=(0.0, 0.0, 0.0))
    return s


def rib_scene_resolved(h: float = 2.65e-3) -> Scene:
    """The rib scene at the frequency where its ~41k-triangle mesh resolves
    about 6 elements per wavelength (0.1 MHz; k h ~ 1), for solve timings."""
    s = rib_scene(h=h, freq=0.1e6)
    s.name = "rib_fat_liver_0.1MHz"
    return s


def kidney_scene(h: float = 1.8e-3, freq: float = 1.0e6) -> Scene:
    """Ellipsoidal kidney (110 x 60 x 40 mm) inside a hollow perinephric fat
    shell whose inner surface is offset 1 mm and outer surface 8 mm from the
    kidney (scaled ellipsoids), in water; focus at the kidney centre.
    h = 1.8 mm gives about 60k triangles."""
    a, b, c = 55e-3, 30e-3, 20e-3
    kid = meshes.rounded_box((a, b, c), 2.0, h)
    outer = meshes.rounded_box((a + 8e-3, b + 8e-3, c + 8e-3), 2.0, h)
    inner = meshes.flip(*meshes.rounded_box((a + 1e-3, b + 1e-3, c + 1e-3), 2.0, h))
    shell_v, shell_t = meshes.merge([outer, inner])
    k0, rho0 = _mat(KIDNEY_SCENE_MEDIA, "water", freq)
    s = Scene(name="kidney_fat", k0=k0, rho0=rho0, freq=freq, c0=1500.0)
    kk, rk = _mat(KIDNEY_SCENE_MEDIA, "kidney", freq)
    kf, rf = _mat(KIDNEY_SCENE_MEDIA, "fat", freq)
    s.domains.append(Domain("kidney", kid[0], kid[1], kk, rk))
    s.domains.append(Domain("fat", shell_v, shell_t, kf, rf))
    s.transducer = bowl_transducer(seed=1, focus=(0.0, 0.0, 0.0))
    return s


# ---------------------------------------------------------------- transducer


def bowl_transducer(seed: int = 0, n_elem: int = 256, R: float = 0.18, aperture: float = 0.2,
                    piston_radius: float = 3e-3, focus=(0.0, 0.0, 0.0), gap: float = 0.4e-3) -> dict:
    """Piston layout on a spherical bowl (radius of curvature R, aperture
    diameter `aperture`) whose geometric focus is `focus`; the bowl lies on
    the +z side of the focus.  Piston centres are drawn by rejection sampling
    (uniform on the cap, minimum centre spacing 2*radius + gap); each piston
    faces the focus.  Returns centres (n,3), normals (n,3), radii (n,)."""
    rng = np.random.default_rng(seed)
    theta_max = math.asin(min(1.0, (aperture / 2.0) / R))
    cos_lo = math.cos(theta_max)
    centres: list[np.ndarray] = []
    f = np.asarray(focus, dtype=np.float64)
    dmin = 2.0 * piston_radius + gap
    tries = 0
    while len(centres) < n_elem:
        tries += 1
        if tries > 200000:
            raise RuntimeError("bowl_transducer: could not place all pistons")
        cz = rng.uniform(cos_lo, 1.0)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        sz = math.sqrt(max(0.0, 1.0 - cz * cz))
        d = np.array([sz * math.cos(phi), sz * math.sin(phi), cz])
        p = f + R * d
        if centres and np.min(np.linalg.norm(np.asarray(centres) - p, axis=1)) < dmin:
            continue
        centres.append(p)
    C = np.asarray(centres)
    N = f[None, :] - C
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    return {"centres": C, "normals": N, "radii": np.full(n_elem, piston_radius), "focus": f}


def focusing_weights(tr: dict, k0: complex, target=None) -> np.ndarray:
    """Uniform-amplitude piston weights phased to focus at `target`:
    arg w_m = -Re(k0) |c_m - target|."""
    t = tr["focus"] if target is None else np.asarray(target, dtype=np.float64)
    d = np.linalg.norm(tr["centres"] - t[None, :], axis=1)
    return np.exp(-1j * k0.real * d)


def random_phase_weights(n_elem: int, n_rhs: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.exp(2j * math.pi * rng.random((n_rhs, n_elem)))


# ---------------------------------------------------------------- vectors


def random_complex(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def smooth_trace_vector(scene: Scene, seed: int = 0) -> np.ndarray:
    """A smooth test vector in system order: per domain [psi (nv); phi (nv)],
    sampled from random low-order harmonics of position."""
    rng = np.random.default_rng(seed)
    out = []
    for d in scene.domains:
        x = d.verts
        ext = np.ptp(x, axis=0).max() or 1.0
        blocks = []
        for _ in range(2):
            w = rng.standard_normal((3, 3)) * (2.0 * math.pi / ext)
            ph = rng.random(3) * 2 * math.pi
            a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
            val = sum(a[i] * np.cos(x @ w[i] + ph[i]) for i in range(3))
            blocks.append(val)
        out.append(np.concatenate(blocks))
    return np.concatenate(out)
