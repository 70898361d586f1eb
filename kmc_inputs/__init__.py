"""Seeded synthetic inputs for the kinetic Monte Carlo hard-sphere gas.

This module only draws initial particle states and states the physical set-up of
each workload (box, boundaries, collision diameter, time step).  It holds none of
the collision-step arithmetic, and both the CUDA library and the CPU oracle
consume exactly the arrays it returns.

Workloads (all with m = 1 and kT/m = 1 unless stated):

* ``equilibrium_box``: uniform positions in a periodic cube, velocity components
  i.i.d. N(0, 1).
* ``piston_tube``: uniform positions in an 8 x 1 x 1 box, periodic in y and z, a
  reflecting wall at x = 0 and a piston at x = 8 moving inward at u_p.
* ``spherical_blast``: periodic unit cube with a central sphere of radius 0.1 at 8x
  the background number density and 100x its temperature.
* ``equal_speed``: the paper's timing runs (Sec. 3 and Sec. 4): uniform positions,
  all particles at the same speed in uniformly random directions, reflecting walls;
  in three dimensions or in the x-y plane (``planar``: vz = 0, z fixed at the middle
  of a thin z extent).

The hard-sphere mean free path is lambda = 1/(sqrt(2) n sigma) with
sigma = pi d0^2, so d0 = sqrt(1/(sqrt(2) pi n lambda)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC = 0
REFLECT = 1
ABSORB = 2


@dataclass
class Setup:
    """Physical set-up of one simulation (shared by both implementations)."""

    n: int
    box: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    piston_x0: float = 0.0
    piston_u: float = 0.0
    d0: float = 0.02
    dt: float = 0.01
    seed: int = 1
    max_rounds: int = 4
    profile_bins: int = 0
    profile_every: int = 0
    profile_range: float = 1.0
    steps: int = 1
    name: str = ""
    planar: bool = False  # two-dimensional dynamics in the x-y plane
    species: object = None  # mixture: uint8 species index per particle id
    masses: tuple = ()      # mixture: mass of each species
    radii: tuple = ()       # mixture: effective radius of each species (contact r_i + r_j)
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Setup":
        return replace(self, **kw)


def d0_for_mean_free_path(number_density: float, lam: float) -> float:
    """Collision diameter giving hard-sphere mean free path ``lam``."""
    sigma = 1.0 / (math.sqrt(2.0) * number_density * lam)
    return math.sqrt(sigma / math.pi)


def _uniform(rng: np.random.Generator, n: int, hi: float) -> np.ndarray:
    x = rng.random(n) * hi
    # keep the half-open interval [0, hi) even if the product rounds up
    return np.minimum(x, np.nextafter(hi, 0.0))


def equilibrium_state(n: int, seed: int, L: float = 1.0, sigma_v: float = 1.0):
    rng = np.random.default_rng(seed)
    pos = [_uniform(rng, n, L) for _ in range(3)]
    vel = [rng.standard_normal(n) * sigma_v for _ in range(3)]
    return pos + vel


def tube_state(n: int, seed: int, box=(8.0, 1.0, 1.0)):
    rng = np.random.default_rng(seed)
    pos = [_uniform(rng, n, float(box[k])) for k in range(3)]
    vel = [rng.standard_normal(n) for _ in range(3)]
    return pos + vel


def blast_state(n: int, seed: int, radius: float = 0.1, density_ratio: float = 8.0,
                temperature_ratio: float = 100.0):
    """Hot dense sphere at the centre of a periodic unit cube."""
    rng = np.random.default_rng(seed)
    vs = 4.0 * math.pi / 3.0 * radius ** 3
    n_hot = int(math.floor(n * density_ratio * vs / (1.0 + (density_ratio - 1.0) * vs) + 0.5))
    out = np.empty((3, n))

    def sample(count, inside):
        got = np.empty((0, 3))
        while got.shape[0] < count:
            m = max(1024, int((count - got.shape[0]) * 1.3))
            p = rng.random((m, 3))
            p = np.minimum(p, np.nextafter(1.0, 0.0))
            r2 = ((p - 0.5) ** 2).sum(axis=1)
            keep = p[(r2 < radius * radius) if inside else (r2 >= radius * radius)]
            got = np.concatenate([got, keep])
        return got[:count]

    out[:, :n_hot] = sample(n_hot, True).T
    out[:, n_hot:] = sample(n - n_hot, False).T
    sig = np.ones(n)
    sig[:n_hot] = math.sqrt(temperature_ratio)
    vel = [rng.standard_normal(n) * sig for _ in range(3)]
    return [out[0].copy(), out[1].copy(), out[2].copy()] + vel, n_hot


# --------------------------------------------------------------------------- #
# Named workloads

def equilibrium_setup(n: int = 4096, seed: int = 1, L: float = 1.0, d0: float = 0.02,
                      dt: float = 0.01, steps: int = 200) -> Setup:
    return Setup(n=n, box=(L, L, L), bc=(PERIODIC,) * 3, d0=d0, dt=dt, seed=seed,
                 steps=steps, name=f"equilibrium_box_n{n}")


def piston_setup(n: int = 1 << 20, seed: int = 2, u_p: float = 2.0, lam: float = 0.02,
                 steps: int = 2000, box=(8.0, 1.0, 1.0), profile_bins: int = 256,
                 profile_every: int = 100) -> Setup:
    vol = box[0] * box[1] * box[2]
    d0 = d0_for_mean_free_path(n / vol, lam)
    dt = 0.1 * lam / math.sqrt(3.0)
    return Setup(n=n, box=tuple(float(b) for b in box), bc=(REFLECT, PERIODIC, PERIODIC),
                 piston_x0=float(box[0]), piston_u=u_p, d0=d0, dt=dt, seed=seed,
                 profile_bins=profile_bins, profile_every=profile_every,
                 profile_range=float(box[0]), steps=steps, name=f"piston_tube_n{n}",
                 extra={"lambda": lam})


def blast_setup(n: int = 1 << 27, seed: int = 3, lam_bg: float = 0.005,
                steps: int = 500, radius: float = 0.1) -> Setup:
    vs = 4.0 * math.pi / 3.0 * radius ** 3
    n_hot = int(math.floor(n * 8.0 * vs / (1.0 + 7.0 * vs) + 0.5))
    n_bg = (n - n_hot) / (1.0 - vs)
    d0 = d0_for_mean_free_path(n_bg, lam_bg)
    dt = 0.05 * lam_bg / 1.0  # v_th of the background read as sqrt(kT/m) = 1
    return Setup(n=n, box=(1.0, 1.0, 1.0), bc=(PERIODIC,) * 3, d0=d0, dt=dt, seed=seed,
                 steps=steps, name=f"spherical_blast_n{n}",
                 extra={"n_hot": n_hot, "radius": radius, "temperature_ratio": 100.0})


def equal_speed_state(n: int, seed: int, box, speed: float = 1.0, planar: bool = False):
    """Uniform positions; velocities of one speed in uniformly random directions (in the
    x-y plane with vz = 0 and z at the middle of the box if planar)."""
    rng = np.random.default_rng(seed)
    pos = [_uniform(rng, n, float(box[k])) for k in range(3)]
    if planar:
        pos[2] = np.full(n, 0.5 * float(box[2]))
        th = rng.random(n) * (2.0 * math.pi)
        vel = [speed * np.cos(th), speed * np.sin(th), np.zeros(n)]
    else:
        g = rng.standard_normal((3, n))
        norm = np.sqrt((g * g).sum(axis=0))
        vel = [speed * g[k] / norm for k in range(3)]
    return pos + vel


def equal_speed_setup(n: int = 4096, seed: int = 11, L: float = 1.0, d0: float = 0.002,
                      dt: float = 0.005, speed: float = 1.0, planar: bool = True,
                      steps: int = 100) -> Setup:
    """The paper's timing workload: a box with reflecting walls, one speed, random
    directions.  Planar: an L x L square, z extent d0 (one cell), a 9-cell stencil."""
    box = (L, L, d0 if planar else L)
    return Setup(n=n, box=box, bc=(REFLECT,) * 3, piston_x0=L, piston_u=0.0, d0=d0, dt=dt,
                 seed=seed, steps=steps, planar=planar,
                 name=f"equal_speed_{'2d' if planar else '3d'}_n{n}", extra={"speed": speed})


def init_spec(setup: Setup) -> dict:
    """Parameters of the same workload for the Philox-based (device-side)
    initialisation: kind 1 = uniform box with Gaussian velocity components of
    standard deviation ``sigma``; 2 = uniform box, one speed, random directions;
    3 = blast (ids below ``n_hot`` uniform in the central sphere with ``sigma_hot``,
    the rest uniform outside it).  The draws themselves are defined by the
    initialisation (not by NumPy), so its arrays differ from ``initial_state``'s
    while following the same distributions."""
    if setup.name.startswith("equal_speed"):
        return {"kind": 2, "speed": float(setup.extra.get("speed", 1.0))}
    if setup.name.startswith("spherical_blast"):
        r = float(setup.extra.get("radius", 0.1))
        return {"kind": 3, "n_hot": int(setup.extra["n_hot"]), "sigma": 1.0,
                "sigma_hot": math.sqrt(float(setup.extra.get("temperature_ratio", 100.0))),
                "center": tuple(0.5 * float(b) for b in setup.box), "radius": r}
    return {"kind": 1, "sigma": 1.0}


def paper_timing_setup(figure: int, seed: int = 17, steps: int = 20) -> Setup:
    """The paper's timing workloads at their stated sizes (Sec. 3, Fig. 1: 10^8
    particles in three dimensions; Sec. 4, Fig. 3: 4 x 10^7 particles in two), with
    one common speed s = 1, random directions and positions, reflecting walls, in a
    unit box.  The paper states neither d0 nor the mean free path; here lambda =
    0.01 (3D: lambda = 1/(sqrt(2) n pi d0^2)) and lambda = 0.001 (2D hard disks:
    lambda = 1/(2 sqrt(2) n d0)), both well below the box (the paper asks for a
    fluid-like gas), and dt = 0.1 lambda / s."""
    if figure == 1:
        n, lam = 10 ** 8, 0.01
        d0 = math.sqrt(1.0 / (math.sqrt(2.0) * math.pi * n * lam))
        return equal_speed_setup(n=n, seed=seed, L=1.0, d0=d0, dt=0.1 * lam, speed=1.0,
                                 planar=False, steps=steps)
    if figure == 3:
        n, lam = 4 * 10 ** 7, 0.001
        d0 = 1.0 / (2.0 * math.sqrt(2.0) * n * lam)
        return equal_speed_setup(n=n, seed=seed, L=1.0, d0=d0, dt=0.1 * lam, speed=1.0,
                                 planar=True, steps=steps)
    raise ValueError("figure must be 1 or 3")


def mixture_setup(n: int = 6000, seed: int = 5, L: float = 1.0, frac_b: float = 0.3,
                  mass_b: float = 4.0, d_a: float = 0.016, d_b: float = 0.032,
                  kT_a: float = 1.0, kT_b: float = 1.0, dt: float = 0.004,
                  steps: int = 100) -> Setup:
    """Binary hard-sphere mixture in a periodic cube (Sec. 2: each particle carries a
    mass and an effective radius): species A (m = 1, diameter d_a) and B (m = mass_b,
    diameter d_b), the first round(frac_b n) ids are B; velocity components of each
    species N(0, kT/m).  d0 (the search reach) is the largest contact distance d_b."""
    n_b = int(round(frac_b * n))
    sp = np.zeros(n, dtype=np.uint8)
    sp[:n_b] = 1
    return Setup(n=n, box=(L, L, L), bc=(PERIODIC,) * 3, d0=max(d_a, d_b), dt=dt, seed=seed,
                 steps=steps, name=f"mixture_n{n}", species=sp, masses=(1.0, mass_b),
                 radii=(0.5 * d_a, 0.5 * d_b), extra={"kT": (kT_a, kT_b)})


def mixture_state(setup: Setup):
    rng = np.random.default_rng(setup.seed)
    n = setup.n
    pos = [_uniform(rng, n, float(setup.box[k])) for k in range(3)]
    kT = np.asarray(setup.extra.get("kT", (1.0,) * len(setup.masses)), dtype=np.float64)
    m = np.asarray(setup.masses, dtype=np.float64)
    sig = np.sqrt(kT / m)[setup.species]
    vel = [rng.standard_normal(n) * sig for _ in range(3)]
    return pos + vel


def initial_state(setup: Setup):
    """Six float64 arrays (x, y, z, vx, vy, vz) in particle-id order."""
    if setup.name.startswith("mixture"):
        return mixture_state(setup)
    if setup.name.startswith("equal_speed"):
        return equal_speed_state(setup.n, setup.seed, setup.box, setup.extra.get("speed", 1.0),
                                 setup.planar)
    if setup.name.startswith("equilibrium"):
        return equilibrium_state(setup.n, setup.seed, setup.box[0])
    if setup.name.startswith("piston"):
        return tube_state(setup.n, setup.seed, setup.box)
    if setup.name.startswith("spherical_blast"):
        return blast_state(setup.n, setup.seed)[0]
    raise ValueError(f"unknown workload {setup.name!r}")


def ensemble_setups(count: int = 256, seed0: int = 1000, lo: int = 1 << 12, hi: int = 1 << 18,
                    steps: int = 500):
    """Batched ensemble: N log-uniform in [lo, hi]; even index an equilibrium box
    (d0 scaled so that n*sigma stays that of the 4096-particle box), odd index a
    piston tube with u_p uniform in [1, 3]."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        if k % 2 == 0:
            s = equilibrium_setup(n=n, seed=seed0 + k, d0=0.02 * math.sqrt(4096.0 / n),
                                  steps=steps)
        else:
            s = piston_setup(n=n, seed=seed0 + k, u_p=float(rng.uniform(1.0, 3.0)),
                             steps=steps, profile_bins=0, profile_every=0)
        out.append(s)
    return out


# --------------------------------------------------------------------------- #
# Serving stream

def splitmix64(state: int):
    """One step of the SplitMix64 generator (Steele, Lea, Flood, OOPSLA 2014):
    returns (new_state, output)."""
    mask = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & mask
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return state, z ^ (z >> 31)


def serving_requests(count: int = 10000, master_seed: int = 7, n_lo: int = 1 << 14,
                     n_hi: int = 1 << 22, steps_lo: int = 100, steps_hi: int = 2000):
    """Request mix of the serving stream: each request is an equilibrium box (the
    4096-particle box's density and d0, box edge (N/4096)^(1/3)) or a piston tube
    (8 x 1 x 1, lambda = 0.02), N log-uniform in [n_lo, n_hi], steps uniform in
    [steps_lo, steps_hi]; per-request seeds from a SplitMix64 chain."""
    state = master_seed
    out = []
    for k in range(count):
        state, seed = splitmix64(state)
        rng = np.random.default_rng(seed)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        seed32 = int(seed & 0x7FFFFFFF)
        if rng.random() < 0.5:
            L = (n / 4096.0) ** (1.0 / 3.0)
            s = equilibrium_setup(n=n, seed=seed32, L=L, steps=steps)
        else:
            s = piston_setup(n=n, seed=seed32, steps=steps, profile_bins=0, profile_every=0)
        out.append(s)
    return out


def mean_loguniform(lo: float, hi: float) -> float:
    return (hi - lo) / math.log(hi / lo)
