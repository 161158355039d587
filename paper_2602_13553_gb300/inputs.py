"""Seeded synthetic inputs for the PIMD workloads.

This module draws inputs only: bead positions, masses and the job mixes of the
batching and serving workloads.  It holds none of the method's arithmetic (no
normal modes, no frequencies, no forces), so both the CUDA path and the CPU
oracle can be fed from it.

Workloads (the synthetic stand-ins for the paper's DP-water runs, Sec. V):
  * ``harmonic``: independent 3D harmonic oscillators (m = 1.008 amu,
    hbar*omega = 0.1 eV), bead positions drawn from a seeded Gaussian.
  * ``water_box``: flexible 3-site water-like molecules (O-H 1.0 A,
    H-O-H 104.5 deg) placed uniformly at random in a cubic periodic box with
    an O-O distance of at least 2.5 A, each with a uniformly random
    orientation; every bead starts at the molecule's rigid geometry plus an
    optional Gaussian jitter.
  * ``replica_mix``: the batched workload -- molecules log-uniform in
    [32, 512], box scaled to 1 g/cm^3, P uniform in {8, 16, 32, 64},
    T uniform in [100, 400] K, H or D masses with probability 1/2.
  * ``serving_trace``: Poisson arrivals, molecule count log-uniform in
    [32, 4096] (96 to 12288 atoms), P log-uniform over {4, ..., 128},
    step count log-uniform in [1000, 50000]; its boxes come from
    ``water_lattice_box`` (oxygens on a randomly displaced subset of a cubic
    lattice, O-O >= 2.5 A), which is linear in the molecule count.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASS_O = 15.999
MASS_H = 1.008
MASS_D = 2.014
WATER_AMU = 18.015
AMU_G = 1.66053906660e-24          # g per amu
# water-like force field: kb (eV/A^2), r0 (A), kth (eV/rad^2), th0 (rad),
# eps (eV), sigma (A), rc (A)
WATER_FF = (45.0, 1.0, 3.3, math.radians(104.5), 6.7e-3, 3.166, 6.0)


def water_ff_for_box(L: float):
    """The water-like force field for a cubic box of edge L: the 6 A O-O cutoff,
    capped at 0.48 L (boxes under 12.5 A, such as the 9.86 A 32-molecule boxes
    of the mixes), which keeps the minimum image valid with a margin."""
    ff = list(WATER_FF)
    ff[6] = min(ff[6], 0.48 * L)
    return tuple(ff)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def harmonic(N: int, P: int, seed: int, std: float, mass: float = MASS_H):
    """x [P][N][3] ~ N(0, std^2) per coordinate, mass [N]."""
    g = rng(seed)
    x = g.normal(0.0, std, size=(P, N, 3))
    return np.ascontiguousarray(x), np.full(N, mass)


def box_length(nmol: int, density_g_cm3: float = 1.0) -> float:
    """Cubic box edge (A) holding nmol water molecules at the given density."""
    vol_cm3 = nmol * WATER_AMU * AMU_G / density_g_cm3
    return (vol_cm3 ** (1.0 / 3.0)) * 1e8


def water_box(nmol: int, L: float, P: int, seed: int, *, r_oo_min: float = 2.5,
              r0: float = 1.0, theta0_deg: float = 104.5, jitter: float = 0.0,
              deuterium: bool = False):
    """Return (x [P][3*nmol][3], mass [3*nmol]) for a random water-like box.

    Atoms are ordered O, H, H per molecule.  Coordinates are unwrapped (the O
    lies in [0, L)^3; hydrogens may stick out by a bond length).  Oxygens are
    placed by random sequential addition: a uniform candidate is kept if no
    placed oxygen lies within r_oo_min (minimum image); the test looks only at
    the 27 periodic cells around the candidate (cells at least r_oo_min wide),
    which is the same decision as a test against every placed oxygen."""
    g = rng(seed)
    O = np.zeros((nmol, 3))
    nc = max(1, int(L // r_oo_min))          # cells per edge, each >= r_oo_min
    cells = {}
    r2min = r_oo_min * r_oo_min
    n = 0
    attempts = 0
    while n < nmol:
        attempts += 1
        if attempts > 2000 * max(nmol, 1):
            raise RuntimeError("water_box: could not place %d molecules in L=%.3f" % (nmol, L))
        p = g.uniform(0.0, L, size=3)
        c = [min(nc - 1, int(p[a] * nc / L)) for a in range(3)]
        near = []
        if nc < 3:
            near = list(range(n))
        else:
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        near.extend(cells.get(((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc), ()))
        if near:
            d = O[near] - p
            d -= L * np.rint(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < r2min:
                continue
        O[n] = p
        cells.setdefault(tuple(c), []).append(n)
        n += 1
    return _molecules(g, O, P, r0, theta0_deg, jitter, deuterium)


def water_lattice_box(nmol: int, L: float, P: int, seed: int, *, r_oo_min: float = 2.5,
                      r0: float = 1.0, theta0_deg: float = 104.5, jitter: float = 0.0,
                      deuterium: bool = False):
    """As water_box, but the oxygens start on a random subset of the sites of
    a k x k x k cubic lattice (k^3 >= nmol), each displaced uniformly within
    the cube that keeps every O-O distance >= r_oo_min: linear in nmol and
    vectorised, for the serving trace's thousands of boxes of up to 4096
    molecules (random sequential addition takes seconds per large box).  At
    1 g/cm^3 the lattice is wide enough from 70 molecules on; smaller boxes
    (and any box whose lattice would be too tight) fall back to water_box."""
    k = 1
    while k ** 3 < nmol:
        k += 1
    a = L / k
    if a < r_oo_min:
        return water_box(nmol, L, P, seed, r_oo_min=r_oo_min, r0=r0, theta0_deg=theta0_deg, jitter=jitter,
                         deuterium=deuterium)
    g = rng(seed)
    sites = g.permutation(k ** 3)[:nmol]
    ijk = np.stack([sites // (k * k), (sites // k) % k, sites % k], axis=1).astype(np.float64)
    delta = 0.5 * (a - r_oo_min)
    O = (ijk + 0.5) * a + g.uniform(-delta, delta, size=(nmol, 3))
    return _molecules(g, O, P, r0, theta0_deg, jitter, deuterium)


def _molecules(g, O, P, r0, theta0_deg, jitter, deuterium):
    """Water-like molecules at oxygen positions O [nmol][3]: a uniformly
    random orientation each, rigid geometry (r0, theta0), every bead a copy
    plus N(0, jitter^2); atoms O, H, H per molecule."""
    nmol = O.shape[0]
    half = math.radians(theta0_deg) / 2.0
    h1 = r0 * np.array([math.sin(half), math.cos(half), 0.0])
    h2 = r0 * np.array([-math.sin(half), math.cos(half), 0.0])
    # one uniformly random orientation per molecule (unit quaternions)
    q = g.normal(size=(nmol, 4))
    q /= np.linalg.norm(q, axis=1)[:, None]
    a, b, c, d = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((nmol, 3, 3))
    R[:, 0, 0] = a * a + b * b - c * c - d * d
    R[:, 0, 1] = 2 * (b * c - a * d)
    R[:, 0, 2] = 2 * (b * d + a * c)
    R[:, 1, 0] = 2 * (b * c + a * d)
    R[:, 1, 1] = a * a - b * b + c * c - d * d
    R[:, 1, 2] = 2 * (c * d - a * b)
    R[:, 2, 0] = 2 * (b * d - a * c)
    R[:, 2, 1] = 2 * (c * d + a * b)
    R[:, 2, 2] = a * a - b * b - c * c + d * d
    x1 = np.zeros((3 * nmol, 3))
    x1[0::3] = O
    x1[1::3] = O + R @ h1
    x1[2::3] = O + R @ h2
    x = np.repeat(x1[None, :, :], P, axis=0)
    if jitter > 0.0:
        x = x + g.normal(0.0, jitter, size=x.shape)
    mH = MASS_D if deuterium else MASS_H
    mass = np.tile(np.array([MASS_O, mH, mH]), nmol)
    return np.ascontiguousarray(x), mass


@dataclass
class Replica:
    nmol: int
    L: float
    P: int
    T: float
    deuterium: bool
    seed: int


def replica_mix(n: int = 256, seed: int = 1, nmol_range=(32, 512), P_choices=(8, 16, 32, 64),
                T_range=(100.0, 400.0)):
    """The batched workload: n independent replicas with uneven sizes."""
    g = rng(seed)
    out = []
    lo, hi = math.log(nmol_range[0]), math.log(nmol_range[1])
    for r in range(n):
        nmol = int(round(math.exp(g.uniform(lo, hi))))
        P = int(g.choice(P_choices))
        T = float(g.uniform(*T_range))
        deut = bool(g.random() < 0.5)
        out.append(Replica(nmol, box_length(nmol), P, T, deut, int(g.integers(1, 2**62))))
    return out


@dataclass
class Job:
    arrival_s: float
    nmol: int
    P: int
    nsteps: int
    T: float
    seed: int


def serving_trace(n_jobs: int = 2000, rate_per_s: float = 50.0, seed: int = 1,
                  nmol_range=(32, 4096), P_choices=(4, 8, 16, 32, 64, 128),
                  step_range=(1000, 50000), T_range=(100.0, 400.0)):
    """Poisson stream of PIMD jobs (the serving workload)."""
    g = rng(seed)
    t = 0.0
    jobs = []
    lo, hi = math.log(nmol_range[0]), math.log(nmol_range[1])
    slo, shi = math.log(step_range[0]), math.log(step_range[1])
    for _ in range(n_jobs):
        t += float(g.exponential(1.0 / rate_per_s))
        nmol = int(round(math.exp(g.uniform(lo, hi))))
        P = int(P_choices[int(g.integers(0, len(P_choices)))])
        nsteps = int(round(math.exp(g.uniform(slo, shi))))
        T = float(g.uniform(*T_range))
        jobs.append(Job(t, nmol, P, nsteps, T, int(g.integers(1, 2**62))))
    return jobs
