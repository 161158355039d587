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
    step count log-uniform in [1000, 50000].
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
    capped at 0.48 L in boxes too small for minimum-image interactions at 6 A
    (the 32-molecule boxes of the mixes are 9.86 A)."""
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


def _random_rotation(g: np.random.Generator) -> np.ndarray:
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def water_box(nmol: int, L: float, P: int, seed: int, *, r_oo_min: float = 2.5,
              r0: float = 1.0, theta0_deg: float = 104.5, jitter: float = 0.0,
              deuterium: bool = False):
    """Return (x [P][3*nmol][3], mass [3*nmol]) for a random water-like box.

    Atoms are ordered O, H, H per molecule.  Coordinates are unwrapped (the O
    lies in [0, L)^3; hydrogens may stick out by a bond length)."""
    g = rng(seed)
    O = np.zeros((nmol, 3))
    n = 0
    attempts = 0
    while n < nmol:
        attempts += 1
        if attempts > 2000 * max(nmol, 1):
            raise RuntimeError("water_box: could not place %d molecules in L=%.3f" % (nmol, L))
        p = g.uniform(0.0, L, size=3)
        if n:
            d = O[:n] - p
            d -= L * np.rint(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < r_oo_min * r_oo_min:
                continue
        O[n] = p
        n += 1
    half = math.radians(theta0_deg) / 2.0
    h1 = r0 * np.array([math.sin(half), math.cos(half), 0.0])
    h2 = r0 * np.array([-math.sin(half), math.cos(half), 0.0])
    x1 = np.zeros((3 * nmol, 3))
    for m in range(nmol):
        R = _random_rotation(g)
        x1[3 * m] = O[m]
        x1[3 * m + 1] = O[m] + R @ h1
        x1[3 * m + 2] = O[m] + R @ h2
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
