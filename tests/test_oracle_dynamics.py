"""Pins of the oracle's integrator (Sec. IV.A, App. D): the P = 1 textbook
BAOAB/OBABO Langevin step, NVE conservation and time reversibility of the
exact free-ring-polymer propagation, determinism of the noise keying."""
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs

KB = 8.617333262e-5
MVV2E = 1.0364269e-4
OMEGA_HO = 0.1 / (4.135667403e-3 / (2 * math.pi))     # hbar omega = 0.1 eV


def _textbook_langevin(orc, x, v, mass, om, T, dt, tau, seed, nsteps, scheme):
    """Ten-line classical Langevin step for one bead (P = 1): no normal modes,
    no springs; the O step uses the oracle's (separately pinned) noise."""
    mm = (mass * MVV2E)[:, None]
    sig = np.sqrt(KB * T / mm)
    force = lambda y: -mm * om * om * y
    F = force(x)
    for s in range(nsteps):
        eta = lambda stream: np.array([orc.gauss3(seed, i, 0, stream, s) for i in range(len(x))])
        if scheme == "BAOAB":
            c1 = math.exp(-dt / tau); c2 = math.sqrt(1 - c1 * c1)
            v = v + 0.5 * dt * F / mm
            x = x + 0.5 * dt * v
            v = c1 * v + c2 * sig * eta(0)
            x = x + 0.5 * dt * v
            F = force(x)
            v = v + 0.5 * dt * F / mm
        else:
            c1 = math.exp(-0.5 * dt / tau); c2 = math.sqrt(1 - c1 * c1)
            v = c1 * v + c2 * sig * eta(0)
            v = v + 0.5 * dt * F / mm
            x = x + dt * v
            F = force(x)
            v = v + 0.5 * dt * F / mm
            v = c1 * v + c2 * sig * eta(1)
    return x, v


@pytest.mark.parametrize("scheme", ["BAOAB", "OBABO"])
def test_single_bead_is_textbook_langevin(orc, scheme):
    g = np.random.default_rng(11)
    N = 12
    x0 = g.normal(0, 0.1, size=(1, N, 3))
    v0 = g.normal(0, 10.0, size=(1, N, 3))
    mass = g.uniform(1.0, 3.0, size=N)
    sim = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), v0=v0,
                  thermostat=1, integrator=0 if scheme == "BAOAB" else 1, seed=9, tau=0.1)
    sim.run(50)
    x, v = _textbook_langevin(orc, x0[0], v0[0], mass, OMEGA_HO, 300.0, 2.5e-4, 0.1, 9, 50, scheme)
    assert np.abs(sim.x[0] - x).max() < 1e-12
    assert np.abs(sim.v[0] - v).max() < 1e-9


@pytest.mark.parametrize("P", [2, 3, 8, 32])
def test_free_ring_polymer_nve_conserves_energy(orc, P):
    """U = 0: the A step is the exact flow of the springs, so K + S is conserved
    to rounding for any dt (here omega_k dt up to ~2.5).  The oracle re-derives
    the modes from x every step, so the rounding of M M^T (~1e-16 .. 1e-14)
    accumulates linearly: 1e-11 over 10^4 steps."""
    g = np.random.default_rng(P)
    N = 16
    x0 = g.normal(0, 0.3, size=(P, N, 3))
    v0 = g.normal(0, 20.0, size=(P, N, 3))
    mass = g.uniform(1.0, 16.0, size=N)
    sim = orc.Sim(x0, mass, T=300.0, dt=1e-3, potential=0, ff=(0.0,), v0=v0, thermostat=0)
    e0 = sim.estimators()
    H0 = e0["K_mode"].sum() + e0["S_mode"].sum()
    sim.run(10000)
    e1 = sim.estimators()
    H1 = e1["K_mode"].sum() + e1["S_mode"].sum()
    assert abs(H1 - H0) / H0 < 1e-11
    assert e1["H"] == pytest.approx(H1, rel=1e-14)


@pytest.mark.parametrize("potential", ["free", "harmonic", "water"])
def test_nve_time_reversal(orc, potential):
    """n NVE steps, negate the normal-mode velocities, n steps: positions return."""
    P = 8
    if potential == "water":
        x0, mass = inputs.water_box(32, 10.5, P, 3, jitter=0.02)
        kw = dict(potential=1, ff=inputs.WATER_FF[:6] + (5.0,), box=(10.5,) * 3)
        dt, n = 2.5e-4, 200
    else:
        g = np.random.default_rng(2)
        x0 = g.normal(0, 0.1, size=(P, 16, 3))
        mass = np.full(16, 1.008)
        kw = dict(potential=0, ff=(0.0 if potential == "free" else OMEGA_HO,))
        dt, n = 2.5e-4, 500
    sim = orc.Sim(x0, mass, T=300.0, dt=dt, thermostat=0, seed=5, **kw)
    sim.run(n)
    sim.v[:] = -sim.v
    sim.run(n)
    assert np.abs(sim.x - x0).max() < 1e-10 * max(1.0, np.abs(x0).max())


def test_harmonic_nve_energy_bounded(orc):
    P, N = 8, 32
    g = np.random.default_rng(4)
    x0 = g.normal(0, 0.1, size=(P, N, 3))
    mass = np.full(N, 1.008)
    sim = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), thermostat=0, seed=2)
    H0 = sim.estimators()["H"]
    Hs = []
    for _ in range(20):
        sim.run(100)
        Hs.append(sim.estimators()["H"])
    assert np.max(np.abs(np.array(Hs) - H0)) / abs(H0) < 2e-3


def test_water_nve_energy_bounded(orc):
    x0, mass = inputs.water_box(64, 12.42, 4, 1, jitter=0.02)
    sim = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, potential=1, ff=inputs.WATER_FF,
                  box=(12.42,) * 3, thermostat=0, seed=1)
    e0 = sim.estimators()
    Hs = []
    for _ in range(10):
        sim.run(20)
        Hs.append(sim.estimators()["H"])
    K = e0["K_mode"].sum()
    assert np.max(np.abs(np.array(Hs) - e0["H"])) < 0.01 * K


def test_thermostat_noise_is_keyed_on_seed_and_step(orc):
    g = np.random.default_rng(5)
    x0 = g.normal(0, 0.1, size=(4, 8, 3))
    mass = np.full(8, 1.008)
    def run(seed, n1, n2):
        s = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), seed=seed, tau=0.1)
        s.run(n1)
        s.run(n2)
        return s.x.copy(), s.v.copy()
    a = run(1, 30, 0)
    b = run(1, 13, 17)          # split runs give the same trajectory (counter-based noise)
    c = run(2, 30, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.allclose(a[0], c[0])


def test_thermal_velocities(orc):
    """Initial normal-mode velocities ~ N(0, P kB T / (m mvv2e)) (ring polymer at P T)."""
    P, N, T = 8, 500, 300.0
    mass = np.full(N, 2.014)
    sim = orc.Sim(np.zeros((P, N, 3)), mass, T=T, dt=1e-3, potential=0, ff=(0.0,), seed=3)
    var = sim.v.var()
    ref = P * KB * T / (2.014 * MVV2E)
    n = sim.v.size
    assert abs(var / ref - 1) < 5 * math.sqrt(2.0 / n)
