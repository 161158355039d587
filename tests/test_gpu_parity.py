"""GPU path (through the C ABI) against the FP64 CPU oracle, element by
element on the same seeded inputs.  Bars: positions and normal-mode
velocities within 1e-10 (per-coordinate relative, RMS floor) after 100 steps
for harmonic systems, within 1e-8 after 50 steps for water-like systems;
estimators within the same bars."""
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import coord_err, pimd, scalar_err  # noqa: F401

pytestmark = pytest.mark.gpu

HBAR = 4.135667403e-3 / (2 * math.pi)
OMEGA_HO = 0.1 / HBAR
EST_KEYS = ("H", "K_PR", "K_VR", "K_CV", "T_ring")
PRESS_KEYS = ("P_PR", "P_MD", "P_CV")


def _pair(orc, pimd, x0, mass, v0=None, **kw):
    integ = kw.pop("integrator", 0)
    thermo = kw.pop("thermostat", 1)
    seed = kw.pop("seed", 1)
    tau = kw.pop("tau", 1.0)
    sim_c = orc.Sim(x0, mass, v0=v0, integrator=integ, thermostat=thermo, seed=seed, tau=tau, **kw)
    sim_g = pimd.Simulation(x0, mass, v0=v0, integrator=integ, thermostat=thermo, seed=seed, tau=tau, **kw)
    return sim_c, sim_g


def _compare_est(eg, ec, tol):
    for k in EST_KEYS:
        assert scalar_err(eg[k], ec[k]) < tol, (k, eg[k], ec[k])
    for k in ("K_mode", "S_mode", "U_bead"):
        assert coord_err(eg[k], ec[k]) < tol, k
    for k in PRESS_KEYS:
        if math.isnan(ec[k]):
            assert math.isnan(eg[k])
        else:
            # pressures are differences of large terms: compare against the scale of the terms
            scale = abs(ec["vir_sum"]) / (3 * ec["volume"]) + abs(ec[k])
            assert abs(eg[k] - ec[k]) < tol * scale, (k, eg[k], ec[k])


def test_harmonic_oscillators_64x8(orc, pimd):
    """64 independent 3D oscillators, m = 1.008, hbar w = 0.1 eV, T = 300 K,
    P = 8, dt = 0.25 fs, centroid tau = 1 ps, critically damped internal
    modes, seeded Gaussian positions, Philox seed 1 (thermal velocities from
    the same keyed stream on both sides)."""
    x0, mass = inputs.harmonic(64, 8, seed=1, std=0.1)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,))
    xg, vg, _ = g.get_state()
    assert coord_err(vg, c.v) < 1e-13        # initial thermal draw
    c.run(100)
    g.step(100)
    xg, vg, st = g.get_state()
    assert st == 100
    assert coord_err(xg, c.x) < 1e-10
    assert coord_err(vg, c.v) < 1e-10
    _compare_est(g.estimators(), c.estimators(), 1e-10)
    # the full 2000-step run of this workload stays on the oracle
    c.run(1900)
    g.step(1900)
    xg, vg, st = g.get_state()
    assert st == 2000
    assert coord_err(xg, c.x) < 1e-9 and coord_err(vg, c.v) < 1e-9


CASES = [
    # P, N, integrator, thermostat
    (1, 5, 0, 1), (2, 37, 0, 1), (3, 37, 1, 1), (5, 300, 0, 0), (7, 1, 1, 1),
    (8, 700, 1, 1), (16, 131, 0, 1), (32, 70, 1, 0), (64, 19, 0, 1), (100, 9, 1, 1),
    (128, 11, 0, 1), (128, 3, 1, 1),
    # grids of >= 4 x 152 blocks: one Philox draw per (atom, mode) in a pre-pass
    (8, 6500, 0, 1), (8, 6500, 1, 1),
]


@pytest.mark.parametrize("P,N,integ,thermo", CASES)
def test_harmonic_shapes_and_splittings(orc, pimd, P, N, integ, thermo):
    """Ragged atom counts (one to many tiles), odd and even P up to 128, both
    splittings, NVE and PILE_L; explicit initial velocities."""
    g0 = np.random.default_rng(P * 1000 + N)
    x0 = g0.normal(0, 0.1, size=(P, N, 3))
    v0 = g0.normal(0, 10.0, size=(P, N, 3))
    mass = g0.choice([1.008, 2.014, 15.999], size=N)
    c, g = _pair(orc, pimd, x0, mass, v0=v0, T=250.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,),
                 integrator=integ, thermostat=thermo, seed=7, tau=0.3)
    c.run(100)
    g.step(60)
    g.step(40)
    xg, vg, st = g.get_state()
    assert st == 100
    assert coord_err(xg, c.x) < 1e-10
    assert coord_err(vg, c.v) < 1e-10
    _compare_est(g.estimators(), c.estimators(), 1e-10)


def _water(nmol, L, P, seed, jitter=0.02):
    return inputs.water_box(nmol, L, P, seed, jitter=jitter)


@pytest.mark.parametrize("integ", [0, 1])
def test_water_64_molecules_P32(orc, pimd, integ):
    """64 water-like molecules in a 12.42 A periodic box (1 g/cm^3), P = 32,
    T = 300 K, dt = 0.5 fs, 50 steps."""
    x0, mass = _water(64, 12.42, 32, 1)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF,
                 box=(12.42,) * 3, integrator=integ)
    c.run(50)
    g.step(50)
    xg, vg, st = g.get_state()
    assert coord_err(xg, c.x) < 1e-8
    assert coord_err(vg, c.v) < 1e-8
    _compare_est(g.estimators(), c.estimators(), 1e-8)


def _skin_crossed(c, nmol, L, steps, skin=1.5):
    """Step the oracle one step at a time and report whether the list
    criterion 2 (centroid drift + bead spread) > skin of the oxygens, counted
    from the initial centroids, is crossed: then the device must have rebuilt
    its lists at least once during the run."""
    def centroids(x):
        return x[:, 0:3 * nmol:3, :].mean(axis=0)
    c0 = centroids(c.x)
    crossed = False
    for _ in range(steps):
        c.run(1)
        cc = centroids(c.x)
        d = cc - c0
        d -= L * np.rint(d / L)
        drift = np.sqrt((d * d).sum(axis=1)).max()
        spread = np.sqrt(((c.x[:, 0:3 * nmol:3, :] - cc[None]) ** 2).sum(axis=2)).max()
        crossed |= 2.0 * (drift + spread) > skin
    return crossed


def test_water_large_box_neighbour_rebuilds(orc, pimd):
    """512 molecules (24.84 A box): the O-O list is a genuine subset, and a
    hot start (900 K) crosses the skin criterion near step 53 of the 80, so
    the lists are rebuilt during the run (one bead chunk per molecule)."""
    x0, mass = _water(512, 24.84, 4, 2, jitter=0.05)
    c, g = _pair(orc, pimd, x0, mass, T=900.0, dt=5e-4, potential=1, ff=inputs.WATER_FF,
                 box=(24.84,) * 3, tau=0.05)
    assert _skin_crossed(c, 512, 24.84, 80)
    g.step(80)
    xg, vg, _ = g.get_state()
    assert coord_err(xg, c.x) < 1e-8
    assert coord_err(vg, c.v) < 1e-8
    _compare_est(g.estimators(), c.estimators(), 1e-8)


@pytest.mark.parametrize("P", [40, 64])
def test_water_two_bead_chunks_neighbour_rebuilds(orc, pimd, P):
    """More than 32 beads: two bead chunks per molecule, each cluster of the
    force kernel rebuilding the same list; a hot start (900 K, 0.05 A
    jitter) crosses the skin near step 55 of the 80, so the lists are
    rebuilt on the device."""
    nmol = 96
    L = inputs.box_length(nmol)
    x0, mass = _water(nmol, L, P, 5, jitter=0.05)
    c, g = _pair(orc, pimd, x0, mass, T=900.0, dt=5e-4, potential=1, ff=inputs.water_ff_for_box(L),
                 box=(L,) * 3, tau=0.05)
    assert _skin_crossed(c, nmol, L, 80)
    g.step(80)
    xg, vg, _ = g.get_state()
    assert coord_err(xg, c.x) < 1e-8
    assert coord_err(vg, c.v) < 1e-8
    _compare_est(g.estimators(), c.estimators(), 1e-8)


def test_checkpoint_resume_is_bitwise(pimd):
    x0, mass = _water(64, 12.42, 8, 3)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(12.42,) * 3, seed=11)
    a = pimd.Simulation(x0, mass, **kw)
    a.step(40)
    xs, vs, st = a.get_state()
    a.step(40)
    xa, va, _ = a.get_state()
    b = pimd.Simulation(x0, mass, **kw)
    b.set_state(xs, vs, st)
    b.step(40)
    xb, vb, stb = b.get_state()
    assert stb == 80
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_deterministic_and_graph_invariant(pimd, monkeypatch):
    x0, mass = _water(64, 12.42, 16, 4)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(12.42,) * 3, seed=3)
    runs = []
    for env in ("0", "0", "1"):
        monkeypatch.setenv("PIMD_NO_GRAPH", env)
        s = pimd.Simulation(x0, mass, **kw)
        s.step(37)
        runs.append(s.get_state())
        s.close()
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and np.array_equal(r[1], runs[0][1])


def test_zero_steps_and_errors(pimd):
    x0, mass = inputs.harmonic(4, 2, seed=1, std=0.1)
    s = pimd.Simulation(x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,))
    x, v, st = s.get_state()
    s.step(0)
    x2, v2, st2 = s.get_state()
    assert st == st2 == 0 and np.array_equal(x, x2) and np.array_equal(v, v2)
    with pytest.raises(pimd.PimdError):
        s.step(-1)
