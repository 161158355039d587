"""GPU path (FP64, through the C ABI) against the FP64 CPU oracle for the
method keywords of Sec. III.C: method pimd (Cartesian beads), fmmode normal,
fmass, sp and fixcom.  Same bars as the normal-mode parity tests: 1e-10 after 100
steps (harmonic), 1e-8 after 50 steps (water-like), estimators within them."""
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import coord_err, pimd, scalar_err  # noqa: F401
from tests.test_gpu_parity import _compare_est, _pair

pytestmark = pytest.mark.gpu

HBAR = 4.135667403e-3 / (2 * math.pi)
OMEGA_HO = 0.1 / HBAR


def _water(nmol, P, seed):
    L = inputs.box_length(nmol)
    x0, mass = inputs.water_box(nmol, L, P, seed, jitter=0.02)
    return x0, mass, dict(potential=1, ff=inputs.water_ff_for_box(L), box=(L, L, L))


def _run_both(c, g, n, bar):
    xg, vg, _ = g.get_state()
    assert coord_err(vg, c.v) < 1e-13          # initial state (thermal draw)
    c.run(n)
    g.step(n)
    xg, vg, st = g.get_state()
    assert st == n
    assert coord_err(xg, c.x) < bar
    assert coord_err(vg, c.v) < bar
    _compare_est(g.estimators(), c.estimators(), bar)


@pytest.mark.parametrize("integrator", [0, 1])
def test_cartesian_harmonic_64x8(orc, pimd, integrator):
    x0, mass = inputs.harmonic(64, 8, seed=1, std=0.1)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,),
                 integrator=integrator, method=1)
    _run_both(c, g, 100, 1e-10)


@pytest.mark.parametrize("integrator", [0, 1])
def test_cartesian_water(orc, pimd, integrator):
    x0, mass, kw = _water(16, 4, 3)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, integrator=integrator, method=1, **kw)
    _run_both(c, g, 50, 1e-8)


@pytest.mark.parametrize("fmmode,fmass", [(1, 1.0), (0, 3.0), (1, 0.5)])
def test_fictitious_masses_harmonic(orc, pimd, fmmode, fmass):
    x0, mass = inputs.harmonic(64, 8, seed=2, std=0.1)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,),
                 fmmode=fmmode, fmass=fmass, tau=0.05)
    _run_both(c, g, 100, 1e-10)


@pytest.mark.parametrize("method,integrator,sp", [(0, 0, 0.5), (0, 1, 2.0), (1, 0, 0.7), (1, 1, 1.5)])
def test_scaled_hbar_harmonic(orc, pimd, method, integrator, sp):
    """Keyword sp (hbar -> sp hbar, only omega_n changes, Eq. 2) on the FP64
    handle, normal modes and Cartesian beads, BAOAB and OBABO."""
    x0, mass = inputs.harmonic(64, 8, seed=5, std=0.1)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,),
                 integrator=integrator, method=method, sp=sp)
    _run_both(c, g, 100, 1e-10)


def test_scaled_hbar_water(orc, pimd):
    x0, mass, kw = _water(16, 8, 6)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, sp=0.6, **kw)
    _run_both(c, g, 50, 1e-8)


def test_fictitious_masses_water_obabo(orc, pimd):
    x0, mass, kw = _water(16, 8, 4)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, integrator=1, fmmode=1, fmass=2.0, **kw)
    _run_both(c, g, 50, 1e-8)


@pytest.mark.parametrize("method,integrator", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_fixcom_water(orc, pimd, method, integrator):
    x0, mass, kw = _water(16, 4, 5)
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, integrator=integrator, method=method,
                 fixcom=1, **kw)
    _run_both(c, g, 50, 1e-8)
    _, vg, _ = g.get_state()
    rows = [0] if method == 0 else range(4)
    scale = (mass[:, None] * np.abs(vg[0])).sum()
    for k in rows:
        assert np.abs((mass[:, None] * vg[k]).sum(axis=0)).max() < 1e-11 * scale


def test_cartesian_checkpoint_resume_is_bitwise(pimd):
    x0, mass, kw = _water(16, 4, 6)
    a = pimd.Simulation(x0, mass, T=300.0, dt=5e-4, method=1, fixcom=1, **kw)
    a.step(30)
    x, v, st = a.get_state()
    a.step(20)
    b = pimd.Simulation(x0, mass, T=300.0, dt=5e-4, method=1, fixcom=1, **kw)
    b.set_state(x, v, st)
    b.step(20)
    xa, va, _ = a.get_state()
    xb, vb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.parametrize("thermostat,integrator", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_bzp_barostat_water(orc, pimd, thermostat, integrator):
    """Isotropic BZP barostat (App. E), NpT (PILE_L) and NpH, BAOAB and OBABO,
    32 molecules x 4 beads, 50 steps: positions, velocities, v_W, box and
    outputs 11-15."""
    x0, mass, kw = _water(32, 4, 7)
    probe = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, thermostat=0, **kw)
    pext = probe.estimators()["P_CV"] * 0.8
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, thermostat=thermostat, barostat=1,
                 pext=pext, taup=0.05, integrator=integrator, **kw)
    _run_both(c, g, 50, 1e-8)
    vw, box = g.get_barostat()
    assert abs(vw - c.vW) < 1e-8 * max(1.0, abs(c.vW))
    assert np.abs(box - c.box).max() < 1e-10 * c.box.max()
    assert abs(box[0] / kw["box"][0] - 1.0) > 1e-6          # the box moved
    eg, ec = g.estimators(), c.estimators()
    for k in ("vW", "K_W", "U_W", "J_W", "enthalpy"):
        assert scalar_err(eg[k], ec[k]) < 1e-8, (k, eg[k], ec[k])


@pytest.mark.parametrize("integrator", [0, 1])
def test_bzp_checkpoint_resume_is_bitwise(pimd, integrator):
    x0, mass, kw = _water(32, 4, 8)
    prm = dict(T=300.0, dt=5e-4, barostat=1, pext=1e-3, taup=0.1, integrator=integrator, **kw)
    a = pimd.Simulation(x0, mass, **prm)
    a.step(30)
    x, v, st = a.get_state()
    vw, box = a.get_barostat()
    a.step(20)
    b = pimd.Simulation(x0, mass, **prm)
    b.set_barostat(vw, box)
    b.set_state(x, v, st)
    b.step(20)
    xa, va, _ = a.get_state()
    xb, vb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert a.get_barostat()[0] == b.get_barostat()[0]


@pytest.mark.parametrize("thermostat,axes,integrator", [(1, 7, 0), (0, 7, 0), (1, 4, 0), (1, 3, 0),
                                                       (1, 7, 1), (1, 2, 1)])
def test_bzp_aniso_barostat_water(orc, pimd, thermostat, axes, integrator):
    """Anisotropic BZP barostat (one v_W per edge in baro_axes), 32 molecules
    x 4 beads, 50 steps: positions, velocities, v_Wa, box and outputs 11-15;
    edges outside the mask stay exactly fixed."""
    x0, mass, kw = _water(32, 4, 9)
    probe = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, thermostat=0, **kw)
    pext = probe.estimators()["P_CV"] * 0.8
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, thermostat=thermostat, barostat=2,
                 baro_axes=axes, pext=pext, taup=0.05, integrator=integrator, **kw)
    _run_both(c, g, 50, 1e-8)
    vw, box = g.get_barostat()
    assert np.abs(vw - c.vWa).max() < 1e-8 * max(1.0, np.abs(c.vWa).max())
    assert np.abs(box - c.box).max() < 1e-10 * c.box.max()
    for a in range(3):
        if axes >> a & 1:
            assert abs(box[a] / kw["box"][a] - 1.0) > 1e-6
        else:
            assert box[a] == kw["box"][a] and vw[a] == 0.0
    eg, ec = g.estimators(), c.estimators()
    for k in ("K_W", "U_W", "J_W", "enthalpy"):
        assert scalar_err(eg[k], ec[k]) < 1e-8, (k, eg[k], ec[k])
    assert np.abs(eg["vWa"] - ec["vWa"]).max() < 1e-8 * max(1.0, np.abs(ec["vWa"]).max())
    assert eg["vW"] == 0.0


def test_bzp_aniso_checkpoint_resume_is_bitwise(pimd):
    x0, mass, kw = _water(32, 4, 10)
    prm = dict(T=300.0, dt=5e-4, barostat=2, baro_axes=5, pext=1e-3, taup=0.1, **kw)
    a = pimd.Simulation(x0, mass, **prm)
    a.step(30)
    x, v, st = a.get_state()
    vw, box = a.get_barostat()
    a.step(20)
    b = pimd.Simulation(x0, mass, **prm)
    b.set_barostat(vw, box)
    b.set_state(x, v, st)
    b.step(20)
    xa, va, _ = a.get_state()
    xb, vb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.get_barostat()[0], b.get_barostat()[0])
    with pytest.raises(pimd.PimdError):
        b.set_barostat(np.array([0.0, 1.0, 0.0]), box)      # y is outside the mask


@pytest.mark.parametrize("barostat,integrator", [(1, 0), (2, 1)])
def test_bzp_barostat_with_fixcom(orc, pimd, barostat, integrator):
    """The barostat and fixcom together: the centroid momentum removal at the
    end of each step composes with the barostat's centroid scaling."""
    x0, mass, kw = _water(32, 4, 11)
    probe = orc.Sim(x0, mass, T=300.0, dt=2.5e-4, thermostat=0, **kw)
    pext = probe.estimators()["P_CV"] * 0.9
    c, g = _pair(orc, pimd, x0, mass, T=300.0, dt=2.5e-4, barostat=barostat, pext=pext, taup=0.05,
                 integrator=integrator, fixcom=1, **kw)
    _run_both(c, g, 50, 1e-8)
    _, vg, _ = g.get_state()
    scale = (mass[:, None] * np.abs(vg[0])).sum()
    assert np.abs((mass[:, None] * vg[0]).sum(axis=0)).max() < 1e-11 * scale
