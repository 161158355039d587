"""Pins of the oracle's method keywords (Sec. III.C, App. A, App. D):
  * method pimd (Cartesian): P = 1 is the textbook Langevin step with
    tau = 1 / (2 omega_n); the Cartesian spring energy (output 2, bead form)
    sums to the normal-mode spring energy; the HO <x^2> matches the exact
    stationary covariance of the discretised Cartesian BAOAB chain; the NVE
    energy error falls as dt^2 (velocity Verlet on the springs);
  * fixcom: the centroid (or per-bead) centre-of-mass momentum vanishes, and a
    system with zero total momentum follows the same trajectory without it;
  * fmmode normal and fmass: internal modes oscillate at omega_k /
    sqrt(mu_k fmass) (omega_n for fmmode normal) in the exact free flow, and
    the HO <x^2> matches the discretised chain with the fictitious masses."""
import math

import numpy as np
import pytest
from scipy import linalg

from paper_2602_13553_gb300 import inputs
from tests.test_oracle_dynamics import _textbook_langevin

KB = 8.617333262e-5
MVV2E = 1.0364269e-4
HBAR = 4.135667403e-3 / (2 * math.pi)
OMEGA_HO = 0.1 / HBAR


def _wn(P, T):
    return P * KB * T / HBAR


def _wk(P, T):
    wn = _wn(P, T)
    return np.array([2 * wn * abs(math.sin(math.pi * k / P)) for k in range(P)])


def _stationary(P, N, T, m, om, seed, orc, cart_v=False):
    wk = _wk(P, T)
    g = np.random.default_rng(seed)
    q = g.normal(size=(P, N, 3)) * np.sqrt(P * KB * T / (m * MVV2E * (om * om + wk * wk)))[:, None, None]
    v = g.normal(size=(P, N, 3)) * math.sqrt(P * KB * T / (m * MVV2E))
    return orc.from_nm(orc.nm_matrix(P), q), v


def discrete_cartesian_x2(P, T, m, om, dt, scale=1.0):
    """<x^2> per dof of the Cartesian BAOAB chain on a harmonic well: the
    spring and well forces are diagonal in the normal modes and the Cartesian
    O step (one friction, isotropic noise) is invariant under the orthogonal
    transform, so mode k is the 2x2 velocity-Verlet map with acceleration
    -(om^2 + w_k^2) q around a friction step; S = G S G^T + b b^T."""
    wk = _wk(P, T)
    tau = scale / (2 * _wn(P, T))
    c1 = math.exp(-dt / tau)
    c2 = math.sqrt(1 - c1 * c1)
    sig = math.sqrt(P * KB * T / (m * MVV2E))
    tot = 0.0
    for k in range(P):
        w2 = om * om + wk[k] ** 2
        Bh = np.array([[1.0, 0.0], [-0.5 * dt * w2, 1.0]])
        Ah = np.array([[1.0, 0.5 * dt], [0.0, 1.0]])
        O = np.diag([1.0, c1])
        G = Bh @ Ah @ O @ Ah @ Bh
        b = Bh @ Ah @ np.array([0.0, c2 * sig])
        tot += linalg.solve_discrete_lyapunov(G, np.outer(b, b))[0, 0]
    return tot / P


def discrete_nm_x2(P, T, m, om, dt, tau, mu):
    """The normal-mode BAOAB chain with fictitious mass factors mu[k]: the
    kick of mode k is -(dt/2) om^2 q / mu_k, the exact free flow rotates at
    w_k / sqrt(mu_k), O uses tau_k = 1 / (2 w_k / sqrt(mu_k)) and the noise
    variance P kB T / (mu_k m mvv2e)."""
    wk = _wk(P, T)
    tot = 0.0
    for k in range(P):
        Bh = np.array([[1.0, 0.0], [-0.5 * dt * om * om / mu[k], 1.0]])
        W = wk[k] / math.sqrt(mu[k])
        if W == 0.0:
            Ah = np.array([[1.0, 0.5 * dt], [0.0, 1.0]])
            tk = tau
        else:
            c, s = math.cos(W * dt / 2), math.sin(W * dt / 2)
            Ah = np.array([[c, s / W], [-W * s, c]])
            tk = 1.0 / (2 * W)
        c1 = math.exp(-dt / tk)
        c2 = math.sqrt(1 - c1 * c1)
        O = np.diag([1.0, c1])
        G = Bh @ Ah @ O @ Ah @ Bh
        b = Bh @ Ah @ np.array([0.0, c2 * math.sqrt(P * KB * T / (mu[k] * m * MVV2E))])
        tot += linalg.solve_discrete_lyapunov(G, np.outer(b, b))[0, 0]
    return tot / P


@pytest.mark.parametrize("scheme", ["BAOAB", "OBABO"])
def test_cartesian_single_bead_is_textbook_langevin(orc, scheme):
    g = np.random.default_rng(21)
    N, T, dt = 10, 300.0, 2.5e-4
    x0 = g.normal(0, 0.1, size=(1, N, 3))
    v0 = g.normal(0, 10.0, size=(1, N, 3))
    mass = g.uniform(1.0, 3.0, size=N)
    sim = orc.Sim(x0, mass, T=T, dt=dt, potential=0, ff=(OMEGA_HO,), v0=v0, thermostat=1,
                  integrator=0 if scheme == "BAOAB" else 1, seed=5, method=orc.PIMD)
    sim.run(40)
    tau = 1.0 / (2 * _wn(1, T))
    x, v = _textbook_langevin(orc, x0[0], v0[0], mass, OMEGA_HO, T, dt, tau, 5, 40, scheme)
    assert np.abs(sim.x[0] - x).max() < 1e-12
    assert np.abs(sim.v[0] - v).max() < 1e-9


def test_cartesian_spring_energy_equals_normal_mode_form(orc):
    P, N, T = 6, 9, 250.0
    g = np.random.default_rng(3)
    x0 = g.normal(0, 0.2, size=(P, N, 3))
    mass = g.uniform(1.0, 16.0, size=N)
    kw = dict(T=T, dt=1e-4, potential=0, ff=(0.0,), v0=np.zeros((P, N, 3)), thermostat=0)
    cart = orc.Sim(x0, mass, method=orc.PIMD, **kw).estimators()
    nm = orc.Sim(x0, mass, method=orc.NMPIMD, **kw).estimators()
    assert cart["S_mode"].sum() == pytest.approx(nm["S_mode"].sum(), rel=1e-12)
    # per bead: neighbours shared half and half, so no bead carries it all
    assert np.all(cart["S_mode"] > 0) and not np.allclose(cart["S_mode"], nm["S_mode"])
    # the primitive estimator depends on positions only: the same in both
    assert cart["K_PR"] == pytest.approx(nm["K_PR"], rel=1e-12)


def test_cartesian_harmonic_x2_matches_discrete_chain(orc):
    P, N, T, m, dt = 8, 64, 300.0, 1.008, 2.5e-4
    x0, v0 = _stationary(P, N, T, m, OMEGA_HO, 7, orc)
    sim = orc.Sim(x0, np.full(N, m), T=T, dt=dt, potential=0, ff=(OMEGA_HO,), v0=v0,
                  thermostat=1, seed=2, method=orc.PIMD)
    sim.run(200)
    nsamp, every = 2000, 10
    acc = np.zeros(N)
    tring = []
    for _ in range(nsamp):
        sim.run(every)
        acc += (sim.x ** 2).mean(axis=(0, 2))
        tring.append(sim.estimators()["T_ring"])
    mean, se = acc.mean() / nsamp, (acc / nsamp).std(ddof=1) / math.sqrt(N)
    ref = discrete_cartesian_x2(P, T, m, OMEGA_HO, dt)
    assert abs(mean - ref) < 3 * se, (mean, ref, se)
    assert abs(np.mean(tring) - P * T) < 0.02 * P * T


def test_cartesian_nve_energy_error_is_second_order(orc):
    P, N, T = 8, 16, 300.0
    g = np.random.default_rng(9)
    x0, v0 = _stationary(P, N, T, 1.008, OMEGA_HO, 9, orc)
    v0 = g.normal(size=(P, N, 3)) * math.sqrt(P * KB * T / (1.008 * MVV2E))
    errs = []
    for dt in (2e-4, 1e-4):
        sim = orc.Sim(x0, np.full(N, 1.008), T=T, dt=dt, potential=0, ff=(OMEGA_HO,), v0=v0,
                      thermostat=0, method=orc.PIMD)
        H0 = sim.estimators()["H"]
        dev = 0.0
        for _ in range(int(round(0.2 / dt / 10))):
            sim.run(10)
            dev = max(dev, abs(sim.estimators()["H"] - H0))
        errs.append(dev / abs(H0))
    assert errs[0] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def _water(nmol, P, seed):
    L = inputs.box_length(nmol)
    x0, mass = inputs.water_box(nmol, L, P, seed, jitter=0.02)
    return x0, mass, dict(potential=1, ff=inputs.water_ff_for_box(L), box=(L, L, L))


@pytest.mark.parametrize("method", [0, 1])
def test_fixcom_zeroes_centre_of_mass_momentum(orc, method):
    P, nmol = 4, 16
    x0, mass, kw = _water(nmol, P, 31)
    common = dict(T=300.0, dt=5e-4, thermostat=1, seed=3, method=method, **kw)
    on = orc.Sim(x0, mass, fixcom=1, **common)
    off = orc.Sim(x0, mass, fixcom=0, **common)
    on.run(25)
    off.run(25)
    rows = [0] if method == 0 else range(P)
    ptot = lambda s, k: (mass[:, None] * s.v[k]).sum(axis=0)
    scale = (mass[:, None] * np.abs(on.v[0])).sum()
    for k in rows:
        assert np.abs(ptot(on, k)).max() < 1e-12 * scale
        assert np.abs(ptot(off, k)).max() > 1e-3 * scale
    if method == 0:   # the internal modes carry no centre-of-mass motion to remove
        assert np.abs(ptot(on, 1)).max() > 1e-3 * scale


def test_fixcom_is_inert_at_zero_momentum(orc):
    """Normal modes, NVE, zero centroid momentum (conserved: the forces sum to
    zero): the removal only takes off rounding.  (Per-bead Cartesian momenta
    are not conserved -- the springs exchange momentum between beads.)"""
    method = 0
    P, nmol = 4, 8
    x0, mass, kw = _water(nmol, P, 32)
    v0 = np.random.default_rng(4).normal(0, 5.0, size=x0.shape)
    v0[0] -= (mass[:, None] * v0[0]).sum(axis=0) / mass.sum()
    runs = []
    for fc in (0, 1):
        s = orc.Sim(x0, mass, T=300.0, dt=5e-4, v0=v0, thermostat=0, method=method, fixcom=fc, **kw)
        s.run(30)
        runs.append(s.x.copy())
    assert np.abs(runs[0] - runs[1]).max() < 1e-11


@pytest.mark.parametrize("fmmode,fmass", [(1, 1.0), (0, 2.5), (1, 0.5)])
def test_internal_modes_oscillate_at_fictitious_frequency(orc, fmmode, fmass):
    """Free ring polymer, NVE: each excited mode follows the exact harmonic
    flow q~_k(t) = A cos(W_k t) with W_k = w_k / sqrt(mu_k fmass)."""
    P, N, T, dt, n = 8, 3, 300.0, 1e-4, 37
    M = orc.nm_matrix(P)
    q = np.zeros((P, N, 3))
    A = 0.05
    q[1:, :, :] = A
    sim = orc.Sim(orc.from_nm(M, q), np.full(N, 2.0), T=T, dt=dt, potential=0, ff=(0.0,),
                  v0=np.zeros((P, N, 3)), thermostat=0, fmmode=fmmode, fmass=fmass)
    sim.run(n)
    qt = orc.to_nm(M, sim.x)
    lam = np.array([4 * math.sin(math.pi * k / P) ** 2 for k in range(P)])
    mu = (lam if fmmode == 1 else np.ones(P)) * fmass
    mu[0] = fmass
    for k in range(1, P):
        W = _wk(P, T)[k] / math.sqrt(mu[k])
        assert qt[k] == pytest.approx(np.full((N, 3), A * math.cos(W * n * dt)), abs=1e-12)
        assert sim.v[k] == pytest.approx(np.full((N, 3), -A * W * math.sin(W * n * dt)), rel=1e-9)
    if fmmode == 1:   # every internal mode at omega_n
        assert np.allclose(_wk(P, T)[1:] / np.sqrt(mu[1:] / fmass), _wn(P, T))


def test_normal_mode_masses_harmonic_x2_matches_discrete_chain(orc):
    P, N, T, m, dt, tau = 8, 64, 300.0, 1.008, 2.5e-4, 0.05
    x0, v0 = _stationary(P, N, T, m, OMEGA_HO, 11, orc)
    lam = np.array([4 * math.sin(math.pi * k / P) ** 2 for k in range(P)])
    mu = lam.copy()
    mu[0] = 1.0
    v0 = v0 / np.sqrt(mu)[:, None, None]
    sim = orc.Sim(x0, np.full(N, m), T=T, dt=dt, potential=0, ff=(OMEGA_HO,), v0=v0,
                  thermostat=1, seed=6, tau=tau, fmmode=1)
    sim.run(200)
    nsamp, every = 2000, 10
    acc = np.zeros(N)
    tring = []
    for _ in range(nsamp):
        sim.run(every)
        acc += (sim.x ** 2).mean(axis=(0, 2))
        tring.append(sim.estimators()["T_ring"])
    mean, se = acc.mean() / nsamp, (acc / nsamp).std(ddof=1) / math.sqrt(N)
    ref = discrete_nm_x2(P, T, m, OMEGA_HO, dt, tau, mu)
    assert abs(mean - ref) < 3 * se, (mean, ref, se)
    assert abs(np.mean(tring) - P * T) < 0.02 * P * T


# ---- BZP barostat (App. E), isotropic, BAOAB, normal modes ------------------

def _bonded_water(nmol, P, seed, L=None):
    L = L or inputs.box_length(nmol)
    x0, mass = inputs.water_box(nmol, L, P, seed, jitter=0.02)
    ff = list(inputs.water_ff_for_box(L))
    ff[4] = 0.0          # no Lennard-Jones: no cutoff discontinuity in the energy
    return x0, mass, dict(potential=1, ff=ff, box=(L, L, L))


def test_bzp_frozen_barostat_is_the_plain_integrator(orc):
    """W -> infinity with v_W = 0: the barostat never moves and the step is the
    normal-mode BAOAB step (the centroid propagator's sinh(a)/v_W -> tA)."""
    x0, mass, kw = _bonded_water(8, 4, 41)
    common = dict(T=300.0, dt=5e-4, thermostat=1, seed=2, **kw)
    a = orc.Sim(x0, mass, barostat=1, pext=1e-3, taup=1e9, **common)
    b = orc.Sim(x0, mass, **common)
    a.run(40)
    b.run(40)
    assert abs(a.vW) < 1e-9          # only the thermal kicks of a huge W
    assert np.abs(a.x - b.x).max() < 1e-12 and np.abs(a.v - b.v).max() < 1e-9


def test_bzp_nph_conserves_the_extended_enthalpy(orc):
    """NpH (no thermostat): output 15, H + K_W + U_W + J_W, is conserved with a
    second-order error; this fixes the n kB T reading of the barostat force and
    the exact kick terms (any other force on v_W drifts at first order)."""
    x0, mass, kw = _bonded_water(16, 4, 42)
    probe = orc.Sim(x0, mass, T=300.0, dt=1e-4, thermostat=0, **kw)
    pext = probe.estimators()["P_CV"]      # start near mechanical balance
    errs = []
    for dt in (2e-4, 1e-4):
        s = orc.Sim(x0, mass, T=300.0, dt=dt, thermostat=0, barostat=1, pext=pext, taup=0.02, vW=2.0, **kw)
        e0 = s.estimators()["enthalpy"]
        dev = 0.0
        for _ in range(int(round(0.04 / dt / 10))):
            s.run(10)
            dev = max(dev, abs(s.estimators()["enthalpy"] - e0))
        errs.append(dev)
        assert abs(s.box[0] / kw["box"][0] - 1.0) > 1e-3     # the box did move
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_bzp_npt_ideal_gas_volume(orc):
    """NpT, free atoms in a periodic box: <V> = (N + 1) kB T / P_ext (the
    isothermal-isobaric measure with dV; the J_W term makes the + 1)."""
    P, N, T = 4, 6, 300.0
    L0 = 10.0
    g = np.random.default_rng(5)
    x0 = np.repeat(g.uniform(0, L0, size=(1, N, 3)), P, axis=0) + g.normal(0, 0.05, size=(P, N, 3))
    mass = np.full(N, 16.0)
    ff = (0.0, 1.0, 0.0, 1.8, 0.0, 1.0, 0.5)      # every force constant zero
    pext = (N + 1) * KB * T / L0 ** 3
    s = orc.Sim(x0, mass, T=T, dt=2e-3, potential=1, ff=ff, box=(L0, L0, L0), thermostat=1, tau=0.05,
                seed=9, barostat=1, pext=pext, taup=0.05)
    s.run(2000)
    vols = []
    for _ in range(3000):
        s.run(20)
        vols.append(s.box.prod())
    from tests._stats import block_mean_sigma
    mu, sig = block_mean_sigma(vols, 30)
    target = (N + 1) * KB * T / pext
    assert abs(mu - target) < 3 * sig, (mu, target, sig)
    assert abs(mu - N * KB * T / pext) > 3 * sig        # distinguishes the + 1


# ---- BZP barostat (App. E), anisotropic: one v_W per box edge --------------

def test_bzp_aniso_nph_conserves_the_extended_enthalpy(orc):
    """NpH with all three edges free: output 15 (with K_W summed over the axes
    and J_W = -n kB T sum_a ln L_a) is conserved with a second-order error, and
    the three edges move apart from one another."""
    x0, mass, kw = _bonded_water(16, 4, 43)
    probe = orc.Sim(x0, mass, T=300.0, dt=1e-4, thermostat=0, **kw)
    pext = probe.estimators()["P_CV"]
    errs = []
    for dt in (2e-4, 1e-4):
        s = orc.Sim(x0, mass, T=300.0, dt=dt, thermostat=0, barostat=2, baro_axes=7, pext=pext,
                    taup=0.02, **kw)
        e0 = s.estimators()["enthalpy"]
        dev = 0.0
        for _ in range(int(round(0.04 / dt / 10))):
            s.run(10)
            dev = max(dev, abs(s.estimators()["enthalpy"] - e0))
        errs.append(dev)
        rel = s.box / kw["box"][0] - 1.0
        assert np.abs(rel).min() > 1e-4                     # every edge moved
        assert np.ptp(rel) > 1e-4                           # and not together
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_bzp_aniso_masked_axes_stay_fixed(orc):
    """baro_axes = z: v_Wx = v_Wy = 0 and L_x, L_y unchanged through NpT; the
    x and y centroid components then follow the barostat-free step."""
    x0, mass, kw = _bonded_water(8, 4, 44)
    s = orc.Sim(x0, mass, T=300.0, dt=5e-4, thermostat=1, seed=3, barostat=2, baro_axes=4,
                pext=1e-3, taup=0.05, **kw)
    s.run(60)
    assert s.vWa[0] == 0.0 and s.vWa[1] == 0.0 and s.vWa[2] != 0.0
    assert s.box[0] == kw["box"][0] and s.box[1] == kw["box"][1]
    assert s.box[2] != kw["box"][2]


def test_bzp_aniso_one_axis_ideal_gas_length(orc):
    """NpT, free atoms, only L_z free: L_z samples L^N exp(-P_ext A L / kB T) dL,
    so <L_z> = (N + 1) kB T / (P_ext L_x L_y)."""
    P, N, T = 4, 6, 300.0
    L0 = 10.0
    g = np.random.default_rng(6)
    x0 = np.repeat(g.uniform(0, L0, size=(1, N, 3)), P, axis=0) + g.normal(0, 0.05, size=(P, N, 3))
    mass = np.full(N, 16.0)
    ff = (0.0, 1.0, 0.0, 1.8, 0.0, 1.0, 0.5)
    pext = (N + 1) * KB * T / L0 ** 3
    s = orc.Sim(x0, mass, T=T, dt=2e-3, potential=1, ff=ff, box=(L0, L0, L0), thermostat=1, tau=0.05,
                seed=11, barostat=2, baro_axes=4, pext=pext, taup=0.05)
    s.run(2000)
    lz = []
    for _ in range(3000):
        s.run(20)
        lz.append(s.box[2])
    from tests._stats import block_mean_sigma
    mu, sig = block_mean_sigma(lz, 30)
    target = (N + 1) * KB * T / (pext * L0 * L0)
    assert abs(mu - target) < 3 * sig, (mu, target, sig)
    assert abs(mu - N * KB * T / (pext * L0 * L0)) > 3 * sig


# ---- BZP barostat with OBABO -------------------------------------------------

@pytest.mark.parametrize("barostat", [1, 2])
def test_bzp_obabo_nph_is_the_baoab_nph(orc, barostat):
    """Without a thermostat OBABO is B A(h) B and BAOAB is B A(h/2) A(h/2) B:
    the barostat's centroid flow composes exactly (e^a e^a = e^2a, and the
    sinh form of two halves at one v_W is the sinh form of the whole), so the
    two NpH trajectories agree to rounding."""
    x0, mass, kw = _bonded_water(8, 4, 45)
    common = dict(T=300.0, dt=2e-4, thermostat=0, barostat=barostat, pext=1e-3, taup=0.05, vW=0.5, **kw)
    a = orc.Sim(x0, mass, integrator=0, **common)
    b = orc.Sim(x0, mass, integrator=1, **common)
    a.run(60)
    b.run(60)
    assert np.abs(a.x - b.x).max() < 1e-11 and np.abs(a.v - b.v).max() < 1e-8
    assert np.abs(a.box - b.box).max() < 1e-11 * a.box.max()
    assert abs(a.box[0] / kw["box"][0] - 1.0) > 1e-5


def test_bzp_obabo_npt_ideal_gas_volume(orc):
    """NpT with OBABO (two O(h/2) per step on particles and on v_W): free atoms
    give <V> = (N + 1) kB T / P_ext as with BAOAB."""
    P, N, T = 4, 6, 300.0
    L0 = 10.0
    g = np.random.default_rng(7)
    x0 = np.repeat(g.uniform(0, L0, size=(1, N, 3)), P, axis=0) + g.normal(0, 0.05, size=(P, N, 3))
    mass = np.full(N, 16.0)
    ff = (0.0, 1.0, 0.0, 1.8, 0.0, 1.0, 0.5)
    pext = (N + 1) * KB * T / L0 ** 3
    s = orc.Sim(x0, mass, T=T, dt=2e-3, potential=1, ff=ff, box=(L0, L0, L0), thermostat=1, tau=0.05,
                seed=13, barostat=1, pext=pext, taup=0.05, integrator=1)
    s.run(2000)
    vols = []
    for _ in range(3000):
        s.run(20)
        vols.append(s.box.prod())
    from tests._stats import block_mean_sigma
    mu, sig = block_mean_sigma(vols, 30)
    target = (N + 1) * KB * T / pext
    assert abs(mu - target) < 3 * sig, (mu, target, sig)
    assert abs(mu - N * KB * T / pext) > 3 * sig
