"""Statistical pins of the oracle (Sec. IV.A, App. A, App. D):
  * the P-bead harmonic-oscillator <x^2> against the exact stationary
    covariance of the discretised BAOAB map (discrete Lyapunov equation) and
    against the continuous finite-P closed form;
  * K_CV = K_VR = K_PR = 1/2 m w^2 <x^2> on the oscillator;
  * equipartition at P T of every PILE_L-thermostatted mode (free ring polymer);
  * free particles in a box: K_PR = 3 N kB T / 2 and P_CV = P_PR = N kB T / V.
Atoms are independent replicas, so the standard error comes from the spread
of per-atom time averages (no autocorrelation estimate needed)."""
import math

import numpy as np
import pytest
from scipy import linalg

from tests._stats import block_mean_sigma

KB = 8.617333262e-5
MVV2E = 1.0364269e-4
HBAR = 4.135667403e-3 / (2 * math.pi)
OMEGA_HO = 0.1 / HBAR


def _modes(P, T):
    wn = P * KB * T / HBAR
    return wn, np.array([2 * wn * abs(math.sin(math.pi * k / P)) for k in range(P)])


def discrete_baoab_x2(P, T, m, om, dt, tau, scale=1.0):
    """<x^2> per Cartesian dof of the discretised BAOAB chain for a harmonic
    oscillator: each normal mode is an independent linear map z' = G z + b eta,
    whose stationary covariance solves S = G S G^T + b b^T."""
    wn, wk = _modes(P, T)
    sig2 = P * KB * T / (m * MVV2E)
    tot = 0.0
    for k in range(P):
        Bh = np.array([[1.0, 0.0], [-0.5 * dt * om * om, 1.0]])
        if wk[k] == 0.0:
            Ah = np.array([[1.0, 0.5 * dt], [0.0, 1.0]])
            tk = tau
        else:
            c, s = math.cos(wk[k] * dt / 2), math.sin(wk[k] * dt / 2)
            Ah = np.array([[c, s / wk[k]], [-wk[k] * s, c]])
            tk = scale / (2 * wk[k])
        c1 = math.exp(-dt / tk)
        c2 = math.sqrt(1 - c1 * c1)
        O = np.diag([1.0, c1])
        G = Bh @ Ah @ O @ Ah @ Bh
        b = Bh @ Ah @ np.array([0.0, c2 * math.sqrt(sig2)])
        S = linalg.solve_discrete_lyapunov(G, np.outer(b, b))
        tot += S[0, 0]
    return tot / P


def continuous_x2(P, T, m, om):
    _, wk = _modes(P, T)
    return KB * T / (m * MVV2E) * np.sum(1.0 / (om * om + wk * wk))


def stationary_init(orc, P, N, T, m, om, seed):
    wn, wk = _modes(P, T)
    g = np.random.default_rng(seed)
    q = g.normal(size=(P, N, 3)) * np.sqrt(P * KB * T / (m * MVV2E * (om * om + wk * wk)))[:, None, None]
    v = g.normal(size=(P, N, 3)) * math.sqrt(P * KB * T / (m * MVV2E))
    M = orc.nm_matrix(P)
    return orc.from_nm(M, q), v


def test_closed_form_values():
    """The finite-P closed form converges to hbar/(2 m w) coth(beta hbar w / 2)."""
    m, T = 1.008, 300.0
    x2_8 = continuous_x2(8, T, m, OMEGA_HO)
    assert x2_8 == pytest.approx(0.0210475, rel=2e-5)
    exact = HBAR / (2 * m * MVV2E * OMEGA_HO) / math.tanh(0.1 / (2 * KB * T))
    assert exact == pytest.approx(0.0216200, rel=2e-5)
    assert continuous_x2(4096, T, m, OMEGA_HO) == pytest.approx(exact, rel=1e-5)


@pytest.mark.parametrize("P,tau", [(8, 0.05), (4, 0.05)])
def test_harmonic_x2_matches_discrete_closed_form(orc, P, tau):
    N, T, m, dt = 64, 300.0, 1.008, 2.5e-4
    x0, v0 = stationary_init(orc, P, N, T, m, OMEGA_HO, seed=100 + P)
    sim = orc.Sim(x0, np.full(N, m), T=T, dt=dt, potential=0, ff=(OMEGA_HO,), v0=v0,
                  thermostat=1, seed=1, tau=tau)
    nsamp, every = 2000, 10
    acc = np.zeros(N)
    kcv, kvr, kpr, tring = [], [], [], []
    for _ in range(nsamp):
        sim.run(every)
        acc += (sim.x ** 2).mean(axis=(0, 2))
        e = sim.estimators()
        kcv.append(e["K_CV"]); kvr.append(e["K_VR"]); kpr.append(e["K_PR"]); tring.append(e["T_ring"])
    per_atom = acc / nsamp
    mean, se = per_atom.mean(), per_atom.std(ddof=1) / math.sqrt(N)
    ref = discrete_baoab_x2(P, T, m, OMEGA_HO, dt, tau)
    assert abs(mean - ref) < 3 * se, (mean, ref, se)
    # the discretisation bias at dt = 0.25 fs is far below the sampling error
    assert abs(ref - continuous_x2(P, T, m, OMEGA_HO)) < 0.2 * se
    # App. A estimators: virial theorem for the harmonic well
    kref = 3 * N * 0.5 * m * MVV2E * OMEGA_HO ** 2 * ref
    for series in (kcv, kvr, kpr):
        mu, s = block_mean_sigma(series, 20)
        assert abs(mu - kref) < 3 * s + 1e-3 * kref, (mu, kref, s)
    mu, s = block_mean_sigma(tring, 20)
    assert abs(mu - P * T) < 3 * s


def test_free_ring_polymer_equipartition(orc):
    """Every mode: <1/2 m v~_k^2> = 1/2 P kB T per dof; k >= 1: the spring
    energy of the mode too (exact for any dt: A and O preserve the free Gibbs
    measure)."""
    P, N, T, dt = 8, 64, 300.0, 1e-3
    mass = np.random.default_rng(0).choice([1.008, 2.014, 15.999], size=N)
    wn, wk = _modes(P, T)
    g = np.random.default_rng(1)
    # collapsed ring polymers, thermal velocities: burn in before sampling
    x0 = np.repeat(g.uniform(-1, 1, size=(1, N, 3)), P, axis=0)
    sim = orc.Sim(x0, mass, T=T, dt=dt, potential=0, ff=(0.0,), thermostat=1, seed=4, tau=0.02)
    sim.run(200)
    M = orc.nm_matrix(P)
    nsamp = 1500
    K = np.zeros((P, N))
    S = np.zeros((P, N))
    mm = mass * MVV2E
    for _ in range(nsamp):
        sim.run(4)
        q = orc.to_nm(M, sim.x)
        K += 0.5 * mm[None, :] * (sim.v ** 2).sum(axis=2)
        S += 0.5 * mm[None, :] * (wk ** 2)[:, None] * (q ** 2).sum(axis=2)
    K /= nsamp
    S /= nsamp
    target = 1.5 * P * KB * T       # per atom (3 dof)
    for k in range(P):
        se = K[k].std(ddof=1) / math.sqrt(N)
        assert abs(K[k].mean() - target) < 3 * se, (k, K[k].mean(), target, se)
        if k > 0:
            se = S[k].std(ddof=1) / math.sqrt(N)
            assert abs(S[k].mean() - target) < 3 * se, (k, S[k].mean(), target, se)


def test_free_particles_pressure_and_primitive_kinetic(orc):
    """U = 0 in a periodic box: <K_PR> = 3 N kB T / 2 (needs the 1/P reading of
    the spring term) and <P_CV> = <P_PR> = N kB T / V (needs the 1/P reading of
    P_PR); P_MD as printed is the pressure of the extended system, N P
    particles at P T: P^2 N kB T / V."""
    P, N, T, dt, L = 4, 64, 300.0, 1e-3, 20.0
    g = np.random.default_rng(2)
    x0 = np.repeat(g.uniform(0, L, size=(1, N, 3)), P, axis=0)
    sim = orc.Sim(x0, np.full(N, 2.014), T=T, dt=dt, potential=0, ff=(0.0,), box=(L, L, L),
                  thermostat=1, seed=8, tau=0.02)
    sim.run(300)
    kpr, pcv, ppr, pmd = [], [], [], []
    for _ in range(4000):
        sim.run(2)
        e = sim.estimators()
        kpr.append(e["K_PR"]); pcv.append(e["P_CV"]); ppr.append(e["P_PR"]); pmd.append(e["P_MD"])
    V = L ** 3
    for series, ref in ((kpr, 1.5 * N * KB * T), (pcv, N * KB * T / V), (ppr, N * KB * T / V),
                        (pmd, P * P * N * KB * T / V)):
        mu, s = block_mean_sigma(series, 20)
        assert abs(mu - ref) < 3 * s, (mu, ref, s)


def test_mode_energies_reported_by_estimators(orc):
    """Outputs 1-2 of App. A on the free ring polymer: <K^(k)> = <S^(k>=1)> =
    3 N P kB T / 2 (pins the m w_n^2 reading of the spring term)."""
    P, N, T = 4, 48, 300.0
    g = np.random.default_rng(3)
    x0 = np.repeat(g.uniform(-1, 1, size=(1, N, 3)), P, axis=0)
    sim = orc.Sim(x0, np.full(N, 1.008), T=T, dt=1e-3, potential=0, ff=(0.0,),
                  thermostat=1, seed=6, tau=0.02)
    sim.run(200)
    Ks, Ss = [], []
    for _ in range(3000):
        sim.run(3)
        e = sim.estimators()
        Ks.append(e["K_mode"]); Ss.append(e["S_mode"])
    Ks, Ss = np.array(Ks), np.array(Ss)
    target = 1.5 * N * P * KB * T
    for k in range(P):
        mu, s = block_mean_sigma(Ks[:, k], 20)
        assert abs(mu - target) < 3 * s
        if k:
            mu, s = block_mean_sigma(Ss[:, k], 20)
            assert abs(mu - target) < 3 * s
    assert abs(Ss[:, 0]).max() < 1e-20


def test_water_primitive_and_centroid_virial_pressures_agree(orc):
    """<P_PR> = <P_CV> on an interacting system (pins the 1/P virial term that
    the printed P_PR line lacks)."""
    from paper_2602_13553_gb300 import inputs
    nmol, P, T = 32, 4, 300.0
    L = inputs.box_length(nmol)
    ff = inputs.WATER_FF[:6] + (4.5,)
    x0, mass = inputs.water_box(nmol, L, P, 5, jitter=0.02)
    sim = orc.Sim(x0, mass, T=T, dt=5e-4, potential=1, ff=ff, box=(L, L, L),
                  thermostat=1, seed=3, tau=0.05)
    sim.run(500)
    ppr, pcv, vir = [], [], []
    for _ in range(2000):
        sim.run(4)
        e = sim.estimators()
        ppr.append(e["P_PR"]); pcv.append(e["P_CV"]); vir.append(e["vir_sum"])
    d = np.array(ppr) - np.array(pcv)
    mu, s = block_mean_sigma(d, 20)
    assert abs(mu) < 3 * s, (mu, s, np.mean(ppr), np.mean(pcv))
    # the test is decisive: dropping the 1/P on the virial term would move
    # P_PR by (P-1)/P <sum_k Tr Xi>/(3V), hundreds of standard errors here
    shift = abs(np.mean(vir)) * (P - 1) / P / (3 * L ** 3)
    assert 3 * s < 0.1 * shift
