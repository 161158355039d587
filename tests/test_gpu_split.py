"""Split precision (FP64 centroid, FP32 bead deviations, internal modes,
forces and transforms) against the FP64 references.  Bars: positions within
1e-4 A of the FP64 oracle after 50 steps; 10k-step estimator averages within
0.1% of the FP64 GPU path driven by the same seeded noise; harmonic <x^2>
within 3 sigma of the discretised closed form."""
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import pimd  # noqa: F401

pytestmark = pytest.mark.gpu

HBAR = 4.135667403e-3 / (2 * math.pi)
OMEGA_HO = 0.1 / HBAR
KB = 8.617333262e-5
MVV2E = 1.0364269e-4


def _max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


@pytest.mark.parametrize("integ", [0, 1])
def test_split_water_512x64_drift_vs_oracle(orc, pimd, integ):
    """512 water-like molecules (24.84 A box), P = 64: after 50 steps the split
    trajectory stays within 1e-4 A of the FP64 oracle."""
    L = 24.84
    x0, mass = inputs.water_box(512, L, 64, 1, jitter=0.02)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(L, L, L), seed=1,
              integrator=integ)
    c = orc.Sim(x0, mass, **kw)
    g = pimd.Simulation(x0, mass, precision=pimd.PREC_SPLIT, **kw)
    c.run(50)
    g.step(50)
    xg, vg, st = g.get_state()
    assert st == 50
    dx = _max_abs(xg, c.x)
    dv = _max_abs(vg, c.v)
    print("split drift after 50 steps: x %.3g A, v %.3g A/ps" % (dx, dv))
    assert dx < 1e-4
    assert dv < 1e-2 * np.abs(c.v).max()


def test_split_harmonic_vs_oracle(orc, pimd):
    x0, mass = inputs.harmonic(64, 8, seed=1, std=0.1)
    kw = dict(T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), seed=1)
    c = orc.Sim(x0, mass, **kw)
    g = pimd.Simulation(x0, mass, precision=pimd.PREC_SPLIT, **kw)
    c.run(100)
    g.step(100)
    xg, vg, _ = g.get_state()
    assert _max_abs(xg, c.x) < 1e-5
    e = g.estimators()
    ec = c.estimators()
    for k in ("K_CV", "K_VR", "K_PR", "T_ring"):
        assert abs(e[k] - ec[k]) < 1e-4 * abs(ec[k]), k


def test_split_estimator_averages_10k_steps(pimd):
    """512 molecules x 64 beads, 10k steps after 1k of equilibration,
    estimators every 100 steps: split and FP64 GPU runs (same inputs, same
    keyed noise) agree on the averages to 0.1%, or to 3 standard errors of the
    difference where the sampling error of a 10k-step mean exceeds 0.1% (the
    pressures: a small mean of large fluctuating terms).  The two runs
    decorrelate chaotically within a few hundred steps, so their means are
    independent samples."""
    from tests._stats import block_mean_sigma
    L = 24.84
    x0, mass = inputs.water_box(512, L, 64, 1, jitter=0.02)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(L, L, L), seed=1)
    names = ("K_CV", "K_PR", "P_CV", "P_PR", "T_ring")
    runs = {}
    for prec in (pimd.PREC_FP64, pimd.PREC_SPLIT):
        s = pimd.Simulation(x0, mass, precision=prec, **kw)
        s.step(1000)
        acc = []
        for _ in range(100):
            s.step(100)
            e = s.estimators()
            acc.append([e[n] for n in names])
        runs[prec] = np.array(acc)
        s.close()
    for i, n in enumerate(names):
        ma, sa = block_mean_sigma(runs[pimd.PREC_FP64][:, i], 10)
        mb, sb = block_mean_sigma(runs[pimd.PREC_SPLIT][:, i], 10)
        diff, sd = abs(ma - mb), math.hypot(sa, sb)
        print("%s fp64 %.6g split %.6g rel %.2e (3 sigma rel %.2e)" % (n, ma, mb, diff / abs(ma), 3 * sd / abs(ma)))
        assert diff < max(1e-3 * abs(ma), 3 * sd), n
        if n in ("K_CV", "T_ring"):
            assert diff < 1e-3 * abs(ma), n


def test_split_harmonic_x2_closed_form(orc, pimd):
    """<x^2> of 4096 oscillators x 8 beads in split precision against the
    exact stationary value of the discretised BAOAB chain."""
    from tests.test_oracle_stats import discrete_baoab_x2, stationary_init
    N, P, T, m, dt, tau = 4096, 8, 300.0, 1.008, 2.5e-4, 0.05
    x0, v0 = stationary_init(orc, P, N, T, m, OMEGA_HO, seed=7)
    s = pimd.Simulation(x0, np.full(N, m), T=T, dt=dt, potential=0, ff=(OMEGA_HO,), v0=v0,
                        precision=pimd.PREC_SPLIT, seed=3, tau=tau)
    acc = np.zeros(N)
    ns = 200
    for _ in range(ns):
        s.step(20)
        x, _, _ = s.get_state()
        acc += (x ** 2).mean(axis=(0, 2))
    per = acc / ns
    mean, se = per.mean(), per.std(ddof=1) / math.sqrt(N)
    ref = discrete_baoab_x2(P, T, m, OMEGA_HO, dt, tau)
    assert abs(mean - ref) < 3 * se, (mean, ref, se)


def test_split_checkpoint_resume_is_bitwise(pimd):
    x0, mass = inputs.water_box(64, 12.42, 16, 3, jitter=0.02)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(12.42,) * 3, seed=11,
              precision=pimd.PREC_SPLIT)
    a = pimd.Simulation(x0, mass, **kw)
    a.step(40)
    a.step(40)
    xa, va, _ = a.get_state()
    b = pimd.Simulation(x0, mass, **kw)
    b.step(40)
    b.step(40)
    xb, vb, _ = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
