"""Split precision (FP64 centroid, FP32 bead deviations, internal modes,
forces and transforms) against the FP64 references.  Bars: positions within
1e-4 A of the FP64 oracle after 50 steps; 10k-step estimator averages within
0.1% of the FP64 path over the same trajectory windows (the FP64 arm tied to
the oracle); harmonic <x^2> within 3 sigma of the discretised closed form."""
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


@pytest.mark.parametrize("P,N", [(8, 64), (16, 37), (32, 50), (64, 21), (128, 13), (12, 40)])
def test_split_harmonic_vs_oracle(orc, pimd, P, N):
    """Split precision on harmonic oscillators: bead counts 8-128 take the
    warp-item step kernel (ragged last tile when N is not a multiple of 8),
    12 the block kernel."""
    x0, mass = inputs.harmonic(N, P, seed=1, std=0.1)
    kw = dict(T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), seed=1)
    c = orc.Sim(x0, mass, **kw)
    g = pimd.Simulation(x0, mass, precision=pimd.PREC_SPLIT, **kw)
    c.run(100)
    g.step(100)
    xg, vg, _ = g.get_state()
    assert _max_abs(xg, c.x) < 1e-5
    e = g.estimators()
    ec = c.estimators()
    for k in ("K_CV", "K_VR", "T_ring"):
        assert abs(e[k] - ec[k]) < 1e-4 * abs(ec[k]), k
    # K_PR (App. A output 5) is the kinetic term 3 P N kB T / 2 minus the
    # spring energy over P, terms P times larger than their difference: its
    # error is measured against the kinetic term (1.5 N kB T_ring)
    assert abs(e["K_PR"] - ec["K_PR"]) < 1e-4 * 1.5 * N * 8.617333262e-5 * ec["T_ring"]


def test_split_estimator_averages_10k_steps(orc, pimd):
    """512 molecules x 64 beads (24.84 A box), 10k steps after 1k of
    equilibration.  The precision error is isolated from the chaotic
    divergence of two independent runs as follows:
    - one FP64 trajectory is checkpointed every 100 steps;
    - from each checkpoint a split-precision handle restarts at the same step
      and runs the same 100-step window with the same keyed noise;
    - both arms sample the estimators every 10 steps, so both averages cover
      the same 10k steps of the same trajectory (1000 samples).
    K_CV, K_PR, P_CV, P_PR and T_ring must agree within 0.1%.  The FP64 arm
    is tied to the oracle: from the first checkpoint, state and estimators
    after 50 steps agree within the 1e-8 water bar."""
    from tests._gpu import coord_err
    L = 24.84
    x0, mass = inputs.water_box(512, L, 64, 1, jitter=0.02)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(L, L, L), seed=1)
    names = ("K_CV", "K_PR", "P_CV", "P_PR", "T_ring")
    ref = pimd.Simulation(x0, mass, precision=pimd.PREC_FP64, **kw)
    ref.step(1000)
    split = None
    acc = {pimd.PREC_FP64: [], pimd.PREC_SPLIT: []}
    for w in range(100):
        xc, vc, st = ref.get_state()
        if split is None:
            split = pimd.Simulation(xc, mass, v0=vc, precision=pimd.PREC_SPLIT, **kw)
        split.set_state(xc, vc, st)
        for j in range(10):
            for arm, sim in ((pimd.PREC_FP64, ref), (pimd.PREC_SPLIT, split)):
                sim.step(10)
                e = sim.estimators()
                acc[arm].append([e[n] for n in names])
            if w == 0 and j == 4:
                # the oracle from the same checkpoint, 50 steps
                c = orc.Sim(xc, mass, v0=vc, **kw)
                c._s.step = st
                c.run(50)
                xg, vg, sg = ref.get_state()
                assert sg == st + 50
                assert coord_err(xg, c.x) < 1e-8 and coord_err(vg, c.v) < 1e-8
                ec = c.estimators()
                for n in ("K_CV", "K_PR", "T_ring"):
                    assert abs(acc[pimd.PREC_FP64][-1][names.index(n)] - ec[n]) < 1e-8 * abs(ec[n]), n
    a = np.array(acc[pimd.PREC_FP64])
    b = np.array(acc[pimd.PREC_SPLIT])
    assert a.shape == (1000, len(names))
    for i, n in enumerate(names):
        ma, mb = a[:, i].mean(), b[:, i].mean()
        rel = abs(ma - mb) / abs(ma)
        print("%s fp64 %.8g split %.8g rel %.2e (largest per-sample rel %.2e)"
              % (n, ma, mb, rel, np.max(np.abs(a[:, i] - b[:, i])) / abs(ma)))
        assert rel < 1e-3, n
    ref.close()
    split.close()


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
