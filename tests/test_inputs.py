"""The seeded synthetic inputs (paper_2602_13553_gb300/inputs.py) against
their stated recipe: box density, the water-like geometry and minimum O-O
separation, the lattice boxes of the serving trace, the replica mix and the
Poisson job stream.  They hold no method arithmetic; these checks make sure
both the oracle and the device path are fed the workloads the design names."""
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs


def _min_image_oo(x, L):
    O = x[0, 0::3, :]
    d = O[:, None, :] - O[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d * d).sum(axis=2))
    np.fill_diagonal(r, np.inf)
    return r.min()


def _check_geometry(x, nmol, L, r0=1.0, theta0=104.5):
    assert x.shape[1] == 3 * nmol and x.shape[2] == 3
    O, H1, H2 = x[0, 0::3], x[0, 1::3], x[0, 2::3]
    assert np.all(O >= 0.0) and np.all(O < L)
    b1 = np.linalg.norm(H1 - O, axis=1)
    b2 = np.linalg.norm(H2 - O, axis=1)
    assert np.allclose(b1, r0, atol=1e-12) and np.allclose(b2, r0, atol=1e-12)
    cos = np.einsum("ij,ij->i", H1 - O, H2 - O) / (b1 * b2)
    assert np.allclose(np.degrees(np.arccos(cos)), theta0, atol=1e-9)


def test_box_length_is_one_gram_per_cm3():
    assert abs(inputs.box_length(64) - 12.42) < 0.01
    assert abs(inputs.box_length(512) - 24.84) < 0.01
    # 18.015 g/mol in L^3: the density comes back
    L = inputs.box_length(300)
    assert abs(300 * inputs.WATER_AMU * inputs.AMU_G / (L * 1e-8) ** 3 - 1.0) < 1e-12


def test_force_field_cutoff_caps_small_boxes():
    assert inputs.WATER_FF[6] == 6.0
    assert inputs.water_ff_for_box(24.84)[6] == 6.0
    for nmol in (32, 64):
        L = inputs.box_length(nmol)
        assert abs(inputs.water_ff_for_box(L)[6] - min(6.0, 0.48 * L)) < 1e-15
        assert inputs.water_ff_for_box(L)[6] < 0.5 * L            # minimum image holds
        assert inputs.water_ff_for_box(L)[:6] == inputs.WATER_FF[:6]


@pytest.mark.parametrize("nmol", [32, 64, 150])
def test_water_box_recipe(nmol):
    L = inputs.box_length(nmol)
    x, mass = inputs.water_box(nmol, L, 4, seed=7)
    _check_geometry(x, nmol, L)
    assert _min_image_oo(x, L) >= 2.5
    assert np.array_equal(x[0], x[3])                       # no jitter: every bead the same
    assert np.array_equal(mass[:3], [inputs.MASS_O, inputs.MASS_H, inputs.MASS_H])
    x2, _ = inputs.water_box(nmol, L, 4, seed=7)
    assert np.array_equal(x, x2)                           # seeded
    _, md = inputs.water_box(nmol, L, 1, seed=7, deuterium=True)
    assert np.array_equal(md[:3], [inputs.MASS_O, inputs.MASS_D, inputs.MASS_D])


def test_water_box_jitter_is_per_bead_gaussian():
    L = inputs.box_length(64)
    x0, _ = inputs.water_box(64, L, 16, seed=3)
    xj, _ = inputs.water_box(64, L, 16, seed=3, jitter=0.05)
    dev = (xj - x0).ravel()
    assert abs(dev.mean()) < 0.005 and abs(dev.std() - 0.05) < 0.003


@pytest.mark.parametrize("nmol", [70, 512, 1000])
def test_lattice_box_recipe(nmol):
    L = inputs.box_length(nmol)
    x, mass = inputs.water_lattice_box(nmol, L, 2, seed=11)
    _check_geometry(x, nmol, L)
    assert _min_image_oo(x, L) >= 2.5 - 1e-9
    assert mass.shape == (3 * nmol,)


def test_lattice_box_falls_back_below_its_range():
    L = inputs.box_length(32)                                # lattice spacing < 2.5 A
    a, _ = inputs.water_lattice_box(32, L, 2, seed=5)
    b, _ = inputs.water_box(32, L, 2, seed=5)
    assert np.array_equal(a, b)


def test_harmonic_inputs():
    x, m = inputs.harmonic(4096, 8, seed=1, std=0.1)
    assert x.shape == (8, 4096, 3) and np.all(m == inputs.MASS_H)
    assert abs(x.std() - 0.1) < 0.002 and abs(x.mean()) < 0.002


def test_replica_mix_recipe():
    reps = inputs.replica_mix(256, seed=1)
    assert len(reps) == 256
    nm = np.array([r.nmol for r in reps])
    assert nm.min() >= 32 and nm.max() <= 512
    # log-uniform over [32, 512]: median near the geometric mean 128
    assert 90 <= np.median(nm) <= 180
    assert {r.P for r in reps} == {8, 16, 32, 64}
    T = np.array([r.T for r in reps])
    assert T.min() >= 100.0 and T.max() <= 400.0
    assert 0.35 <= np.mean([r.deuterium for r in reps]) <= 0.65
    assert all(abs(r.L - inputs.box_length(r.nmol)) < 1e-12 for r in reps)
    assert len({r.seed for r in reps}) == 256
    bead_atoms = sum(3 * r.nmol * r.P for r in reps)
    assert 3.0e6 < bead_atoms < 5.0e6                        # ~4 M bead-atoms


def test_serving_trace_recipe():
    jobs = inputs.serving_trace(2000, 50.0, seed=1)
    t = np.array([j.arrival_s for j in jobs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0 / 50.0) < 0.1 / 50.0       # Poisson at 50 jobs/s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1        # exponential gaps
    nm = np.array([j.nmol for j in jobs])
    assert nm.min() >= 32 and nm.max() <= 4096
    assert 250 <= np.median(nm) <= 450                       # geometric mean of [32, 4096] is 362
    Ps = np.array([j.P for j in jobs])
    assert set(Ps.tolist()) == {4, 8, 16, 32, 64, 128}
    for P in (4, 8, 16, 32, 64, 128):
        assert 0.12 < np.mean(Ps == P) < 0.22
    st = np.array([j.nsteps for j in jobs])
    assert st.min() >= 1000 and st.max() <= 50000
    assert abs(math.log(np.median(st)) - 0.5 * (math.log(1000) + math.log(50000))) < 0.2
