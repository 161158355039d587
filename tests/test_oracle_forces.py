"""Pins of the oracle's force fields: central finite differences of the
energy, Newton's third law, the virial against -dU/ds under uniform scaling,
and special cases with known answers."""
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs

FF = inputs.WATER_FF


def _fd_check(energy, x, F, h=1e-5, rel=1e-7, n=40, seed=0):
    g = np.random.default_rng(seed)
    scale = np.abs(F).max()
    idx = g.choice(x.size, size=min(n, x.size), replace=False)
    for flat in idx:
        xp = x.copy().ravel(); xm = x.copy().ravel()
        xp[flat] += h; xm[flat] -= h
        fd = -(energy(xp.reshape(x.shape)) - energy(xm.reshape(x.shape))) / (2 * h)
        assert abs(fd - F.ravel()[flat]) <= rel * scale + 1e-9, (flat, fd, F.ravel()[flat])


def test_harmonic_force_fd_and_virial(orc):
    g = np.random.default_rng(1)
    x = g.normal(0, 0.2, size=(10, 3))
    mass = g.uniform(1, 16, size=10)
    om = 151.9
    F, U, W = orc.force_harmonic(mass, om, x)
    _fd_check(lambda y: orc.force_harmonic(mass, om, y)[1], x, F)
    assert W == pytest.approx(float(np.sum(x * F)), rel=1e-14)
    assert W == pytest.approx(-2.0 * U, rel=1e-12)   # harmonic: r.F = -2U


@pytest.mark.parametrize("nmol,L,seed", [(64, 12.42, 1), (40, 12.6, 2)])
def test_water_force_fd(orc, nmol, L, seed):
    x, _ = inputs.water_box(nmol, L, 1, seed, jitter=0.05)
    x = x[0]
    box = (L, L, L)
    F, U, W = orc.force_water(box, FF, x)
    _fd_check(lambda y: orc.force_water(box, FF, y)[1], x, F, n=60)


def test_water_newton_third_law(orc):
    x, _ = inputs.water_box(64, 12.42, 1, 3, jitter=0.05)
    F, U, W = orc.force_water((12.42,) * 3, FF, x[0])
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).max() * len(F)


def test_water_virial_is_scaling_derivative(orc):
    """Tr Xi = sum r.f = -dU/ds when every coordinate and the box scale by s."""
    L = 12.42
    x, _ = inputs.water_box(64, L, 1, 4, jitter=0.05)
    x = x[0]
    F, U, W = orc.force_water((L,) * 3, FF, x)
    e = 1e-6
    Up = orc.force_water(((1 + e) * L,) * 3, FF, (1 + e) * x)[1]
    Um = orc.force_water(((1 - e) * L,) * 3, FF, (1 - e) * x)[1]
    assert W == pytest.approx(-(Up - Um) / (2 * e), rel=2e-6, abs=1e-7)


def test_water_rigid_isolated_molecule_is_at_rest(orc):
    """A molecule at (r0, theta0) with no oxygen within the cutoff feels no force."""
    x, _ = inputs.water_box(1, 20.0, 1, 5)
    F, U, W = orc.force_water((20.0,) * 3, FF, x[0])
    assert abs(U) < 1e-24 and np.abs(F).max() < 1e-12


def test_water_single_bond_is_hooke(orc):
    """Stretch one O-H bond along its axis: F_H = -kb (r - r0) along the bond,
    and the angle term stays zero (the geometry is unchanged in angle)."""
    x, _ = inputs.water_box(1, 20.0, 1, 6)
    x = x[0].copy()
    d = x[1] - x[0]
    x[1] = x[0] + d * 1.05
    F, U, W = orc.force_water((20.0,) * 3, FF, x)
    kb, r0 = FF[0], FF[1]
    r = np.linalg.norm(x[1] - x[0])
    assert U == pytest.approx(0.5 * kb * (r - r0) ** 2, rel=1e-12)
    assert np.allclose(F[1], -kb * (r - r0) * (x[1] - x[0]) / r, rtol=1e-12, atol=1e-14)


def test_water_lj_cutoff_and_minimum_image(orc):
    """Two molecules: LJ acts across the periodic boundary by minimum image and
    vanishes just beyond the cutoff."""
    L = 14.0
    base, _ = inputs.water_box(2, 40.0, 1, 7, r_oo_min=20.0)
    base = base[0]
    mol0 = base[0:3] - base[0]
    mol1 = base[3:6] - base[3]
    rc = FF[6]
    def U_at(sep):
        x = np.vstack([mol0 + np.array([0.5, 1.0, 1.0]),
                       mol1 + np.array([0.5 - sep, 1.0, 1.0]) + np.array([L, 0, 0])])
        return orc.force_water((L, L, L), FF, x)[1]
    eps, sig = FF[4], FF[5]
    for sep in (3.0, 4.5, 5.99):
        ref = 4 * eps * ((sig / sep) ** 12 - (sig / sep) ** 6)
        assert U_at(sep) == pytest.approx(ref, rel=1e-10)
    assert abs(U_at(rc + 1e-3)) < 1e-20
