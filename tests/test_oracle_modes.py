"""Pins of the normal-mode transform (App. B, Eqs. A1-A3) and of the ring
polymer frequencies (Eq. 2, App. D)."""
import math

import numpy as np
import pytest
from scipy import constants as sc

PS = list(range(1, 21)) + [31, 32, 33, 64, 100, 127, 128]


def cyclic_second_difference(P):
    A = 2.0 * np.eye(P)
    for j in range(P):
        A[j, (j + 1) % P] -= 1.0
        A[j, (j - 1) % P] -= 1.0
    if P == 1:
        A[:] = 0.0
    if P == 2:
        A = np.array([[2.0, -2.0], [-2.0, 2.0]])
    return A


@pytest.mark.parametrize("P", PS)
def test_nm_matrix_orthogonal(orc, P):
    M = orc.nm_matrix(P)
    assert np.abs(M @ M.T - np.eye(P)).max() <= 1e-14 * max(1, P / 8)


@pytest.mark.parametrize("P", [p for p in PS if p != 2])
def test_nm_matrix_diagonalises_ring(orc, P):
    """Rows of M are eigenvectors of the ring's second-difference matrix with
    eigenvalue lambda_k = 4 sin^2(k pi / P) (Eq. A2)."""
    M = orc.nm_matrix(P)
    lam = orc.mode_lambda(P)
    A = cyclic_second_difference(P)
    D = M @ A @ M.T
    assert np.abs(D - np.diag(lam)).max() <= 1e-13 * max(1, P / 8)


def test_ring_P2_spring(orc):
    """P = 2: the spring sum counts the bond twice (r0-r1 and r1-r0)."""
    M = orc.nm_matrix(2)
    lam = orc.mode_lambda(2)
    x = np.array([0.3, -1.1])
    q = M @ x
    spring_cart = (x[0] - x[1]) ** 2 + (x[1] - x[0]) ** 2
    assert spring_cart == pytest.approx(np.sum(lam * q * q), rel=1e-14)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 8, 9, 16, 32, 64, 128])
def test_nm_matrix_is_scaled_real_dft(orc, P):
    """Row-by-row check of Eq. (A1) against numpy's FFT: row 0 = mean * sqrt(P),
    row P/2 = alternating sum, cos rows = Re, sin rows i > P/2 = -Im of the DFT
    at frequency i (signs as printed)."""
    g = np.random.default_rng(P)
    x = g.normal(size=P)
    M = orc.nm_matrix(P)
    q = M @ x
    X = np.fft.fft(x)          # X_i = sum_j x_j exp(-2 pi i ij/P)
    for i in range(P):
        if i == 0:
            ref = X[0].real / math.sqrt(P)
        elif P % 2 == 0 and i == P // 2:
            ref = X[i].real / math.sqrt(P)
        elif i <= P // 2:
            ref = math.sqrt(2.0 / P) * X[i].real
        else:
            ref = -math.sqrt(2.0 / P) * X[i].imag
        assert q[i] == pytest.approx(ref, abs=1e-13 * max(1.0, np.abs(x).sum()))


def test_omega_n_and_modes(orc):
    """Eq. (2) with CODATA k_B and hbar from scipy; omega_k = 2 omega_n sin(pi k/P)."""
    for P, T, sp in [(8, 300.0, 1.0), (32, 300.0, 1.0), (64, 150.0, 0.5), (1, 10.0, 1.0)]:
        wn = orc.omega_n(P, T, sp)
        ref = P * sc.k * T / (sp * sc.hbar) * 1e-12   # 1/ps
        assert wn == pytest.approx(ref, rel=1e-6)
        w = orc.mode_omega(P, T, sp)
        for k in range(P):
            assert w[k] == pytest.approx(2 * wn * abs(math.sin(math.pi * k / P)), rel=1e-13, abs=1e-12)


def test_to_from_nm_roundtrip(orc):
    g = np.random.default_rng(0)
    for P in (1, 3, 8, 32):
        x = g.normal(size=(P, 17, 3))
        M = orc.nm_matrix(P)
        q = orc.to_nm(M, x)
        assert np.allclose(q, np.einsum("ij,jna->ina", M, x), rtol=0, atol=1e-13)
        assert np.abs(orc.from_nm(M, q) - x).max() < 1e-13
