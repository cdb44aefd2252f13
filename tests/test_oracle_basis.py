"""Pins for the oracle's basis functions (Eqs. 1.1-1.9), independent of the recurrence."""
import math

import numpy as np
import pytest
from scipy.special import lpmv

from oracle import psum_oracle as O


def _definition(u, p):
    """R^_n^m from the complex definition, Eqs. 1.1-1.4.1 and 1.7, via scipy's P_n^m."""
    r = np.linalg.norm(u, axis=1)
    theta = np.arccos(np.clip(u[:, 2] / r, -1, 1))
    az = np.arctan2(u[:, 1], u[:, 0])
    out = np.zeros(((p + 1) ** 2, u.shape[0]))
    for n in range(p + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            alpha = (-1) ** n * math.sqrt(4 * math.pi / ((2 * n + 1) * math.factorial(n - m)
                                                         * math.factorial(n + m)))
            Nnm = (-1) ** m * math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - am)
                                        / math.factorial(n + am))
            R = alpha * r ** n * Nnm * lpmv(am, n, np.cos(theta)) * np.exp(1j * m * az)
            Rt = R.real if m >= 0 else R.imag                     # Eq. 1.4
            out[n * (n + 1) + m] = math.sqrt(math.factorial(n - m) * math.factorial(n + m)) * Rt
    return out


@pytest.mark.parametrize("p", [1, 6, 14])
def test_recurrence_matches_definition(p):
    rng = np.random.default_rng(10 + p)
    u = rng.normal(size=(64, 3)) * 0.5
    B = O.regular_basis(u, p)
    ref = _definition(u, p)
    scale = np.maximum(1.0, np.abs(ref).max(axis=1, keepdims=True))
    assert np.max(np.abs(B - ref) / scale) < 1e-13


def test_low_order_values():
    # Eq. 1.6: R~_1^1 = -x/2, R~_1^-1 = y/2, and Eq. 1.7 multiplies by sqrt(0! 2!)
    u = np.array([[0.3, -0.7, 0.2]])
    B = O.regular_basis(u, 2)
    s2 = math.sqrt(2.0)
    assert B[O.basis_index(0, 0), 0] == 1.0
    assert B[O.basis_index(1, 1), 0] == pytest.approx(-0.3 / 2 * s2, rel=1e-15)
    assert B[O.basis_index(1, -1), 0] == pytest.approx(-0.7 / 2 * s2, rel=1e-15)
    assert B[O.basis_index(1, 0), 0] == pytest.approx(-0.2, rel=1e-15)
    # (3 z^2 - r^2)/4 * 2 for n = 2, m = 0 (Legendre P_2)
    x, y, z = u[0]
    assert B[O.basis_index(2, 0), 0] == pytest.approx((2 * z * z - x * x - y * y) / 2, rel=1e-14)


def test_z_axis_reduces_to_powers():
    # On the z axis P_n(1) = 1 and P_n^m(1) = 0 (m != 0): R^_n^0 = (-z)^n, the rest vanish.
    z = np.linspace(-1.3, 1.3, 7)
    u = np.stack([np.zeros_like(z), np.zeros_like(z), z], axis=1)
    p = 12
    B = O.regular_basis(u, p)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            expect = (-z) ** n if m == 0 else 0.0
            assert np.allclose(B[O.basis_index(n, m)], expect, rtol=1e-13, atol=1e-13)


def test_homogeneous_and_parity():
    rng = np.random.default_rng(3)
    u = rng.normal(size=(20, 3))
    p = 10
    B1 = O.regular_basis(u, p)
    B2 = O.regular_basis(-0.5 * u, p)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            t = O.basis_index(n, m)
            assert np.allclose(B2[t], (-0.5) ** n * B1[t], rtol=1e-12, atol=1e-14)


def test_harmonic():
    # every R^ solves Laplace's equation: 7-point Laplacian, Richardson-extrapolated in h
    rng = np.random.default_rng(4)
    u = rng.normal(size=(10, 3)) * 0.6
    p = 9

    def lap(h):
        out = -6 * O.regular_basis(u, p)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            out = out + O.regular_basis(u + e, p) + O.regular_basis(u - e, p)
        return out / (h * h)

    L = (4 * lap(1e-3) - lap(2e-3)) / 3
    scale = np.abs(O.regular_basis(u, p)).max(axis=1, keepdims=True) + 1.0
    assert np.max(np.abs(L) / scale) < 1e-6


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    u = rng.normal(size=(12, 3)) * 0.6
    p, h = 12, 1e-5
    B, G = O.regular_basis(u, p, grad=True)
    assert np.array_equal(B, O.regular_basis(u, p))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (O.regular_basis(u + e, p) - O.regular_basis(u - e, p)) / (2 * h)
        scale = np.abs(fd).max(axis=1, keepdims=True) + 1.0
        assert np.max(np.abs(G[:, k, :] - fd) / scale) < 1e-8
