"""Pins for the oracle's box integrals (App. B) and the mean of phi_near (App. C)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import psum_oracle as O


@pytest.mark.parametrize("d", [(1.0, 1.0, 1.0), (1.0, 1.5, 2.0)])
def test_box_integrals_exact_and_closed_form(d):
    p = 12
    R0 = O.circumradius(d)
    Rb = O.box_integrals(d, p, R0)
    assert Rb[0] == pytest.approx(1.0, abs=1e-15)
    # exactness of the floor(p/2)+1 point rule (Eq. A2): more points change nothing
    assert np.allclose(Rb, O.box_integrals(d, p, R0, nq=p // 2 + 5), rtol=1e-12, atol=1e-15)
    # odd degrees vanish on the symmetric box: R^_n(-u) = (-1)^n R^_n(u)
    for n in range(1, p + 1, 2):
        for m in range(-n, n + 1):
            assert abs(Rb[O.basis_index(n, m)]) < 1e-15
    # R^_2^0 = (2z^2 - x^2 - y^2)/2 and <u_k^2> = d_k^2 / (12 R0^2)
    d1, d2, d3 = d
    expect = (2 * d3 ** 2 - d1 ** 2 - d2 ** 2) / (24 * R0 ** 2)
    assert Rb[O.basis_index(2, 0)] == pytest.approx(expect, rel=1e-13, abs=1e-16)


def test_cube_centre_classical_value():
    # Potential at the centre of a uniform unit cube: 3 ln(2 + sqrt 3) - pi/2.
    v = O.block_potential(np.zeros((1, 3)), [-0.5] * 3, [0.5] * 3)[0]
    assert v == pytest.approx(3 * math.log(2 + math.sqrt(3)) - math.pi / 2, rel=1e-14)
    # At a corner: a quarter of the centre value of the cube of edge 2 divided by 8 -> half.
    c = O.block_potential(np.array([[0.5, 0.5, 0.5]]), [-0.5] * 3, [0.5] * 3)[0]
    assert c == pytest.approx(0.5 * v, rel=1e-13)
    # scaling: U scales like length^2
    v2 = O.block_potential(np.zeros((1, 3)), [-1.5] * 3, [1.5] * 3)[0]
    assert v2 == pytest.approx(9 * v, rel=1e-13)


def test_block_potential_outside_matches_cubature():
    lo, hi = np.array([-1.5, -2.25, -3.0]), np.array([1.5, 2.25, 3.0])
    for x in ([2.1, 0.3, -0.7], [0.2, -2.9, 3.4], [4.0, 4.0, 4.0]):
        val, err = integrate.tplquad(
            lambda z, y, xx: 1.0 / math.sqrt((xx - x[0]) ** 2 + (y - x[1]) ** 2 + (z - x[2]) ** 2),
            lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], epsabs=1e-12, epsrel=1e-11)
        got = O.block_potential(np.array([x]), lo, hi)[0]
        assert got == pytest.approx(val, rel=1e-9)


def test_block_potential_poisson_and_far_field():
    lo, hi = np.array([-1.5, -1.5, -3.0]), np.array([1.5, 1.5, 3.0])
    h = 1e-3
    for x, lap_expect in (([0.2, -0.3, 0.4], -4 * math.pi), ([2.0, 0.3, 0.1], 0.0)):
        x = np.array(x)
        lap = -6 * O.block_potential(x[None], lo, hi)[0]
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            lap += O.block_potential((x + e)[None], lo, hi)[0] + O.block_potential((x - e)[None], lo, hi)[0]
        assert lap / h ** 2 == pytest.approx(lap_expect, abs=2e-4)
    far = np.array([[300.0, -400.0, 1200.0]])
    V = float(np.prod(hi - lo))
    assert O.block_potential(far, lo, hi)[0] == pytest.approx(V / np.linalg.norm(far), rel=1e-5)


def test_near_mean_sums_box_averages_of_all_images():
    # Eq. pfx4 for one unit charge at the centre of the unit cube: the p = 0 term is the
    # classical centre value, the 26 image terms are smooth integrals done by Gauss quadrature.
    d = np.array([1.0, 1.0, 1.0])
    t, w = np.polynomial.legendre.leggauss(40)
    g = 0.5 * t
    Y = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).reshape(-1) / 8.0
    ref = 3 * math.log(2 + math.sqrt(3)) - math.pi / 2
    for i1 in (-1, 0, 1):
        for i2 in (-1, 0, 1):
            for i3 in (-1, 0, 1):
                if i1 == i2 == i3 == 0:
                    continue
                pvec = np.array([i1, i2, i3], dtype=float)
                ref += float(W @ (1.0 / np.linalg.norm(Y - pvec, axis=1)))
    got = O.near_mean(np.zeros((1, 3)), np.ones(1), d)
    assert got == pytest.approx(ref, rel=1e-12)
