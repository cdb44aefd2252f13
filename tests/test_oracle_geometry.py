"""Pins for the oracle's "set" geometry: R0, check points, partners, fitting matrix, QR."""
import math

import numpy as np
import pytest

from oracle import psum_oracle as O

BOXES = [(1.0, 1.0, 1.0), (1.0, 1.5, 2.0), (1.0, 1.0, 2.0), (2.0, 1.2, 1.0)]


@pytest.mark.parametrize("d", BOXES)
def test_circumradius_and_checkpoints(d):
    R0 = O.circumradius(d)
    # the circumsphere passes through the box corners (set step 1)
    assert R0 == pytest.approx(0.5 * math.sqrt(sum(v * v for v in d)), rel=1e-15)
    Y = O.fibonacci_checkpoints(400, R0)
    assert Y.shape == (400, 3)
    assert np.allclose(np.linalg.norm(Y, axis=1), R0, rtol=1e-14)
    # quasi-uniform: every point has a neighbour, none closer than 0.5 of the mean spacing
    D = np.linalg.norm(Y[:, None] - Y[None], axis=2) + np.eye(400) * 10
    spacing = R0 * math.sqrt(4 * math.pi / 400)
    assert D.min() > 0.5 * spacing
    assert D.min(axis=1).max() < 1.5 * spacing


@pytest.mark.parametrize("d", BOXES)
def test_partners_are_periodic_images_inside_sphere(d):
    R0 = O.circumradius(d)
    Y = O.fibonacci_checkpoints(300, R0)
    Yt = O.periodic_partners(Y, d)
    diff = Y - Yt
    nz = np.abs(diff) > 0
    assert np.all(nz.sum(axis=1) == 1)                     # one coordinate shifted
    k = np.argmax(nz, axis=1)
    assert np.allclose(np.abs(diff[np.arange(300), k]), np.asarray(d)[k], rtol=1e-15)
    assert np.all(np.linalg.norm(Yt, axis=1) < R0)         # y~ in S0 (set step 3)
    assert np.all(np.max(np.abs(Y) / np.asarray(d), axis=1) > 0.5)   # y outside the box


def test_constant_column_dropped_and_rank_condition():
    d, p = (1.0, 1.0, 1.0), 6
    R0 = O.circumradius(d)
    Y = O.fibonacci_checkpoints(120, R0)
    Yt = O.periodic_partners(Y, d)
    full = (O.regular_basis(Y / R0, p) - O.regular_basis(Yt / R0, p)).T
    assert np.all(full[:, 0] == 0.0)                       # A_l1 = 0 (Sec. 3)
    A = O.fit_matrix(Y, Yt, p, R0)
    assert A.shape == (120, (p + 1) ** 2 - 1)
    assert np.array_equal(A, full[:, 1:])
    # fewer equations than unknowns cannot be full rank (Sec. 4.1, rank condition)
    with pytest.raises(O.RankDeficient):
        O.qr_factor(O.fit_matrix(Y[:40], Yt[:40], p, R0))


@pytest.mark.parametrize("d,p,M", [((1, 1, 1), 8, 200), ((1, 1.5, 2), 16, 800), ((1, 1, 2), 12, 400)])
def test_qr_solution_matches_svd_least_squares(d, p, M):
    pl = O.Plan(d, p, M)
    rng = np.random.default_rng(p)
    f = rng.normal(size=M)
    c_qr = O.qr_solve(pl.factors, f)
    c_svd = np.linalg.lstsq(pl.A, f, rcond=None)[0]
    assert np.linalg.norm(c_qr - c_svd) <= 1e-12 * np.linalg.norm(c_svd) * max(1.0, np.linalg.cond(pl.A) / 100)
    # normal equations hold: A^T (A c - f) = 0
    res = pl.A.T @ (pl.A @ c_qr - f)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(pl.A.T @ f)
