"""ORACLE -- test infrastructure only.

A plain, slow, double-precision CPU implementation of the periodisation
method of Gumerov & Duraiswami, "A method to compute periodic sums"
(arXiv 1310.4374).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the product never does, and it
shares no code with the CUDA path.

It follows the two algorithms of Sec. 2.3 step by step:

  "set" (Sec. 2.3.1): circumradius R0 (step 1), check points on the sphere
  (step 2), periodic partners (step 3), fitting matrix A (step 4), its
  rank-revealing QR (step 5), box integrals of the basis (step 6, App. B).

  "get" (Sec. 2.3.2): near-field image sum at targets and check points
  (steps 1, 3; Eq. 3), right-hand side f (step 4, Eq. 8), least-squares
  coefficients (step 5, Eq. 10), constant C1 from the zero-mean condition
  (step 6, Eqs. pfx3-pfx4, App. C), far field and its gradient at the
  targets (step 7, Eqs. 1.6-1.9) and the sum (step 8).

Readings where the paper is silent (each is listed in the design notes):
  * check points: a spherical Fibonacci lattice of M points on radius R0;
  * partner of y: shift the coordinate k with the largest |y_k|/d_k by
    -sign(y_k) d_k (ties go to the lowest k);
  * basis functions are evaluated at y/R0 (same span, better scaling);
  * the near block Omega_b is the (2K+1)^3 block of boxes (default K=1,
    i.e. the box and its 26 neighbours); optionally the ball S_b of radius
    lambda R0 (get step 2), a source image kept iff |x + p|^2 <= Rb^2;
  * the RBF basis of Eq. 5 (optional) puts its kernel centres on a spherical
    Fibonacci lattice on S_b (the paper used Thomson points, not available);
  * rank tolerance of the QR: |R_kk| >= 1e-13 |R_11|;
  * C1 sets the mean of phi over the box to zero (the Ewald convention,
    App. D Eq. e6), and the mean of phi_near uses the closed-form Newtonian
    potential of the uniform (2K+1)d block (the union of the box images);
  * p is the maximum degree, so there are P = (p+1)^2 basis functions.

parity pinned: every function here is checked in ``tests/`` against the
definition it restates (Eqs. 1.1-1.4.1 through scipy's Legendre functions,
adaptive cubature for the block potential, SVD least squares), against
closed forms, and, for the whole method, against the NaCl Madelung constant
(Eq. st1) and an independent classic Ewald sum (App. D).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import scipy.linalg

from . import build as _build

# ---------------------------------------------------------------------------
# "set", step 1: circumradius of the box (Sec. 2.3.1)
# ---------------------------------------------------------------------------


def circumradius(d) -> float:
    d = np.asarray(d, dtype=np.float64)
    return 0.5 * math.sqrt(float(np.sum(d * d)))


# ---------------------------------------------------------------------------
# "set", step 2: L check points on the sphere of radius R0 (Sec. 2.2).
# Reading: spherical Fibonacci lattice, z_l = 1 - (2l+1)/M, azimuth l*pi*(3-sqrt 5).
# ---------------------------------------------------------------------------


def fibonacci_checkpoints(M: int, R0: float) -> np.ndarray:
    l = np.arange(M, dtype=np.float64)
    z = 1.0 - (2.0 * l + 1.0) / M
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    az = l * math.pi * (3.0 - math.sqrt(5.0))
    return R0 * np.stack([rho * np.cos(az), rho * np.sin(az), z], axis=1)


def gauss_checkpoints(p: int, R0: float) -> np.ndarray:
    """The Gauss spherical grid of Sec. 2.2 (ii): polar angles at the zeros of the Legendre
    polynomial P_{p+1}(cos theta), 2p+1 equispaced azimuths (from 0), radius R0.  With the
    paper's truncation number p' = p + 1 this is its L = 2p'^2 - p' points."""
    t, _ = np.polynomial.legendre.leggauss(p + 1)
    theta = np.arccos(t)
    az = 2.0 * math.pi * np.arange(2 * p + 1) / (2 * p + 1)
    TH, AZ = np.meshgrid(theta, az, indexing="ij")
    return R0 * np.stack([np.sin(TH) * np.cos(AZ), np.sin(TH) * np.sin(AZ), np.cos(TH)],
                         axis=-1).reshape(-1, 3)


# ---------------------------------------------------------------------------
# "set", step 3: periodic partner of every check point (Sec. 2.3.1, Eq. 7).
# Two coordinates are kept, the coordinate k with the largest |y_k|/d_k is
# shifted by one period towards the box, so the partner lies inside S0.
# ---------------------------------------------------------------------------


def periodic_partners(Y: np.ndarray, d) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64)
    k = np.argmax(np.abs(Y) / d, axis=1)          # first maximum on ties
    Yt = Y.copy()
    rows = np.arange(Y.shape[0])
    Yt[rows, k] -= np.sign(Y[rows, k]) * d[k]
    return Yt


# ---------------------------------------------------------------------------
# Basis: real regular solid harmonics by the recurrence of Eq. 1.6,
# renormalised by Eq. 1.7, stacked by Eq. 1.8 (0-based t = n(n+1) + m).
# Gradients by differentiating every step of the recurrence (forward mode).
# ---------------------------------------------------------------------------


def basis_index(n: int, m: int) -> int:
    return n * (n + 1) + m


def num_terms(p: int) -> int:
    return (p + 1) * (p + 1)


def regular_basis(u: np.ndarray, p: int, grad: bool = False):
    """R^_n^m(u) for 0 <= n <= p, -n <= m <= n at points u (npts, 3).

    Returns B (P, npts) and, with ``grad``, G (P, 3, npts) = dB/du.
    """
    u = np.asarray(u, dtype=np.float64)
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    npts = u.shape[0]
    r2 = x * x + y * y + z * z
    P = num_terms(p)
    Rt = np.zeros((P, npts))
    Gt = np.zeros((P, 3, npts)) if grad else None
    ex = np.array([1.0, 0.0, 0.0])[:, None]
    ey = np.array([0.0, 1.0, 0.0])[:, None]
    ez = np.array([0.0, 0.0, 1.0])[:, None]
    I = basis_index

    # Eq. 1.6, first line: R~_0^0 = 1, R~_1^1 = -x/2, R~_1^-1 = y/2
    Rt[I(0, 0)] = 1.0
    if p >= 1:
        Rt[I(1, 1)] = -0.5 * x
        Rt[I(1, -1)] = 0.5 * y
        if grad:
            Gt[I(1, 1)] = -0.5 * ex
            Gt[I(1, -1)] = 0.5 * ey
    # Eq. 1.6, second line: the sectoral functions, |m| = 2, 3, ...
    for m in range(2, p + 1):
        a, b = Rt[I(m - 1, m - 1)], Rt[I(m - 1, -(m - 1))]
        Rt[I(m, m)] = -(x * a + y * b) / (2 * m)
        Rt[I(m, -m)] = (y * a - x * b) / (2 * m)
        if grad:
            ga, gb = Gt[I(m - 1, m - 1)], Gt[I(m - 1, -(m - 1))]
            Gt[I(m, m)] = -(ex * a + x * ga + ey * b + y * gb) / (2 * m)
            Gt[I(m, -m)] = (ey * a + y * ga - ex * b - x * gb) / (2 * m)
    # Eq. 1.6, third line: R~_{|m|+1}^m = -z R~_{|m|}^m
    # Eq. 1.6, fourth line: the three-term recurrence in n for n >= |m| + 2
    for m in range(-p, p + 1):
        am = abs(m)
        if am + 1 <= p:
            Rt[I(am + 1, m)] = -z * Rt[I(am, m)]
            if grad:
                Gt[I(am + 1, m)] = -(ez * Rt[I(am, m)] + z * Gt[I(am, m)])
        for n in range(am + 2, p + 1):
            den = (n - am) * (n + am)
            Rt[I(n, m)] = -((2 * n - 1) * z * Rt[I(n - 1, m)] + r2 * Rt[I(n - 2, m)]) / den
            if grad:
                Gt[I(n, m)] = -((2 * n - 1) * (ez * Rt[I(n - 1, m)] + z * Gt[I(n - 1, m)])
                                + 2.0 * u.T * Rt[I(n - 2, m)] + r2 * Gt[I(n - 2, m)]) / den
    # Eq. 1.7: R^_n^m = sqrt((n-m)! (n+m)!) R~_n^m
    for n in range(p + 1):
        for m in range(-n, n + 1):
            s = math.sqrt(math.factorial(n - m) * math.factorial(n + m))
            Rt[I(n, m)] *= s
            if grad:
                Gt[I(n, m)] *= s
    return (Rt, Gt) if grad else Rt


# ---------------------------------------------------------------------------
# "set", step 4: fitting matrix A_lt = R_t(y_l) - R_t(y~_l) (Eq. 8), with the
# constant function t = 1 removed because its column is zero (Sec. 3).
# ---------------------------------------------------------------------------


# ---------------------------------------------------------------------------
# The RBF basis of Eq. 5: R_t(y) = K(y - x_t^(s)) = 1/|y - x_t^(s)| with the
# kernel centres x_t^(s) outside the ball S_b.  Reading: S centres on a spherical
# Fibonacci lattice of radius Rs (the paper's Thomson points are not available).
# ---------------------------------------------------------------------------


def rbf_centres(S: int, Rs: float) -> np.ndarray:
    return fibonacci_checkpoints(S, Rs)


def rbf_basis(y: np.ndarray, centres: np.ndarray, grad: bool = False):
    """R_t(y) = 1/|y - x_t| (S, npts) and, with ``grad``, dR_t/dy (S, 3, npts)."""
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    r = y[None, :, :] - centres[:, None, :]                 # (S, npts, 3)
    dist = np.sqrt(np.sum(r * r, axis=2))
    B = 1.0 / dist
    if not grad:
        return B
    G = -(r / dist[:, :, None] ** 3).transpose(0, 2, 1)     # (S, 3, npts)
    return B, G


def fit_matrix_rbf(Y: np.ndarray, Yt: np.ndarray, centres: np.ndarray) -> np.ndarray:
    """A_lt = R_t(y_l) - R_t(y~_l) for the RBF basis (Eq. 8 with Eq. 5), (M, S).  No
    constant column arises: the constant C_1 is a separate unknown, fixed by the mean."""
    return (rbf_basis(Y, centres) - rbf_basis(Yt, centres)).T.copy()


def fit_matrix(Y: np.ndarray, Yt: np.ndarray, p: int, R0: float) -> np.ndarray:
    B = regular_basis(Y / R0, p)
    Bt = regular_basis(Yt / R0, p)
    return (B - Bt)[1:, :].T.copy()          # (M, P-1)


# ---------------------------------------------------------------------------
# "set" step 5 / "get" step 5: least squares by rank-revealing QR (Eqs. 9-10).
# ---------------------------------------------------------------------------

RANK_TOL = 1e-13


class RankDeficient(ValueError):
    pass


def qr_factor(A: np.ndarray):
    Q, R, piv = scipy.linalg.qr(A, mode="economic", pivoting=True)
    diag = np.abs(np.diag(R))
    if diag.size == 0 or A.shape[0] < A.shape[1] or np.any(diag < RANK_TOL * diag[0]):
        raise RankDeficient("fitting matrix is rank deficient")
    return Q, R, piv


def qr_solve(factors, f: np.ndarray) -> np.ndarray:
    Q, R, piv = factors
    z = scipy.linalg.solve_triangular(R, Q.T @ f, lower=False)
    c = np.empty_like(z)
    c[piv] = z
    return c


# ---------------------------------------------------------------------------
# "set", step 6: box integrals R_t^(0) = (1/V0) int_box R_t dV (Eq. pfx3) by the
# tensor Gauss-Legendre rule of App. B (Eq. A1) with N_q = floor(p/2) + 1
# points per axis, exact for the degree-p polynomials R_t (Eq. A2).
# ---------------------------------------------------------------------------


def box_integrals(d, p: int, R0: float, nq: int | None = None) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64)
    if nq is None:
        nq = p // 2 + 1
    t, w = np.polynomial.legendre.leggauss(nq)
    X, Y, Z = np.meshgrid(0.5 * d[0] * t, 0.5 * d[1] * t, 0.5 * d[2] * t, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).reshape(-1)
    pts = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    B = regular_basis(pts / R0, p)
    return (B @ W) / 8.0


# ---------------------------------------------------------------------------
# Mean of phi_near over the box (Eq. pfx4, App. C).  The near block is the
# union of the box images, so sum_p Phi_0(x + p) = U(x)/V0 with U the Newtonian
# potential int dV(y)/|y - x| of the uniform block.  U is written out by the
# classical closed form for a rectangular prism (sum over its 8 corners).
# ---------------------------------------------------------------------------


def _log_plus_r(a, b, c, r):
    """log(a + r) with r = sqrt(a^2 + b^2 + c^2), without cancellation for a < 0."""
    out = np.empty_like(a)
    pos = a >= 0
    out[pos] = np.log(a[pos] + r[pos])
    neg = ~pos
    bc = b[neg] ** 2 + c[neg] ** 2
    with np.errstate(divide="ignore"):
        out[neg] = np.log(bc / (r[neg] - a[neg]))
    return out


def _prism_primitive(X, Y, Z):
    r = np.sqrt(X * X + Y * Y + Z * Z)
    F = np.zeros_like(X)
    with np.errstate(divide="ignore", invalid="ignore"):
        for a, b, c in ((X, Y, Z), (Y, Z, X), (Z, X, Y)):
            # a b log(c + r)
            coef = a * b
            term = np.where(coef != 0.0, coef * _log_plus_r(c, a, b, r), 0.0)
            F = F + term
            # -(a^2/2) atan(b c / (a r))
            term = np.where(a != 0.0, -0.5 * a * a * np.arctan(b * c / (a * r)), 0.0)
            F = F + term
    return F


def block_potential(x: np.ndarray, lo, hi) -> np.ndarray:
    """U(x) = int_{lo}^{hi} dV(y) / |y - x| for points x (n, 3)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    U = np.zeros(x.shape[0])
    for sx, bx in ((-1.0, lo[0]), (1.0, hi[0])):
        for sy, by in ((-1.0, lo[1]), (1.0, hi[1])):
            for sz, bz in ((-1.0, lo[2]), (1.0, hi[2])):
                U += sx * sy * sz * _prism_primitive(bx - x[:, 0], by - x[:, 1], bz - x[:, 2])
    return U


def near_mean(x, q, d, K=(1, 1, 1), Rb: float = 0.0) -> float:
    """<phi_near>_box = sum_j q_j Phi_0(x_j) over the near set (Eq. pfx4).

    Without trimming the near set is the whole block of boxes, whose union gives
    U/V0 of the (2K+1)d block.  With the ball S_b of radius Rb (get step 2) every kept
    source image x_i - p contributes Phi_0(x_i - p) = U_box(x_i - p)/V0."""
    d = np.asarray(d, dtype=np.float64)
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    if Rb <= 0.0:
        half = 0.5 * (2 * np.asarray(K) + 1) * d
        U = block_potential(x, -half, half)
        return float(np.dot(q, U) / np.prod(d))
    total = 0.0
    for i1 in range(-K[0], K[0] + 1):
        for i2 in range(-K[1], K[1] + 1):
            for i3 in range(-K[2], K[2] + 1):
                xs = x - np.array([i1, i2, i3]) * d
                keep = np.sum(xs * xs, axis=1) <= Rb * Rb
                if np.any(keep):
                    total += float(np.dot(q[keep], block_potential(xs[keep], -0.5 * d, 0.5 * d)))
    return total / float(np.prod(d))


# ---------------------------------------------------------------------------
# "get", steps 1-3: near-field image sum (Eq. 3) -- the plain C loops of
# direct_sum.c.
# ---------------------------------------------------------------------------

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_near_sum.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp,
                                        ctypes.POINTER(ctypes.c_int32), dp, dp]
        lib.oracle_near_sum.restype = None
        lib.oracle_near_sum_ball.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp,
                                             ctypes.POINTER(ctypes.c_int32), ctypes.c_double, dp, dp]
        lib.oracle_near_sum_ball.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def near_sum(targets, x, q, d, K=(1, 1, 1), grad: bool = True, Rb: float = 0.0):
    lib = _load()
    targets = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    d = np.ascontiguousarray(d, dtype=np.float64)
    Karr = np.ascontiguousarray(K, dtype=np.int32)
    phi = np.zeros(targets.shape[0])
    g = np.zeros((targets.shape[0], 3)) if grad else None
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_near_sum_ball(targets.shape[0], targets.ctypes.data_as(dp), x.shape[0],
                             x.ctypes.data_as(dp), q.ctypes.data_as(dp), d.ctypes.data_as(dp),
                             Karr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(Rb),
                             phi.ctypes.data_as(dp), g.ctypes.data_as(dp) if grad else None)
    return (phi, g) if grad else phi


# ---------------------------------------------------------------------------
# The whole method.
# ---------------------------------------------------------------------------


class Plan:
    """Algorithm "set" (Sec. 2.3.1) for box d, maximum degree p, M check points."""

    def __init__(self, d, p: int, M: int, K=(1, 1, 1), checkpoints=None, lam: float = 0.0,
                 basis: str = "spherical", n_rbf: int = 256, rbf_radius: float = 0.0):
        """checkpoints: None (Fibonacci lattice of M points), "gauss" (the Gauss spherical
        grid; M is then (p+1)(2p+1)) or an explicit (M, 3) array on the sphere of radius R0.
        lam > 0 trims the near set to the ball of radius Rb = lam R0 (get step 2); the block
        of images is then the smallest one that covers the ball.
        basis "rbf" takes the n_rbf kernel functions of Eq. 5, centred at radius
        rbf_radius R0 (0: on S_b, i.e. at lambda_eff R0); P is then n_rbf + 1 (C_1 first)."""
        self.d = np.asarray(d, dtype=np.float64)
        self.p, self.K = int(p), tuple(int(k) for k in K)
        self.basis = basis
        if basis not in ("spherical", "rbf"):
            raise ValueError(basis)
        self.P = num_terms(p) if basis == "spherical" else int(n_rbf) + 1
        self.R0 = circumradius(self.d)                                   # step 1
        self.Rb = float(lam) * self.R0 if lam and lam > 0 else 0.0
        if self.Rb > 0.0:
            self.K = tuple(int(math.ceil(self.Rb / dk + 0.5)) for dk in self.d)
            self.lambda_eff = float(lam)
        else:   # the largest ball about the centre inside the block
            self.lambda_eff = float(min(0.5 * (2 * k + 1) * dk for k, dk in zip(self.K, self.d))) / self.R0
        if checkpoints is None:                                          # step 2
            self.Y = fibonacci_checkpoints(M, self.R0)
        elif isinstance(checkpoints, str) and checkpoints == "gauss":
            self.Y = gauss_checkpoints(self.p, self.R0)
        else:
            self.Y = np.asarray(checkpoints, dtype=np.float64)
        self.M = int(self.Y.shape[0])
        self.Yt = periodic_partners(self.Y, self.d)                      # step 3
        if basis == "spherical":
            self.A = fit_matrix(self.Y, self.Yt, self.p, self.R0)        # step 4
            self.factors = qr_factor(self.A)                             # step 5
            self.Rbox = box_integrals(self.d, self.p, self.R0)           # step 6
        else:
            Rs = (rbf_radius if rbf_radius and rbf_radius > 0 else self.lambda_eff) * self.R0
            self.centres = rbf_centres(int(n_rbf), Rs)
            self.A = fit_matrix_rbf(self.Y, self.Yt, self.centres)       # step 4
            self.factors = qr_factor(self.A)                             # step 5
            # step 6: the box mean of R_t is the single box's Newtonian potential at the
            # centre over V0 (App. C applies to the RBF far field, end of Sec. 3)
            self.Rbox = np.empty(self.P)
            self.Rbox[0] = 1.0
            self.Rbox[1:] = block_potential(self.centres, -0.5 * self.d, 0.5 * self.d) / float(np.prod(self.d))

    def coefficients(self, x, q, mean: str = "zero"):
        """"get" steps 3-6: near sums at the check points, f, C_2..C_P and C_1."""
        phi_y = near_sum(self.Y, x, q, self.d, self.K, grad=False, Rb=self.Rb)
        phi_yt = near_sum(self.Yt, x, q, self.d, self.K, grad=False, Rb=self.Rb)
        f = phi_yt - phi_y                                               # step 4
        C = np.zeros(self.P)
        C[1:] = qr_solve(self.factors, f)                                # step 5
        if mean == "zero":                                               # step 6
            C[0] = -near_mean(x, q, self.d, self.K, self.Rb) - float(np.dot(C[1:], self.Rbox[1:]))
        elif mean != "none":
            raise ValueError(mean)
        return C, f

    def far_field(self, C, targets, grad: bool = True):
        """"get" step 7: phi_far = sum_t C_t R_t(y/R0) and its gradient (Eqs. 1.8-1.9)."""
        targets = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
        if self.basis == "rbf":
            if grad:
                B, G = rbf_basis(targets, self.centres, grad=True)
                return C[0] + C[1:] @ B, np.einsum("t,tkn->nk", C[1:], G)
            return C[0] + C[1:] @ rbf_basis(targets, self.centres), None
        if grad:
            B, G = regular_basis(targets / self.R0, self.p, grad=True)
            return C @ B, np.einsum("t,tkn->nk", C, G) / self.R0
        return C @ regular_basis(targets / self.R0, self.p), None

    def evaluate(self, x, q, targets=None, grad: bool = True, mean: str = "zero",
                 parts: bool = False):
        """Algorithm "get" (Sec. 2.3.2).  Targets default to the sources (Y0 = X0)."""
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        q = np.asarray(q, dtype=np.float64).reshape(-1)
        if targets is None:
            targets = x
        C, f = self.coefficients(x, q, mean)
        if grad:
            phi_n, g_n = near_sum(targets, x, q, self.d, self.K, grad=True, Rb=self.Rb)  # step 3
        else:
            phi_n, g_n = near_sum(targets, x, q, self.d, self.K, grad=False, Rb=self.Rb), None
        phi_f, g_f = self.far_field(C, targets, grad)                         # step 7
        out = {"phi": phi_n + phi_f, "grad": (g_n + g_f) if grad else None}   # step 8
        if parts:
            out.update(phi_near=phi_n, grad_near=g_n, phi_far=phi_f, grad_far=g_f, C=C, f=f)
        return out


def energy_and_gradients(plan: "Plan", x, q, mean: str = "zero"):
    """E = 1/2 sum_j q_j phi(x_j) of the discrete method and its exact derivatives.

    With phi = phi_near + phi_far, C_{2..P} = A^+ f and f linear in q, the adjoint
    of the fit gives, for w_t = sum_j q_j R_t(x_j/R0) and u = (A^+)^T w,
        psi(x) = sum_l u_l [G(y~_l - x) - G(y_l - x)]   (G: the near-block kernel),
        dE/dq_k = phi_near(x_k) + phi_far(x_k)/2 + psi(x_k)/2,
        dE/dx_k = q_k [grad phi_near + grad phi_far / 2 + grad psi / 2](x_k).
    (The C_1 term contributes C_1/2 to dE/dq through sum_j q_j; it vanishes from E.)
    """
    if plan.basis != "spherical":
        raise NotImplementedError("energy derivatives with the RBF basis")
    if plan.Rb > 0.0:
        # with the ball the near set moves with each source, and the zero-mean constant
        # C_1 depends on which images are kept: the derivation above does not cover it
        raise NotImplementedError("energy derivatives of a ball-trimmed near set")
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    out = plan.evaluate(x, q, mean=mean, parts=True)
    B = regular_basis(x / plan.R0, plan.p)
    w = B[1:] @ q                                              # moments, t = 2..P
    Q, R, piv = plan.factors
    # A^+ = Pi R^-1 Q^T, so (A^+)^T w = Q R^-T (Pi^T w)
    u = Q @ scipy.linalg.solve_triangular(R, w[piv], trans="T", lower=False)
    src = np.concatenate([plan.Yt, plan.Y])
    c = np.concatenate([u, -u])
    psi, gpsi = near_sum(x, src, c, plan.d, plan.K, grad=True, Rb=plan.Rb)
    E = 0.5 * float(np.dot(q, out["phi"]))
    dEdq = out["phi_near"] + 0.5 * out["phi_far"] + 0.5 * psi
    dEdx = q[:, None] * (out["grad_near"] + 0.5 * out["grad_far"] + 0.5 * gpsi)
    return {"E": E, "dEdq": dEdq, "dEdx": dEdx, "psi": psi, "grad_psi": gpsi, "u": u, "w": w, **out}


def periodic_sum(x, q, d, p: int, M: int, targets=None, K=(1, 1, 1), grad: bool = True,
                 mean: str = "zero", parts: bool = False, checkpoints=None, lam: float = 0.0,
                 basis: str = "spherical", n_rbf: int = 256, rbf_radius: float = 0.0):
    """phi and grad phi of the periodic Coulomb sum at the targets (default: the sources)."""
    return Plan(d, p, M, K, checkpoints, lam, basis, n_rbf, rbf_radius).evaluate(
        x, q, targets, grad=grad, mean=mean, parts=parts)


def energy(x, q, d, p: int, M: int, K=(1, 1, 1)) -> float:
    """E = 1/2 sum_i q_i phi(x_i) (self term K(0) = 0 excluded, images included)."""
    out = periodic_sum(x, q, d, p, M, K=K, grad=False)
    return 0.5 * float(np.dot(q, out["phi"]))


def relative_l2(a, ref) -> float:
    """Eq. st2: ||a - ref||_2 / ||ref||_2 with the RMS norm over the sample."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    return float(np.sqrt(np.mean((a - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))
