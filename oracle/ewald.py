"""ORACLE -- test infrastructure only.

Classic Ewald summation of the periodic Coulomb sum (App. D), used to check
the oracle's periodisation against an independent route to the same
conditionally convergent sum.

The kernel is split as in Eq. e1, K = erfc(xi r)/r + erf(xi r)/r, with
K_1(0) = -2 xi / sqrt(pi) so that K(0) = 0.  The short-range part (Eq. e3) is
summed directly over every image within the real-space cutoff; the smooth part
(Eqs. e4-e5) is summed exactly over reciprocal vectors k != 0 (the k = 0
harmonic is zeroed, which gives the zero-mean potential of Eq. e6) instead of
on an FFT grid.  No surface (dipole) term is added.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def ewald(targets, x, q, d, xi: float | None = None, grad: bool = True,
          digits: float = 6.2, chunk: int = 4096):
    """phi and grad phi of the periodic sum at ``targets`` by Ewald summation.

    ``digits`` sets both cutoffs: erfc(xi r_c) and exp(-k_c^2 / (4 xi^2)) are
    about exp(-digits^2) (~2e-17 for the default).
    """
    targets = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    d = np.asarray(d, dtype=np.float64)
    V = float(np.prod(d))
    if xi is None:
        xi = 3.5 / float(np.min(d))
    rc = digits / xi
    kc = 2.0 * xi * digits
    nt = targets.shape[0]
    phi = np.zeros(nt)
    g = np.zeros((nt, 3))

    # real-space part (Eq. e3): every image of every source within rc
    nimg = [int(math.ceil(rc / d[k])) + 1 for k in range(3)]
    shifts = np.array([(i, j, k) for i in range(-nimg[0], nimg[0] + 1)
                       for j in range(-nimg[1], nimg[1] + 1)
                       for k in range(-nimg[2], nimg[2] + 1)], dtype=np.float64) * d
    two_over_sqrtpi = 2.0 / math.sqrt(math.pi)
    tchunk = max(1, 2_000_000 // max(1, x.shape[0]))
    for s0 in range(0, nt, tchunk):
        t = targets[s0:s0 + tchunk]
        ph = np.zeros(t.shape[0])
        gg = np.zeros((t.shape[0], 3))
        for sh in shifts:
            r = t[:, None, :] - (x[None, :, :] + sh)          # (nt, ns, 3)
            rr = np.sqrt(np.sum(r * r, axis=2))
            mask = (rr > 0) & (rr < rc)
            rs = np.where(mask, rr, 1.0)
            e = np.where(mask, erfc(xi * rs) / rs, 0.0)
            ph += e @ q
            if grad:
                dk = np.where(mask, -(e / rs + two_over_sqrtpi * xi * np.exp(-(xi * rs) ** 2) / rs)
                              / rs, 0.0)                      # (1/r) d/dr [erfc(xi r)/r]
                gg += np.einsum("ts,tsk->tk", dk * q[None, :], r)
            # self term K_1(0) = -2 xi / sqrt(pi) (Eq. e1) where a target sits on a source
            zero = rr == 0
            if np.any(zero):
                ph += -two_over_sqrtpi * xi * (zero.astype(np.float64) @ q)
        phi[s0:s0 + tchunk] = ph
        g[s0:s0 + tchunk] = gg

    # reciprocal part (Eqs. e4-e5), k = 2 pi (n1/d1, n2/d2, n3/d3), k != 0
    nk = [int(math.ceil(kc * d[k] / (2 * math.pi))) for k in range(3)]
    n1, n2, n3 = np.meshgrid(np.arange(-nk[0], nk[0] + 1), np.arange(-nk[1], nk[1] + 1),
                             np.arange(-nk[2], nk[2] + 1), indexing="ij")
    kv = 2 * math.pi * np.stack([n1.reshape(-1) / d[0], n2.reshape(-1) / d[1],
                                 n3.reshape(-1) / d[2]], axis=1)
    k2 = np.sum(kv * kv, axis=1)
    keep = (k2 > 0) & (k2 <= kc * kc)
    kv, k2 = kv[keep], k2[keep]
    coef = (4 * math.pi / V) * np.exp(-k2 / (4 * xi * xi)) / k2
    for s0 in range(0, kv.shape[0], chunk):
        kk = kv[s0:s0 + chunk]
        cc = coef[s0:s0 + chunk]
        S = np.exp(-1j * (x @ kk.T)).T @ q                    # structure factor S(k)
        E = np.exp(1j * (targets @ kk.T))                     # (nt, nk)
        Z = E * (cc * S)[None, :]
        phi += np.real(Z).sum(axis=1)
        if grad:
            g += -(np.imag(Z) @ kk)
    return (phi, g) if grad else phi
