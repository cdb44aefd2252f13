"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws positions and charges; it holds none of the method's
arithmetic.  Both the CUDA path (through the tests and the benchmark) and the
CPU oracle receive the arrays it returns.

Workloads (positions in the half-open box [-d/2, d/2)^3, Sec. 1):

* ``uniform_pm1``  -- N uniform points in the unit cube, half +1 and half -1
  charges, shuffled (random +-1 charges in a unit cube, Sec. 4.2).
* ``rock_salt``    -- the NaCl lattice: n^3 ions on a simple cubic grid of
  spacing d/n with alternating charges (Sec. 4.1, Eq. st1), optionally with
  Gaussian jitter of 0.05 spacing.
* ``uniform_gauss`` -- N uniform points in a rectangular box, Gaussian
  charges shifted to zero net charge (box aspect ratios, Table 5).
* ``batch``        -- many independent systems of uneven size, box shape and
  expansion degree.
* ``dipole_pairs`` -- tight +-q dipole pairs at uniform random centres in an
  elongated box (wrapped periodically into the box).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class System:
    """One periodic system: box, expansion degree p, check-point count M."""

    x: np.ndarray          # (N, 3) float64, inside [-d/2, d/2)
    q: np.ndarray          # (N,) float64, sum zero
    d: tuple               # box edge lengths (d1, d2, d3)
    p: int                 # maximum degree of the local expansion
    M: int                 # number of check points
    name: str = ""
    meta: dict = field(default_factory=dict)
    K: tuple = (1, 1, 1)   # near block: images |i_k| <= K_k of the box (Eq. 3)

    @property
    def N(self) -> int:
        return int(self.x.shape[0])


def _clip_into_box(x: np.ndarray, d) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64)
    hi = np.nextafter(d / 2, 0.0)
    return np.minimum(np.maximum(x, -d / 2), hi)


def _wrap_into_box(x: np.ndarray, d) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64)
    y = x - d * np.floor(x / d + 0.5)
    return _clip_into_box(y, d)


def uniform_pm1(N: int = 1000, p: int = 8, M: int = 200, seed: int = 0) -> System:
    """N uniform points in the unit cube, N/2 charges +1 and N/2 charges -1."""
    if N % 2:
        raise ValueError("N must be even for a +-1 neutral system")
    rng = np.random.default_rng(seed)
    d = (1.0, 1.0, 1.0)
    x = _clip_into_box(rng.uniform(-0.5, 0.5, size=(N, 3)), d)
    q = np.concatenate([np.ones(N // 2), -np.ones(N // 2)])
    rng.shuffle(q)
    return System(x, q, d, p, M, name=f"uniform_pm1_N{N}_p{p}_M{M}")


def rock_salt(n: int = 16, p: int = 12, M: int = 400, jitter: bool = False,
              seed: int = 1, d: float = 1.0) -> System:
    """Rock-salt lattice of n^3 ions (n even) in a cube of edge d.

    Ion (i, j, k) sits at ((i + 1/2) a - d/2, ...) with a = d/n and charge
    (-1)^(i+j+k).  Nearest-neighbour distance is a, so q_i phi(x_i) a equals
    minus the Madelung constant of NaCl for every ion.
    """
    if n % 2:
        raise ValueError("n must be even for a neutral periodic rock-salt cell")
    a = d / n
    idx = np.arange(n)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    x = np.stack([(I + 0.5) * a - d / 2, (J + 0.5) * a - d / 2, (K + 0.5) * a - d / 2],
                 axis=-1).reshape(-1, 3)
    q = ((-1.0) ** (I + J + K)).reshape(-1).astype(np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        x = _clip_into_box(x + rng.normal(0.0, 0.05 * a, size=x.shape), (d, d, d))
    name = f"rock_salt_{n}^3{'_jitter' if jitter else ''}_p{p}_M{M}"
    return System(x, q, (d, d, d), p, M, name=name, meta={"spacing": a})


def uniform_gauss(N: int = 100_000, d=(1.0, 1.5, 2.0), p: int = 16, M: int = 800,
                  seed: int = 2) -> System:
    """N uniform points in a rectangular box, q ~ N(0,1) minus its mean."""
    rng = np.random.default_rng(seed)
    d = tuple(float(v) for v in d)
    x = _clip_into_box(rng.uniform(-0.5, 0.5, size=(N, 3)) * np.asarray(d), d)
    q = rng.normal(0.0, 1.0, size=N)
    q = q - q.mean()
    return System(x, q, d, p, M, name=f"uniform_gauss_N{N}_d{d}_p{p}_M{M}")


def dipole_pairs(n_pairs: int = 100_000, d=(1.0, 1.0, 2.0), p: int = 16, M: int = 800,
                 sep: float = 0.01, charge: float = 0.8, seed: int = 4) -> System:
    """Tight dipoles: +q at c + sep/2 e, -q at c - sep/2 e, c uniform, e a random unit vector."""
    rng = np.random.default_rng(seed)
    d = tuple(float(v) for v in d)
    c = rng.uniform(-0.5, 0.5, size=(n_pairs, 3)) * np.asarray(d)
    e = rng.normal(size=(n_pairs, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    xp = _wrap_into_box(c + 0.5 * sep * d[0] * e, d)
    xm = _wrap_into_box(c - 0.5 * sep * d[0] * e, d)
    x = np.empty((2 * n_pairs, 3))
    x[0::2], x[1::2] = xp, xm
    q = np.empty(2 * n_pairs)
    q[0::2], q[1::2] = charge, -charge
    return System(x, q, d, p, M, name=f"dipole_pairs_{n_pairs}_d{d}_p{p}_M{M}")


# The batch mixes three (p, M) settings, as in the uniform choice p in {8, 12, 16}.
BATCH_PM = ((8, 200), (12, 400), (16, 800))


def batch(B: int = 256, n_lo: int = 500, n_hi: int = 20000, seed: int = 3) -> list:
    """B independent neutral +-1 systems of uneven size and box shape.

    N is log-uniform in [n_lo, n_hi] (rounded down to even), d = (1, U[1,2], U[1,2])
    and (p, M) is drawn uniformly from ``BATCH_PM``.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        N = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        N -= N % 2
        d = (1.0, float(rng.uniform(1.0, 2.0)), float(rng.uniform(1.0, 2.0)))
        p, M = BATCH_PM[int(rng.integers(0, len(BATCH_PM)))]
        x = _clip_into_box(rng.uniform(-0.5, 0.5, size=(N, 3)) * np.asarray(d), d)
        q = np.concatenate([np.ones(N // 2), -np.ones(N // 2)])
        rng.shuffle(q)
        out.append(System(x, q, d, p, M, name=f"batch{b}_N{N}", K=batch_near_block(d)))
    return out


def batch_near_block(d) -> tuple:
    """Configuration rule of the batch workload: the 3x3x3 block, widened along the short
    axes of flat boxes.  The largest ball about the box centre inside the 3x3x3 block has
    radius 1.5 min(d); when that is under 1.1 times the circumscribed radius |d|/2 (the
    truncation error then barely falls with p), K_k = max(1, ceil(1.25 |d|/(2 d_k) - 1/2))
    makes it at least 1.25 times."""
    h = 0.5 * math.sqrt(sum(v * v for v in d))
    if 1.5 * min(d) >= 1.1 * h:
        return (1, 1, 1)
    return tuple(max(1, int(math.ceil(1.25 * h / v - 0.5))) for v in d)


def config(k: int, small: bool = False):
    """The five benchmark workloads (1-based); ``small`` gives a reduced copy
    the oracle finishes in seconds but that still spans several tiles."""
    if k == 1:
        return uniform_pm1(N=1000 if not small else 402, p=8, M=200, seed=0)
    if k == 2:
        return rock_salt(n=16 if not small else 8, p=12, M=400)
    if k == 3:
        return uniform_gauss(N=100_000 if not small else 3001, d=(1.0, 1.5, 2.0),
                             p=16, M=800, seed=2)
    if k == 4:
        return batch(B=256, seed=3) if not small else batch(B=6, n_lo=60, n_hi=1500, seed=3)
    if k == 5:
        return dipole_pairs(n_pairs=100_000 if not small else 1500, d=(1.0, 1.0, 2.0),
                            p=16, M=800, seed=4)
    raise ValueError(k)
