"""Agreement of a GPU result with its reference, norm-wise and element by element.

eps2 is the error metric of Eq. st2 (Sec. 4.1): the RMS of the difference over the RMS
of the reference.  Beside it every comparison bounds each single difference,
|a_i - ref_i| / (rms(ref) + |ref_i|), so that a few wrong values cannot hide in the norm (at
N values a norm dilutes one wrong value by 1/sqrt(N)); a wrong value scores about 1/2.
The |ref_i| in the scale keeps values far above the rms (the field of a charge with a close
neighbour, say) to the relative accuracy of the arithmetic instead of an absolute one.
The bound is MAX_FACTOR times the eps2 tolerance: for errors that are sums of many
independent roundings the largest of N values sits about sqrt(2 ln N) (under 5 for
N <= 3e5) rms widths out, so at an eps2 right at its tolerance the largest value still has
a margin of two.
"""
import numpy as np

MAX_FACTOR = 10.0


def errors(a, ref, scale=None):
    """(eps2, max_i |a_i - ref_i| / (s + |ref_i|)) with s = rms(ref), or `scale` where given."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    rms = float(np.sqrt(np.mean(ref ** 2))) if scale is None else float(scale)
    d = a - ref
    return float(np.sqrt(np.mean(d ** 2)) / rms), float(np.max(np.abs(d) / (rms + np.abs(ref))))


def assert_close(a, ref, tol, what="", max_tol=None, scale=None):
    e2, emax = errors(a, ref, scale)
    mt = MAX_FACTOR * tol if max_tol is None else max_tol
    assert e2 < tol and emax < mt, (f"{what}: eps2 {e2:.3e} (tol {tol:.1e}), "
                                    f"max element {emax:.3e} (tol {mt:.1e})")
    return e2, emax


def full_size_sample(x, d, n=4096, cluster=1100, seed=0):
    """Sorted indices of n charges for a sampled full-size comparison: every charge of three
    compact clusters -- the `cluster` charges nearest (in box-normalised max norm) to the
    corners of the box where the spatial (Hilbert) order of the charges starts, (-1/2, -1/2,
    -1/2), and ends, (1/2, -1/2, -1/2), and to its centre -- so that whole target tiles at both
    ends of the order and in the middle are compared, plus charges drawn at random up to n."""
    x = np.asarray(x, dtype=np.float64)
    u = x / np.asarray(d, dtype=np.float64)              # in [-1/2, 1/2)
    picks = set()
    for c in ((-0.5, -0.5, -0.5), (0.5, -0.5, -0.5), (0.0, 0.0, 0.0)):
        dist = np.max(np.abs(u - np.asarray(c)), axis=1)
        picks.update(np.argsort(dist, kind="stable")[:cluster].tolist())
    rng = np.random.default_rng(seed)
    rest = np.setdiff1d(np.arange(len(x)), np.fromiter(picks, dtype=np.int64))
    need = max(0, min(n, len(x)) - len(picks))
    picks.update(rng.choice(rest, size=need, replace=False).tolist())
    return np.sort(np.fromiter(picks, dtype=np.int64))
