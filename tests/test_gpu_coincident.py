"""Charges that share a position (Eq. 1: K(0) = 0 drops every pair at distance zero, not only a
charge and itself).  Sorted along the spatial order, charges at one position are neighbours,
but a group boundary can fall between them; the float32 and float-float paths then form their
offset from two different group origins, and the rounding of those offsets leaves a tiny
nonzero distance.  The near units take such pairs as coincident (coincident_r2 in
csrc/near_common.cuh), so every path matches the FP64 oracle, which drops exact zeros.

Cases: every position holding three charges (group boundaries of 128 fall inside triples),
and clumps of 130 charges at one point (a group of identical positions, radius 0, spilling
into the next group) among uniform charges; both charge kernels, all three precisions."""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import assert_close
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32c": 1e-6, "ff": 1e-10}
D = (1.0, 1.5, 2.0)


def _triples():
    rng = np.random.default_rng(3)
    base = (rng.uniform(-0.5, 0.5, (1200, 3)) * np.asarray(D))
    x = np.repeat(base, 3, axis=0)
    q = rng.normal(size=len(x))
    q -= q.mean()
    return W.System(x, q, D, 8, 200, name="triples")


def _clumps():
    rng = np.random.default_rng(4)
    pts = rng.uniform(-0.45, 0.45, (6, 3)) * np.asarray(D)
    x = np.concatenate([np.repeat(pts, 130, axis=0), rng.uniform(-0.5, 0.5, (2400, 3)) * np.asarray(D)])
    q = rng.normal(size=len(x))
    q -= q.mean()
    return W.System(x, q, D, 8, 200, name="clumps")


CASES = {"triples": _triples, "clumps": _clumps}
_REF = {}


@pytest.mark.parametrize("pairs", ["one-sided", "symmetric"])
@pytest.mark.parametrize("precision", ["fp64", "fp32c", "ff"])
@pytest.mark.parametrize("name", list(CASES))
def test_coincident_charges_match_the_oracle(name, precision, pairs):
    s = CASES[name]()
    if name not in _REF:
        _REF[name] = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, mean="zero", parts=True)
    ref = _REF[name]
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, pairs=pairs)
    try:
        phi, g = pc(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.q, device="cuda"))
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
    assert_close(phi, ref["phi"], TOL[precision], f"{name}/{precision}/{pairs} phi")
    assert_close(g, ref["grad"], TOL[precision], f"{name}/{precision}/{pairs} grad")
