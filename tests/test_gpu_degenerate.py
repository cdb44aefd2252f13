"""Degenerate inputs on the GPU against the oracle, every precision and both charge kernels.

* Charges that share a position (Eq. 1: K(0) = 0 drops every pair at distance zero, not only a
  charge and itself).  Sorted along the spatial order, charges at one position are neighbours,
  but a group boundary can fall between them; the float32 and float-float paths then form their
  offset from two different group origins, and the rounding of those offsets leaves a tiny
  nonzero distance.  The near units take such pairs as coincident (coincident_r2 in
  csrc/psum_internal.cuh), so every path matches the FP64 oracle, which drops exact zeros.
  Cases: every position holding three charges (group boundaries of 128 fall inside triples),
  and clumps of 130 charges at one point (a group of identical positions, radius 0, spilling
  into the next group) among uniform charges.
* Flat geometries: all charges in one plane, all on one line (groups of zero extent along
  one or two axes), and charges on the box's lower faces (the half-open box's boundary).
* A tight cluster: 1500 charges within about 1e-6 of one point among uniform ones.

The float-float path forms offsets from group origins with about 48 bits, an absolute error of
about 2^-48 of the group radius; where pairs sit far closer than their groups' size -- a 1e-6
cluster whose first and last charges share groups with the uniform ones around it, a line
whose groups are long and thin -- its relative accuracy falls to that ratio (measured: 4e-9 on
the cluster, 1.3e-10 on the line) and the test holds it to the bound stated per case; FP64
forms offsets from absolute positions and keeps 1e-10 throughout."""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import assert_close
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32c": 1e-6, "ff": 1e-10}
FF_TOL = {"line": 1e-9, "tight": 1e-7}      # the float-float path where pairs are far below group size
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


def _with_charges(x, seed, name):
    q = np.random.default_rng(seed).normal(size=len(x))
    q -= q.mean()
    return W.System(np.ascontiguousarray(x), q, D, 8, 200, name=name)


def _plane():
    x = np.random.default_rng(21).uniform(-0.5, 0.5, (2500, 3)) * np.asarray(D)
    x[:, 2] = 0.0
    return _with_charges(x, 31, "plane")


def _line():
    x = np.random.default_rng(22).uniform(-0.5, 0.5, (2500, 3)) * np.asarray(D)
    x[:, 1] = 0.0
    x[:, 2] = 0.0
    return _with_charges(x, 32, "line")


def _tight():
    rng = np.random.default_rng(23)
    x = np.concatenate([0.2 + 1e-6 * rng.normal(size=(1500, 3)), rng.uniform(-0.5, 0.5, (1500, 3)) * np.asarray(D)])
    return _with_charges(x, 33, "tight")


def _faces():
    x = np.random.default_rng(24).uniform(-0.5, 0.5, (2500, 3)) * np.asarray(D)
    x[:800, 0] = -0.5 * D[0]
    x[800:1600, 1] = -0.5 * D[1]
    return _with_charges(x, 34, "faces")


CASES = {"triples": _triples, "clumps": _clumps, "plane": _plane, "line": _line, "tight": _tight,
         "faces": _faces}
_REF = {}


@pytest.mark.parametrize("pairs", ["one-sided", "symmetric"])
@pytest.mark.parametrize("precision", ["fp64", "fp32c", "ff"])
@pytest.mark.parametrize("name", list(CASES))
def test_degenerate_inputs_match_the_oracle(name, precision, pairs):
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
    tol = FF_TOL.get(name, TOL["ff"]) if precision == "ff" else TOL[precision]
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
    assert_close(phi, ref["phi"], tol, f"{name}/{precision}/{pairs} phi")
    assert_close(g, ref["grad"], tol, f"{name}/{precision}/{pairs} grad")


@pytest.mark.parametrize("precision,pairs", [("fp32c", "one-sided"), ("fp32c", "symmetric"), ("ff", "auto")])
def test_degenerate_systems_in_one_batch(precision, pairs):
    """The batch tables carry each system's coincidence threshold (charge and check-point
    launches, both charge kernels): coincident triples, clumps and a plane in one batch."""
    systems = [CASES[n]() for n in ("triples", "clumps", "plane")]
    pb = B.PeriodicBatch(systems, precision=precision, pairs=pairs)
    try:
        x = torch.as_tensor(np.concatenate([s.x for s in systems]), device="cuda")
        q = torch.as_tensor(np.concatenate([s.q for s in systems]), device="cuda")
        phi, g = pb(x, q)
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
        for b, s in enumerate(systems):
            if s.name not in _REF:
                _REF[s.name] = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, mean="zero", parts=True)
            sl = slice(pb.offsets[b], pb.offsets[b + 1])
            assert np.all(np.isfinite(phi[sl])) and np.all(np.isfinite(g[sl]))
            assert_close(phi[sl], _REF[s.name]["phi"], TOL[precision], f"batch {s.name}/{precision}/{pairs} phi")
            assert_close(g[sl], _REF[s.name]["grad"], TOL[precision], f"batch {s.name}/{precision}/{pairs} grad")
    finally:
        pb.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "ff"])
def test_evaluation_points_on_charges_in_other_groups(precision):
    """Evaluation points at a subset of the charge positions (plus points between them): sorted
    and grouped on their own, so a point and the charge it sits on lie in different groups; the
    pair is dropped (K(0) = 0) as in the oracle, which skips exact zeros."""
    s = _triples()
    rng = np.random.default_rng(9)
    y = np.concatenate([s.x[rng.choice(len(s.x), 700, replace=False)],
                        rng.uniform(-0.5, 0.5, (300, 3)) * np.asarray(D)])
    ref = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, targets=y, parts=True)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision)
    try:
        phi, g = pc.at(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.q, device="cuda"),
                       torch.as_tensor(y, device="cuda"))
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
    assert_close(phi, ref["phi"], TOL[precision], f"points/{precision} phi")
    assert_close(g, ref["grad"], TOL[precision], f"points/{precision} grad")
