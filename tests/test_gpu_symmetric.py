"""GPU parity of the symmetric charge kernel (PSUM_PAIRS_SYMMETRIC).

The pair (i, j, p) and its mirror (j, i, -p) are one distance apart, so the kernels form
one offset and one 1/r for both and add the source's terms (the reaction) as well as the
target's; the tiles' pairs (a < b) each run once with every image of the block, a tile
against itself runs one-sided.  They compute the same sums as the one-sided kernels in a
different rounding order, so both are held to the path's bound (relative L2 error, Eq. st2:
1e-6 FP32C, 1e-10 FP64 and float-float) against the FP64 oracle, and to each other (1e-6, 1e-12,
1e-11).  The cases cover one to five tiles of
512 charges, a last tile with a single charge, partly filled chunks, a tight cluster (every
unit near), close dipole pairs (the float-float near units on both sides of a pair), a wider
near block and every image grouping of the work items.
"""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import MAX_FACTOR, errors
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32c": 1e-6, "fp64": 1e-10, "ff": 1e-10}
TOL_BETWEEN = {"fp32c": 1e-6, "fp64": 1e-12, "ff": 1e-11}     # symmetric against one-sided


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _run(s, pairs, K=(1, 1, 1), precision="fp32c"):
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, K=K, pairs=pairs)
    try:
        phi, g = pc(_dev(s.x), _dev(s.q))
        return phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()


def _eps(a, b):
    """max(eps2, (largest element error) / MAX_FACTOR): under a tolerance only if the norm and
    every single value are within it (parity_check)."""
    e2, emax = errors(a, b)
    return max(e2, emax / MAX_FACTOR)


def _clustered(N=2000, seed=11):
    # every charge within 0.06 of one point: all tile pairs are near units (float-float
    # offsets and compensated sums on both sides of every pair)
    rng = np.random.default_rng(seed)
    x = 0.06 * rng.normal(size=(N, 3)) / 3.0
    x = np.clip(x, -0.49, 0.49)
    q = rng.normal(size=N)
    q -= q.mean()
    return W.System(x, q, (1.0, 1.0, 1.0), 8, 200, name=f"clustered_{N}")


CASES = [
    ("clustered_2000", lambda: _clustered(), (1, 1, 1)),
    ("one_tile_402", lambda: W.config(1, small=True), (1, 1, 1)),
    ("two_tiles_513", lambda: W.uniform_gauss(N=513, d=(1.0, 1.5, 2.0), p=8, M=200, seed=5), (1, 1, 1)),
    ("three_tiles_1300", lambda: W.uniform_gauss(N=1300, d=(1.0, 1.5, 2.0), p=12, M=400, seed=6), (1, 1, 1)),
    ("cfg3_small_3001", lambda: W.config(3, small=True), (1, 1, 1)),
    ("dipoles_2400", lambda: W.dipole_pairs(n_pairs=1200, d=(1.0, 1.0, 2.0), p=12, M=400, seed=7), (1, 1, 1)),
    ("wide_block_1100", lambda: W.uniform_gauss(N=1100, d=(2.0, 1.0, 1.0), p=8, M=200, seed=8), (2, 1, 1)),
]


_REF = {}


@pytest.mark.parametrize("precision", ["fp32c", "fp64", "ff"])
@pytest.mark.parametrize("name,make,K", CASES, ids=[c[0] for c in CASES])
def test_symmetric_kernel_against_oracle_and_one_sided(name, make, K, precision):
    s = make()
    phi_s, g_s = _run(s, "symmetric", K, precision)
    phi_o, g_o = _run(s, "one-sided", K, precision)
    if name not in _REF:
        _REF[name] = O.Plan(s.d, s.p, s.M, K=K).evaluate(s.x, s.q, mean="zero", parts=True)
    ref = _REF[name]
    tol = TOL[precision]
    for phi, g, what in ((phi_s, g_s, "symmetric"), (phi_o, g_o, "one-sided")):
        e_phi, e_g = _eps(phi, ref["phi"]), _eps(g, ref["grad"])
        assert e_phi < tol and e_g < tol, f"{name}/{precision}/{what}: eps2 phi {e_phi:.3e}, grad {e_g:.3e}"
    tb = TOL_BETWEEN[precision]
    assert _eps(phi_s, phi_o) < tb and _eps(g_s, g_o) < tb


def test_symmetric_kernel_is_deterministic():
    s = W.uniform_gauss(N=2900, d=(1.0, 1.5, 2.0), p=8, M=200, seed=9)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c", pairs="symmetric")
    try:
        x, q = _dev(s.x), _dev(s.q)
        phi0, g0 = pc(x, q)
        for _ in range(3):
            phi, g = pc(x, q)
            assert torch.equal(phi, phi0) and torch.equal(g, g0)
    finally:
        pc.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64", "ff"])
def test_automatic_choice_matches_the_forced_kernels(precision):
    # FP32C takes the symmetric kernel automatically from 12 tiles of 512 charges, FF from 6,
    # FP64 at every size
    s = W.uniform_gauss(N=16 * 512 + 77, d=(1.0, 1.5, 2.0), p=8, M=200, seed=10)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision)
    try:
        assert B.psum_pair_kernel(pc.plan, s.N)[0] == "symmetric"
        small = {"fp32c": (11 * 512, "one-sided"), "ff": (5 * 512, "one-sided"), "fp64": (1000, "symmetric")}
        n, kernel = small[precision]
        assert B.psum_pair_kernel(pc.plan, n)[0] == kernel
        if precision == "ff":
            assert B.psum_pair_kernel(pc.plan, 6 * 512)[0] == "symmetric"
    finally:
        pc.close()
    phi_a, g_a = _run(s, "auto", precision=precision)
    phi_s, g_s = _run(s, "symmetric", precision=precision)
    phi_o, g_o = _run(s, "one-sided", precision=precision)
    assert np.array_equal(phi_a, phi_s) and np.array_equal(g_a, g_s)
    tb = TOL_BETWEEN[precision]
    assert _eps(phi_s, phi_o) < tb and _eps(g_s, g_o) < tb
