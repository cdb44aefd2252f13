"""GPU tests of the symmetric charge kernel's banded partial sums and of the refined float32
terms (PSUM_TERMS_REFINED).

Bands: a system whose square of tile-pair partial slots passes the band cap runs the pair
kernel band by band (row tiles a0 <= a < a1), each band's slots reduced into the float64
near-field sums before the next.  The slots hold the same values as in one band (every slot
is written by one work item, whatever the band), so banded and single-band results differ only
by the grouping of float64 additions: held to 1e-13 against each other and to the path's bound
against the oracle.  A test hook lowers the cap so that small systems run many bands.

Refined terms: 1/r as the rsqrt estimate plus its Newton correction fused into the sums, exact
offsets (Fast2Sum) and the target offsets rounded once -- parity against the oracle at the
FP32C bound, never a larger error than the fast terms by more than the sampling noise.
"""
import numpy as np
import pytest

from oracle import psum_oracle as O
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W
from parity_check import assert_close, errors, full_size_sample

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32c": 1e-6, "fp64": 1e-10, "ff": 1e-10}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _run(s, precision="fp32c", band_bytes=0, terms="fast", pairs="auto", graph=False):
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, pairs=pairs, terms=terms)
    try:
        B.psum_debug_band_bytes(pc.plan, band_bytes)
        kernel = B.psum_pair_kernel(pc.plan, s.N)[0]
        nbytes, bands = B.psum_scratch_bytes(pc.plan, s.N)
        x, q = _dev(s.x), _dev(s.q)
        if graph:
            phi = torch.empty(s.N, dtype=torch.float64, device="cuda")
            g = torch.empty((s.N, 3), dtype=torch.float64, device="cuda")
            for _ in range(2):
                B.psum_eval_graph(pc.plan, x, q, phi, g, check=True)
        else:
            phi, g = pc(x, q)
        return phi.cpu().numpy(), g.cpu().numpy(), kernel, bands, nbytes
    finally:
        pc.close()


_REF = {}


def _oracle(s):
    if s.name not in _REF:
        _REF[s.name] = O.periodic_sum(s.x, s.q, s.d, s.p, s.M, parts=True)
    return _REF[s.name]


# band caps that split these systems into many bands: float32 slots are 16 KiB (4 x 512
# doubles), float64 slots 4 KiB (4 x 128)
BANDED = [("fp32c", 20_000, 4 << 20), ("ff", 6_000, 1 << 20), ("fp64", 5_000, 1 << 19)]


@pytest.mark.parametrize("precision,N,cap", BANDED, ids=[b[0] for b in BANDED])
def test_bands_match_one_band_and_the_oracle(precision, N, cap):
    s = W.uniform_gauss(N=N, d=(1.0, 1.5, 2.0), p=8, M=200, seed=40 + N % 7)
    p1, g1, k1, b1, n1 = _run(s, precision)
    pb, gb, kb, bb, nb = _run(s, precision, band_bytes=cap)
    assert k1 == kb == "symmetric"
    assert b1 == 1 and bb > 3, (b1, bb)
    assert nb < n1
    # the same slot values, reduced in another grouping of float64 additions
    assert_close(pb, p1, 1e-13, "phi banded vs one band")
    assert_close(gb, g1, 1e-13, "grad banded vs one band")
    rng = np.random.default_rng(1)
    k = np.sort(rng.choice(s.N, size=512, replace=False))
    ref = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, targets=s.x[k])
    assert_close(pb[k], ref["phi"], TOL[precision], "phi banded vs oracle")
    assert_close(gb[k], ref["grad"], TOL[precision], "grad banded vs oracle")


def test_bands_are_deterministic_and_replay_in_a_graph():
    s = W.uniform_gauss(N=9000, d=(1.0, 1.0, 1.0), p=8, M=200, seed=44)
    a = _run(s, band_bytes=2 << 20)
    b = _run(s, band_bytes=2 << 20)
    c = _run(s, band_bytes=2 << 20, graph=True)
    assert a[3] > 1
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])


def test_last_band_of_a_ragged_system():
    # 23 tiles in bands of 2: the last band holds one tile; the last tile holds one charge.  A
    # first band of width 2 takes 2 x 2 x 23 - 4 slots of 4 x 512 doubles per image group.
    s = W.uniform_gauss(N=22 * 512 + 1, d=(1.0, 1.5, 2.0), p=8, M=200, seed=45)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        n_g = B.psum_pair_kernel(pc.plan, s.N)[1]
    finally:
        pc.close()
    p1, g1, _, _, _ = _run(s)
    pb, gb, _, bb, _ = _run(s, band_bytes=(2 * 2 * 23 - 4) * n_g * 16384)
    assert bb == 12
    assert_close(pb, p1, 1e-13, "phi")
    assert_close(gb, g1, 1e-13, "grad")


REFINED = [("cfg5_small", lambda: W.config(5, small=True)),
           ("cfg3_small", lambda: W.config(3, small=True)),
           ("dipoles_6000", lambda: W.dipole_pairs(n_pairs=3000, p=12, M=400, seed=46)),
           ("ragged_1025", lambda: W.uniform_gauss(N=1025, d=(1.0, 1.5, 2.0), p=8, M=200, seed=47))]


@pytest.mark.parametrize("name,make", REFINED, ids=[r[0] for r in REFINED])
def test_refined_terms_against_the_oracle(name, make):
    s = make()
    ref = _oracle(s)
    pf, gf, kf, _, _ = _run(s, pairs="symmetric")
    pr, gr, kr, _, _ = _run(s, pairs="symmetric", terms="refined")
    assert kf == kr == "symmetric"
    assert_close(pr, ref["phi"], TOL["fp32c"], f"{name} refined phi")
    assert_close(gr, ref["grad"], TOL["fp32c"], f"{name} refined grad")
    # the refinement removes roundings of the potential's terms: never clearly worse
    assert errors(pr, ref["phi"])[0] <= 1.05 * errors(pf, ref["phi"])[0]


def test_refined_terms_in_bands():
    s = W.dipole_pairs(n_pairs=6000, p=12, M=400, seed=48)
    p1, g1, _, _, _ = _run(s, terms="refined")
    pb, gb, _, bb, _ = _run(s, terms="refined", band_bytes=2 << 20)
    assert bb > 1
    assert_close(pb, p1, 1e-13, "phi")
    assert_close(gb, g1, 1e-13, "grad")


def test_half_million_charges_in_bands_under_2_gb():
    # 977 tiles of 512: the full square of partial slots would take 15.6 GB; the bands keep the
    # scratch under 2 GB.  1024 sampled charges (clusters at both ends of the spatial order and
    # in the middle) against the oracle.
    s = W.uniform_gauss(N=500_000, d=(1.0, 1.5, 2.0), p=8, M=200, seed=49)
    phi, g, kernel, bands, nbytes = _run(s)
    assert kernel == "symmetric" and bands > 1
    assert nbytes < 2_000_000_000, nbytes
    k = full_size_sample(s.x, s.d, 1024, cluster=300, seed=49)
    ref = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, targets=s.x[k])
    assert_close(phi[k], ref["phi"], TOL["fp32c"], "phi")
    assert_close(g[k], ref["grad"], TOL["fp32c"], "grad")
