"""The benchmark's full-size workloads on the GPU, checked where the oracle can follow:
sampled outputs of the 200k-charge dipole system (forward and the exact adjoint), the full
256-system batch against single-system evaluations and, for its smallest systems, against
the oracle, and the symmetric float64 and float-float kernels at 50k charges on sampled
targets."""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import assert_close, full_size_sample
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# The float32 path's error grows with the cancellation of the near sum: each of the
# 27 x 200k terms a charge sums carries about one float32 ulp of its own size (offsets, r^2,
# rsqrt, product), so the potential's error is about u sqrt(sum of squared terms), here
# ~20 times the potential's rms (~100, dominated by each charge's partner at 0.01).  Measured
# against the float-float path: epsilon_2(phi) 5.9e-7, 1.0e-6 and 1.65e-6 for 2e4, 6e4 and 2e5
# charges with the fast terms, 3.5e-7, 5.6e-7 and 8.7e-7 with the refined ones (at 2e5 in the
# Hilbert order of the charges: 1.33e-6 and 8.3e-7)
# (PSUM_TERMS_REFINED: float-float offsets and 1/r fused into the sums), while the field stays
# at 2.1-2.6e-7.  The float-float path holds the float64 tolerance at full size.
TOL = {"fp32c": {"phi": 1e-6, "grad": 1e-6, "adj": 1e-6}, "ff": {"phi": 1e-10, "grad": 1e-10, "adj": 1e-9}}

DIPOLE_CASES = [("fp32c", "refined"), ("ff", "fast"),
                pytest.param("fp32c", "fast", marks=pytest.mark.xfail(
                    strict=False, reason="fast float32 terms: eps2(phi) 1.33e-6 at 2e5 dipole charges, "
                                         "the per-term rounding floor; PSUM_TERMS_REFINED meets 1e-6"))]


@pytest.mark.parametrize("precision,terms", DIPOLE_CASES)
def test_dipole_system_forward_and_adjoint_on_sampled_charges(precision, terms):
    s = W.config(5)                                   # 100k tight dipoles, 200k charges
    tol = TOL[precision]
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, terms=terms)
    try:
        x, q = _dev(s.x), _dev(s.q)
        phi, g = pc(x, q)
        dEdq, dEdx = torch.empty_like(q), torch.empty_like(x)
        B.psum_energy_backward(pc.plan, x, q, phi, g, None, dEdq, dEdx)
        torch.cuda.synchronize()
    finally:
        pc.close()
    k = full_size_sample(s.x, s.d, 4096, seed=5)
    pl = O.Plan(s.d, s.p, s.M)
    ref = pl.evaluate(s.x, s.q, targets=s.x[k], parts=True)
    phi_s, g_s = phi.cpu().numpy()[k], g.cpu().numpy()[k]
    assert_close(phi_s, ref["phi"], tol["phi"])
    assert_close(g_s, ref["grad"], tol["grad"])
    # the exact adjoint at the sampled charges: psi from the check points with u = (A^+)^T w
    w = O.regular_basis(s.x / pl.R0, pl.p)[1:] @ s.q
    Q, R, piv = pl.factors
    import scipy.linalg
    u = Q @ scipy.linalg.solve_triangular(R, w[piv], trans="T", lower=False)
    psi, gpsi = O.near_sum(s.x[k], np.concatenate([pl.Yt, pl.Y]), np.concatenate([u, -u]), pl.d, pl.K)
    dq_ref = ref["phi_near"] + 0.5 * ref["phi_far"] + 0.5 * psi
    dx_ref = s.q[k, None] * (ref["grad_near"] + 0.5 * ref["grad_far"] + 0.5 * gpsi)
    dq = dEdq.cpu().numpy()[k]
    # dE/dq is defined up to a constant (the charges sum to zero): compare differences
    assert_close(dq - dq.mean(), dq_ref - dq_ref.mean(), tol["adj"])
    assert_close(dEdx.cpu().numpy()[k], dx_ref, tol["adj"])


def test_full_batch_against_single_evaluations_and_the_oracle():
    systems = W.config(4)                             # 256 systems, 1.42M charges
    pb = B.PeriodicBatch(systems, precision="fp32c")
    try:
        x = _dev(np.concatenate([s.x for s in systems]))
        q = _dev(np.concatenate([s.q for s in systems]))
        phi, g = pb(x, q, use_graph=True)
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
        offsets = list(pb.offsets)
        # the single evaluations run the kernel family the autotuner chose (the two
        # families round differently)
        pairs = "symmetric" if B.psum_batch_get_info(pb.batch)["variant"] == 2 else "one-sided"
    finally:
        pb.close()
    rng = np.random.default_rng(8)
    for b in rng.choice(len(systems), size=6, replace=False):
        s = systems[b]
        pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c", K=s.K, pairs=pairs)
        try:
            p1, g1 = pc(_dev(s.x), _dev(s.q))
        finally:
            pc.close()
        sl = slice(offsets[b], offsets[b + 1])
        assert_close(phi[sl], p1.cpu().numpy(), 1e-7, s.name)
        assert_close(g[sl], g1.cpu().numpy(), 1e-7, s.name)
    small = sorted(range(len(systems)), key=lambda b: systems[b].N)[:2]
    small.append(next(b for b in range(len(systems)) if tuple(systems[b].K) != (1, 1, 1)))
    for b in small:
        s = systems[b]
        ref = O.periodic_sum(s.x, s.q, s.d, s.p, s.M, K=s.K)
        sl = slice(offsets[b], offsets[b + 1])
        assert_close(phi[sl], ref["phi"], 1e-6, s.name)
        assert_close(g[sl], ref["grad"], 1e-6, s.name)


@pytest.mark.parametrize("precision", ["fp64", "ff"])
def test_symmetric_float64_class_kernels_at_50k_charges_on_sampled_targets(precision):
    # the symmetric float64 and float-float kernels over 98 tiles of 512 (391 of 128), every
    # image in one group, against the oracle on 1024 sampled charges (FP64 tolerance)
    s = W.uniform_gauss(N=50_000, d=(1.0, 1.5, 2.0), p=16, M=800, seed=21)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision)
    try:
        assert B.psum_pair_kernel(pc.plan, s.N)[0] == "symmetric"
        phi, g = pc(_dev(s.x), _dev(s.q))
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()
    k = full_size_sample(s.x, s.d, 1024, cluster=300, seed=21)
    ref = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, targets=s.x[k], parts=True)
    assert_close(phi[k], ref["phi"], 1e-10)
    assert_close(g[k], ref["grad"], 1e-10)


def test_symmetric_kernel_at_300k_charges_on_sampled_targets():
    # 586 tiles, 172 000 work items: 5.6 GB of tile-pair partial sums in one band, run as bands
    # of 1.5 GiB; 1024 sampled charges against the oracle
    s = W.uniform_gauss(N=300_000, d=(1.0, 1.5, 2.0), p=8, M=200, seed=22)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        assert B.psum_pair_kernel(pc.plan, s.N)[0] == "symmetric"
        phi, g = pc(_dev(s.x), _dev(s.q))
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()
    k = full_size_sample(s.x, s.d, 1024, cluster=300, seed=22)
    ref = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, targets=s.x[k], parts=True)
    # measured 4.2e-7 (phi) and 2.2e-7 (field): the FP32C bound holds here
    assert_close(phi[k], ref["phi"], 1e-6)
    assert_close(g[k], ref["grad"], 1e-6)
