"""GPU energy derivatives (torch.autograd.Function) against the oracle's exact adjoint,
finite differences and the analytic forces q grad phi."""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import MAX_FACTOR, errors
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32c": 1e-6}


def _dev(a, grad=False):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda", requires_grad=grad)


def _rel(a, b):
    """max(eps2, (max error / rms) / MAX_FACTOR): below a tolerance only if both the norm
    and every single value are within it (parity_check)."""
    e2, emax = errors(a, b)
    return max(e2, emax / MAX_FACTOR)


_REF = {}


def oracle_grads(s):
    if s.name not in _REF:
        _REF[s.name] = O.energy_and_gradients(O.Plan(s.d, s.p, s.M), s.x, s.q)
    return _REF[s.name]


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_autograd_matches_oracle_adjoint(precision):
    from paper_1310_4374_gb300.autograd import PeriodicCoulombEnergy

    s = W.config(5, small=True)
    ref = oracle_grads(s)
    mod = PeriodicCoulombEnergy(s.d, s.p, s.M, precision=precision)
    try:
        x = _dev(s.x, grad=True)
        q = _dev(s.q, grad=True)
        E = mod(x, q)
        E.backward()
        assert abs(float(E) - ref["E"]) <= TOL[precision] * abs(ref["E"]) * 10
        e_x = _rel(x.grad.cpu().numpy(), ref["dEdx"])
        # dE/dq is defined up to a constant on the neutral subspace: compare centred values
        gq = q.grad.cpu().numpy()
        e_q = _rel(gq - gq.mean(), ref["dEdq"] - ref["dEdq"].mean())
        assert e_x < TOL[precision] and e_q < TOL[precision], (e_x, e_q)
    finally:
        mod.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_two_forwards_through_one_module_share_one_backward(precision):
    # each forward keeps its own fitted coefficients: E1 + E2 over two different systems of
    # one box (the second forward refits the plan) backpropagates into both exactly
    from paper_1310_4374_gb300.autograd import PeriodicCoulombEnergy

    s1 = W.config(5, small=True)
    s2 = W.dipole_pairs(n_pairs=1200, d=s1.d, p=s1.p, M=s1.M, seed=41)
    r1, r2 = oracle_grads(s1), oracle_grads(s2)
    mod = PeriodicCoulombEnergy(s1.d, s1.p, s1.M, precision=precision)
    try:
        x1, q1 = _dev(s1.x, grad=True), _dev(s1.q, grad=True)
        x2, q2 = _dev(s2.x, grad=True), _dev(s2.q, grad=True)
        E1 = mod(x1, q1)
        E2 = mod(x2, q2)
        (E1 + E2).backward()
        for x, q, ref in ((x1, q1, r1), (x2, q2, r2)):
            e_x = _rel(x.grad.cpu().numpy(), ref["dEdx"])
            gq = q.grad.cpu().numpy()
            e_q = _rel(gq - gq.mean(), ref["dEdq"] - ref["dEdq"].mean())
            assert e_x < TOL[precision] and e_q < TOL[precision], (e_x, e_q)
    finally:
        mod.close()


def test_upstream_gradient_scales_the_result():
    from paper_1310_4374_gb300.autograd import PeriodicCoulombEnergy

    s = W.config(1)
    mod = PeriodicCoulombEnergy(s.d, s.p, s.M, precision="fp64")
    try:
        x = _dev(s.x, grad=True)
        q = _dev(s.q, grad=True)
        (3.0 * mod(x, q)).backward()
        g3 = x.grad.clone()
        x.grad = None
        q.grad = None
        mod(x, q).backward()
        assert torch.allclose(g3, 3.0 * x.grad, rtol=1e-14, atol=0)
    finally:
        mod.close()


def test_fp64_backward_is_the_derivative_of_the_gpu_energy():
    # central differences of the GPU's own FP64 energy
    s = W.uniform_gauss(N=400, d=(1.0, 1.0, 2.0), p=10, M=300, seed=31)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp64")
    try:
        def energy(xx, qq):
            x = _dev(xx)
            q = _dev(qq)
            phi, g = pc(x, q)
            E = torch.empty(1, dtype=torch.float64, device="cuda")
            B.psum_energy(pc.plan, q, phi, E)
            return float(E), (x, q, phi, g)

        E0, (x, q, phi, g) = energy(s.x, s.q)
        dEdq = torch.empty_like(q)
        dEdx = torch.empty_like(x)
        B.psum_energy_backward(pc.plan, x, q, phi, g, None, dEdq, dEdx)
        dEdx = dEdx.cpu().numpy()
        dEdq = dEdq.cpu().numpy()
        h = 1e-6
        for j, k in ((0, 0), (17, 2), (250, 1)):
            xp, xm = s.x.copy(), s.x.copy()
            xp[j, k] += h
            xm[j, k] -= h
            fd = (energy(xp, s.q)[0] - energy(xm, s.q)[0]) / (2 * h)
            assert fd == pytest.approx(dEdx[j, k], rel=1e-6, abs=1e-6)
        for a, b in ((3, 8), (100, 301)):
            qp, qm = s.q.copy(), s.q.copy()
            qp[a] += h
            qp[b] -= h
            qm[a] -= h
            qm[b] += h
            fd = (energy(s.x, qp)[0] - energy(s.x, qm)[0]) / (2 * h)
            assert fd == pytest.approx(dEdq[a] - dEdq[b], rel=1e-6, abs=1e-6)
    finally:
        pc.close()


def test_forces_agree_with_the_analytic_field():
    # the exact adjoint differs from q grad phi only by the method's truncation error
    s = W.config(5, small=True)
    ref = oracle_grads(s)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        x = _dev(s.x)
        q = _dev(s.q)
        phi, g = pc(x, q)
        dEdx = torch.empty_like(x)
        B.psum_energy_backward(pc.plan, x, q, phi, g, None, None, dEdx)
        force_field = s.q[:, None] * ref["grad"]
        assert _rel(dEdx.cpu().numpy(), force_field) < 1e-5
    finally:
        pc.close()


@pytest.mark.parametrize("precision", ["fp32c", "ff", "fp64"])
@pytest.mark.parametrize("checks", ["layers", "points"])
def test_backward_check_sources_in_both_forms_with_a_wider_block(precision, checks):
    # psi from the check points as the two image layers (float32 packing: each point twice, with
    # +u_l and the upper layer's images, -u_l and the lower's) or as the 2M points; a flat box
    # with K = (2, 1, 1), whose classes have layers of 9 and 15 images (padded lists)
    s = W.uniform_gauss(N=1500, d=(1.0, 2.0, 2.0), p=10, M=300, seed=33)
    K = (2, 1, 1)
    ref = O.energy_and_gradients(O.Plan(s.d, s.p, s.M, K=K), s.x, s.q)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, K=K, checks=checks)
    try:
        assert B.psum_check_form(pc.plan) == checks
        x, q = _dev(s.x), _dev(s.q)
        phi, g = pc(x, q)
        dEdq, dEdx = torch.empty_like(q), torch.empty_like(x)
        B.psum_energy_backward(pc.plan, x, q, phi, g, None, dEdq, dEdx)
        torch.cuda.synchronize()
        assert B.psum_sync(pc.plan) == B.PSUM_OK
        tol = TOL.get(precision, 1e-10)
        if precision == "ff" and checks == "points":
            # the point form subtracts psi's two 45-image sums at y~ and y, which agree to about
            # three digits on this flat box: float-float's ~1e-13 per term leaves ~2e-10 in the
            # field (measured 2.2e-10; the layer form, which never forms the common part, meets
            # 1e-10, and the automatic choice takes it here)
            tol = 1e-9
        gq = dEdq.cpu().numpy()
        e_q = _rel(gq - gq.mean(), ref["dEdq"] - ref["dEdq"].mean())
        e_x = _rel(dEdx.cpu().numpy(), ref["dEdx"])
        assert e_q < tol and e_x < tol, (e_q, e_x)
    finally:
        pc.close()
