"""The right-hand side of the fit in its two-layer form: the partner
y~_l = y_l - s d_k e_k sees the near block shifted by one period along k, so
phi_near(y~_l) - phi_near(y_l) is the image layer i_k = s(K_k + 1) minus the layer
i_k = -s K_k, summed at y_l alone (algorithm "get", step 3; Eq. 3).  The GPU path with
each form against the FP64 oracle, and the two forms against each other.

Tolerances (relative L2 error over all charges): FP32C 1e-6, FF and FP64 1e-10.
"""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import assert_close
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32c": 1e-6, "ff": 1e-10, "fp64": 1e-10}
# the two forms round differently; their coefficients agree to the float32 pair sums'
# accuracy amplified by the pseudo-inverse (FP32C), or to float64 accuracy (FF, FP64)
C_TOL = {"fp32c": 1e-4, "ff": 1e-9, "fp64": 1e-9}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# (name, system, plan keywords): class sizes from a handful of points (one partly filled
# group per class, empty groups in the last tile) to several groups per class; an
# anisotropic block whose layers differ in size (zero-weight padding images); the Gauss grid;
# the RBF basis; no mean condition
CASES = [
    ("uniform_pm1_402_M200", lambda: W.uniform_pm1(N=402, p=8, M=200, seed=4), {}),
    ("gauss_3001_p16_M800", lambda: W.uniform_gauss(N=3001, d=(1.0, 1.5, 2.0), p=16, M=800, seed=5), {}),
    ("aniso_K121", lambda: W.uniform_gauss(N=1500, d=(1.0, 1.0, 2.0), p=10, M=300, seed=6), {"K": (1, 2, 1)}),
    ("gauss_grid_p12", lambda: W.uniform_gauss(N=2000, d=(1.0, 1.5, 2.0), p=12, M=325, seed=7),
     {"points": "gauss"}),
    ("small_M40", lambda: W.uniform_gauss(N=130, d=(1.0, 1.0, 1.0), p=4, M=40, seed=8), {}),
    ("mean_none", lambda: W.uniform_gauss(N=900, d=(2.0, 1.0, 1.5), p=8, M=200, seed=9), {"mean": "none"}),
    ("rbf_64", lambda: W.uniform_gauss(N=700, d=(1.0, 1.0, 1.0), p=8, M=200, seed=10),
     {"basis": "rbf", "n_rbf": 64}),
]


def _oracle(s, kw):
    pl = O.Plan(s.d, s.p, s.M, K=kw.get("K", (1, 1, 1)),
                checkpoints="gauss" if kw.get("points") == "gauss" else None,
                basis=kw.get("basis", "spherical"), n_rbf=kw.get("n_rbf", 256))
    return pl.evaluate(s.x, s.q, mean=kw.get("mean", "zero"))


def _gpu(s, precision, checks, kw):
    M = 0 if kw.get("points") == "gauss" else s.M
    pc = B.PeriodicCoulomb(s.d, s.p, M, precision=precision, checks=checks, **kw)
    try:
        form = B.psum_check_form(pc.plan)
        phi, g = pc(_dev(s.x), _dev(s.q))
        return phi.cpu().numpy(), g.cpu().numpy(), np.asarray(pc.coefficients()), form
    finally:
        pc.close()


@pytest.mark.parametrize("precision", ["fp32c", "ff", "fp64"])
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_layers_against_oracle_and_points(name, make, kw, precision):
    s = make()
    ref = _oracle(s, kw)
    phi_l, g_l, C_l, form_l = _gpu(s, precision, "layers", kw)
    phi_p, g_p, C_p, form_p = _gpu(s, precision, "points", kw)
    assert (form_l, form_p) == ("layers", "points")
    tol = TOL[precision]
    for phi, g, what in ((phi_l, g_l, "layers"), (phi_p, g_p, "points")):
        assert_close(phi, ref["phi"], tol, f"{what} phi")
        assert_close(g, ref["grad"], tol, f"{what} grad")
    if kw.get("basis") == "rbf":
        # the equivalent sources of Eq. 5 are an ill-conditioned basis: the fit fixes the field
        # to the method's accuracy, not each coefficient; compare the two forms' fields instead
        assert_close(phi_l, phi_p, 2 * tol, "phi layers vs points")
        assert_close(g_l, g_p, 2 * tol, "grad layers vs points")
        return
    e_C = np.linalg.norm(C_l - C_p) / np.linalg.norm(C_p)
    assert e_C < C_TOL[precision], f"coefficients of the two forms differ by {e_C:.3e}"


def test_automatic_check_form():
    # the layers where they apply and need no more (tile, image) units than the 2M points, and
    # (float32) where the per-class offsets fit the kernel's shared memory
    s = W.uniform_gauss(N=300, d=(1.0, 1.5, 2.0), p=8, M=200, seed=1)
    expect = [({"precision": "fp32c", "M": 200}, "layers"),     # 1 tile x 18 against 1 x 27
              ({"precision": "ff", "M": 400}, "layers"),
              ({"precision": "fp64", "M": 200}, "layers"),      # tiles of 128: 2 x 18 against 4 x 27
              ({"precision": "fp32c", "M": 200, "K": (3, 3, 1)}, "points"),   # 98 layer images
              ({"precision": "fp64", "M": 200, "K": (3, 3, 1)}, "layers"),
              ({"precision": "fp32c", "M": 400, "checks": "points"}, "points"),
              ({"precision": "fp64", "M": 200, "checks": "points"}, "points"),
              ({"precision": "fp32c", "M": 800, "lam": 1.5}, "points"), ({"precision": "fp64", "M": 200, "lam": 1.5}, "points")]
    for kw, form in expect:
        kw = dict(kw)
        M = kw.pop("M")
        pc = B.PeriodicCoulomb(s.d, s.p, M, **kw)
        try:
            assert B.psum_check_form(pc.plan) == form, (M, kw)
        finally:
            pc.close()


def test_layers_deterministic_and_graph_replay():
    # fixed work items and reduction order: repeated evaluations and a graph replay of the
    # layered plan give identical bits
    s = W.uniform_gauss(N=2500, d=(1.0, 1.5, 2.0), p=12, M=400, seed=11)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        x, q = _dev(s.x), _dev(s.q)
        a = pc(x, q)[0].cpu().numpy()
        b = pc(x, q)[0].cpu().numpy()
        phi = torch.empty(len(s.q), dtype=torch.float64, device="cuda")
        g = torch.empty((len(s.q), 3), dtype=torch.float64, device="cuda")
        B.psum_eval_graph(pc.plan, x, q, phi, g)
        B.psum_eval_graph(pc.plan, x, q, phi, g)
        c = phi.cpu().numpy()
        assert np.array_equal(a, b) and np.array_equal(a, c)
    finally:
        pc.close()


@pytest.mark.parametrize("precision", ["fp32c", "ff", "fp64"])
def test_batch_with_mixed_check_forms(precision):
    # systems whose plans take the two-layer form and systems whose plans take the point
    # form in one batch: each against the oracle and against its single evaluation
    systems = W.config(4, small=True)
    forms = ["points" if b % 3 == 1 else "layers" for b in range(len(systems))]
    # a widened block K = (2, 1, 1) among the layered systems (layers of 15 and 9 images)
    assert any(tuple(s.K) != (1, 1, 1) and f == "layers" for s, f in zip(systems, forms))
    pb = B.PeriodicBatch(systems, precision=precision, checks=forms)
    try:
        assert [B.psum_check_form(p) for p in pb.plans] == forms
        x = torch.as_tensor(np.concatenate([s.x for s in systems]), dtype=torch.float64, device="cuda")
        q = torch.as_tensor(np.concatenate([s.q for s in systems]), dtype=torch.float64, device="cuda")
        phi, g = pb(x, q)
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
        for b, (s, form) in enumerate(zip(systems, forms)):
            sl = slice(pb.offsets[b], pb.offsets[b + 1])
            ref = O.periodic_sum(s.x, s.q, s.d, s.p, s.M, K=s.K)
            assert_close(phi[sl], ref["phi"], TOL[precision], (b, form, "phi"))
            assert_close(g[sl], ref["grad"], TOL[precision], (b, form, "grad"))
            pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, K=s.K, checks=form)
            try:
                p1, g1 = pc(_dev(s.x), _dev(s.q))
            finally:
                pc.close()
            single_tol = 1e-7 if precision == "fp32c" else 1e-12
            assert_close(phi[sl], p1.cpu().numpy(), single_tol, (b, form))
            assert_close(g[sl], g1.cpu().numpy(), single_tol, (b, form))
    finally:
        pb.close()
