"""Evaluation at separate points y of the box (psum_eval_points) against the oracle's
"get" with targets Y0 (Sec. 2.3.2), and periodicity of the GPU result across the faces."""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import assert_close
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "ff": 1e-10, "fp32c": 1e-6}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _points(T, d, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.5, 0.5, (T, 3)) * np.asarray(d)


def _at(s, y, precision, **kw):
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, **kw)
    try:
        phi, g = pc.at(_dev(s.x), _dev(s.q), _dev(y))
        return phi.cpu().numpy(), g.cpu().numpy()
    finally:
        pc.close()


@pytest.mark.parametrize("precision", ["fp64", "ff", "fp32c"])
@pytest.mark.parametrize("name,make,T", [("cfg1", lambda: W.config(1), 700),
                                         ("cfg3_small", lambda: W.config(3, small=True), 1500),
                                         ("ragged", lambda: W.uniform_pm1(N=130, p=8, M=200, seed=4), 129)])
def test_points_match_oracle(name, make, T, precision):
    s = make()
    y = _points(T, s.d, 17)
    phi, g = _at(s, y, precision)
    ref = O.Plan(s.d, s.p, s.M).evaluate(s.x, s.q, targets=y, parts=True)
    assert_close(phi, ref["phi"], TOL[precision])
    # Float-float offsets keep about 2^-48 of the group-relative coordinates (groups of 128
    # points span ~0.4 of the box at 3000 charges), not of the offset: random points that
    # fall very close to a charge see field terms with a relative error near 1e-12, which
    # leaves the field's epsilon_2 at about 1.1e-10 (measured) where float64 keeps 1e-12.
    gtol = 3e-10 if precision == "ff" else TOL[precision]
    assert_close(g, ref["grad"], gtol)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_points_at_the_charges_equal_psum_eval(precision):
    s = W.config(3, small=True)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision)
    try:
        x, q = _dev(s.x), _dev(s.q)
        phi, g = pc(x, q)
        phi2, g2 = pc.at(x, q, x.clone())          # K(0) = 0 drops every self pair
    finally:
        pc.close()
    tol = 1e-13 if precision == "fp64" else 1e-7
    assert_close(phi2.cpu().numpy(), phi.cpu().numpy(), tol)
    assert_close(g2.cpu().numpy(), g.cpu().numpy(), tol)


def test_points_with_trimming_rbf_and_gauss_grid():
    s = W.uniform_pm1(N=800, p=15, M=496, seed=12)
    y = _points(300, s.d, 5)
    for kw, okw in ((dict(lam=1.5), dict(lam=1.5)),
                    (dict(points="gauss", basis="rbf"), dict(checkpoints="gauss", basis="rbf"))):
        M = 0 if kw.get("points") == "gauss" else s.M
        pc = B.PeriodicCoulomb(s.d, s.p, M, precision="fp64", **kw)
        try:
            phi, g = pc.at(_dev(s.x), _dev(s.q), _dev(y))
        finally:
            pc.close()
        ref = O.Plan(s.d, s.p, M, **okw).evaluate(s.x, s.q, targets=y, parts=True)
        assert_close(phi.cpu().numpy(), ref["phi"], 1e-10, kw)
        assert_close(g.cpu().numpy(), ref["grad"], 1e-10, kw)


@pytest.mark.parametrize("d", [(1.0, 1.0, 1.0), (1.0, 1.0, 2.0)])
def test_gpu_potential_is_periodic_across_faces(d):
    # Eq. 7: the method makes phi periodic; points on the face x_k = -d_k/2 and just inside
    # the opposite face (the largest float64 below d_k/2) see the same potential and field
    rng = np.random.default_rng(9)
    N = 400
    x = rng.uniform(-0.5, 0.5, (N, 3)) * np.asarray(d)
    q = rng.normal(size=N)
    q -= q.mean()
    s = W.System(x, q, d, 20, 900, K=(1, 1, 1) if d[2] == 1.0 else (2, 2, 1))
    lo, hi = [], []
    for k in range(3):
        y = rng.uniform(-0.45, 0.45, (8, 3)) * np.asarray(d)
        y[:, k] = -d[k] / 2
        y2 = y.copy()
        y2[:, k] = np.nextafter(d[k] / 2, 0.0)
        lo.append(y)
        hi.append(y2)
    Y = np.concatenate(lo + hi)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp64", K=s.K)
    try:
        phi, g = pc.at(_dev(s.x), _dev(s.q), _dev(Y))
    finally:
        pc.close()
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    n = len(Y) // 2
    scale = np.sqrt(np.mean(phi ** 2))
    assert np.max(np.abs(phi[:n] - phi[n:])) < 1e-6 * scale
    assert np.max(np.abs(g[:n] - g[n:])) < 1e-5 * np.sqrt(np.mean(g ** 2))


def test_points_outside_the_box_are_reported():
    s = W.uniform_pm1(N=200, p=6, M=100, seed=2)
    y = _points(10, s.d, 3)
    y[4, 1] = 0.5                                  # the half-open box excludes +d/2
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        with pytest.raises(B.PsumError) as e:
            pc.at(_dev(s.x), _dev(s.q), _dev(y))
        assert e.value.status == B.PSUM_ERR_OUT_OF_BOX
    finally:
        pc.close()
