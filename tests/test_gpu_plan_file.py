"""Plan files (psum_plan_save / psum_plan_load): the set stage's factorisation kept on disk
(Sec. 2.1 recommends storing the decomposition) gives a plan that evaluates exactly as the
original, for every precision, point scheme, basis and near set; a file whose options no
longer give the stored check points is refused."""
import time

import numpy as np
import pytest

from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("fp32c", {}), ("fp32c", {"terms": "refined"}), ("fp64", {"points": "gauss"}),
         ("ff", {"lam": 1.5}), ("fp64", {"basis": "rbf"})]


def _eval(plan, s):
    x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
    q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
    phi = torch.empty(s.N, dtype=torch.float64, device="cuda")
    g = torch.empty((s.N, 3), dtype=torch.float64, device="cuda")
    B.psum_eval(plan, x, q, phi, g, check=True)
    return phi.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("precision,kw", CASES, ids=[f"{c[0]}-{'-'.join(c[1]) or 'default'}" for c in CASES])
def test_loaded_plan_evaluates_exactly_as_the_saved_one(tmp_path, precision, kw):
    s = W.config(3, small=True)
    M = 0 if kw.get("points") == "gauss" else s.M
    t0 = time.perf_counter()
    pc = B.PeriodicCoulomb(s.d, s.p, M, precision=precision, **kw)
    t_create = time.perf_counter() - t0
    path = tmp_path / "plan.psum"
    loaded = None
    try:
        B.psum_plan_save(pc.plan, path)
        t0 = time.perf_counter()
        loaded = B.psum_plan_load(path)
        t_load = time.perf_counter() - t0
        assert B.psum_plan_info(loaded) == pc.info
        a = _eval(pc.plan, s)
        b = _eval(loaded, s)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        P = pc.info["P"]
        assert np.array_equal(B.psum_get_coeffs(pc.plan, P), B.psum_get_coeffs(loaded, P))
        print(f"plan create {t_create * 1e3:.1f} ms, load {t_load * 1e3:.1f} ms")
    finally:
        if loaded is not None:
            B.psum_destroy(loaded)
        pc.close()


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for c in data:
        h ^= c
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_file_whose_options_give_other_check_points_is_refused(tmp_path):
    s = W.config(1)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp64")
    path = tmp_path / "plan.psum"
    try:
        B.psum_plan_save(pc.plan, path)
    finally:
        pc.close()
    raw = bytearray(path.read_bytes())
    # psum_opts starts after the magic word and its size; its first field is d[0]: a longer box
    # gives other check points, so the stored factorisation belongs to another matrix
    off = 8 + 4
    d0 = np.frombuffer(bytes(raw[off:off + 8]), dtype="<f8")[0]
    raw[off:off + 8] = np.array([d0 * 1.25], dtype="<f8").tobytes()
    raw[-8:] = _fnv1a(bytes(raw[:-8])).to_bytes(8, "little")
    path.write_bytes(bytes(raw))
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_load(path)
    assert e.value.status == B.PSUM_ERR_IO
