"""psum_eval_graph: the single-system evaluation captured into a CUDA graph and replayed."""
import numpy as np
import pytest

from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision,pairs", [("fp32c", "one-sided"), ("fp32c", "symmetric"), ("fp64", "one-sided"),
                                            ("fp64", "symmetric"), ("ff", "one-sided"), ("ff", "symmetric")])
def test_graph_replay_equals_psum_eval_and_follows_new_inputs(precision, pairs):
    s = W.config(1, small=True)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, pairs=pairs)
    try:
        x, q = _dev(s.x), _dev(s.q)
        ref_phi, ref_g = pc(x, q)
        phi, g = torch.empty_like(ref_phi), torch.empty_like(ref_g)
        for _ in range(3):                               # capture, then replays
            B.psum_eval_graph(pc.plan, x, q, phi, g, check=True)
            assert torch.equal(phi, ref_phi) and torch.equal(g, ref_g)
        q.mul_(-1.0)                                     # new charges in the same buffer
        B.psum_eval_graph(pc.plan, x, q, phi, g, check=True)
        assert torch.equal(phi, -ref_phi) and torch.equal(g, -ref_g)
        q.mul_(-1.0)
        q[0] += 0.5                                      # not neutral: reported by psum_sync
        B.psum_eval_graph(pc.plan, x, q, phi, g)
        assert B.psum_sync(pc.plan) == B.PSUM_ERR_NONNEUTRAL
        assert torch.isnan(phi).all()
    finally:
        pc.close()


def test_graph_recaptures_for_other_buffers_and_sizes():
    pc = None
    try:
        a = W.uniform_pm1(N=300, p=8, M=200, seed=1)
        b = W.uniform_pm1(N=700, p=8, M=200, seed=2)
        pc = B.PeriodicCoulomb(a.d, 8, 200, precision="fp32c")
        for s in (a, b, a):
            x, q = _dev(s.x), _dev(s.q)
            ref_phi, ref_g = pc(x, q)
            phi, g = torch.empty_like(ref_phi), torch.empty_like(ref_g)
            B.psum_eval_graph(pc.plan, x, q, phi, g, check=True)
            assert torch.equal(phi, ref_phi) and torch.equal(g, ref_g)
    finally:
        if pc is not None:
            pc.close()
