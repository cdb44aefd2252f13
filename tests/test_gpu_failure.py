"""Failure path of the bounded device-side waits: a chunk-copy wait that runs out (the test
hook arms the barrier for bytes that never come) is reported as PSUM_ERR_TIMEOUT with NaN
outputs, and the next evaluation on the same context is exact again."""
import numpy as np
import pytest

from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,pairs", [("fp32c", "one-sided"), ("fp32c", "symmetric"), ("ff", "auto")])
def test_copy_wait_that_runs_out_is_reported_and_the_context_survives(precision, pairs):
    s = W.config(1, small=True)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, pairs=pairs)
    try:
        x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
        q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
        phi0, g0 = pc(x, q)
        B.psum_debug_inject_timeout(pc.plan, True)
        phi = torch.empty_like(q)
        grad = torch.empty_like(x)
        B.psum_eval(pc.plan, x, q, phi, grad)
        assert B.psum_sync(pc.plan) == B.PSUM_ERR_TIMEOUT
        assert torch.isnan(phi).all() and torch.isnan(grad).all()
        B.psum_debug_inject_timeout(pc.plan, False)
        phi1, g1 = pc(x, q)
        assert torch.equal(phi1, phi0) and torch.equal(g1, g0)
    finally:
        pc.close()
