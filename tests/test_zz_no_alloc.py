"""psum_eval_noalloc: the evaluation entry point for callers that cannot allocate device
memory when they evaluate (inside a stream capture, in a real-time loop that cannot take
the synchronisation of cudaMalloc, or under a runtime that owns all device memory).  It
takes its scratch from a fixed device array inside the library, so its results must match
psum_eval's within the parity tolerances, call after call on the shared array.

This file is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32c": 1e-6}


def _rel(a, b):
    a = a.detach().cpu().numpy().reshape(-1)
    b = b.detach().cpu().numpy().reshape(-1)
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_noalloc_matches_psum_eval_on_two_calls(precision):
    systems = [W.uniform_gauss(N=3001, d=(1.0, 1.5, 2.0), p=16, M=800, seed=2),
               W.uniform_gauss(N=5000, d=(1.0, 1.5, 2.0), p=16, M=800, seed=7)]
    pc = B.PeriodicCoulomb(systems[0].d, 16, 800, precision=precision)
    try:
        for s in systems:                     # two calls in a row on the shared array
            x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
            q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
            ref_phi, ref_g = pc(x, q)
            phi = torch.full_like(ref_phi, float("nan"))
            g = torch.full_like(ref_g, float("nan"))
            B.psum_eval_noalloc(pc.plan, x, q, phi, g, check=True)
            assert torch.isfinite(phi).all() and torch.isfinite(g).all()
            assert _rel(phi, ref_phi) < TOL[precision]
            assert _rel(g, ref_g) < TOL[precision]
    finally:
        pc.close()


def test_noalloc_rejects_inputs_beyond_its_scratch():
    s = W.uniform_gauss(N=200_000, d=(1.0, 1.0, 1.0), p=8, M=200, seed=3)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
        q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
        phi = torch.empty(s.N, dtype=torch.float64, device="cuda")
        with pytest.raises(B.PsumError) as e:
            B.psum_eval_noalloc(pc.plan, x, q, phi)
        assert e.value.status == B.PSUM_ERR_ARG
    finally:
        pc.close()
