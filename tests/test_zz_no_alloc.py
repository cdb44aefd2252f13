"""psum_eval_noalloc: the evaluation entry point for callers that cannot allocate device
memory when they evaluate (inside a stream capture, in a real-time loop that cannot take
the synchronisation of cudaMalloc, or under a runtime that owns all device memory).  It
takes its scratch from a fixed device array inside the library, so its results must match
psum_eval's within the parity tolerances, call after call on the shared array.

This file is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import pytest

from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W
from parity_check import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32c": 1e-6}


def _np(t):
    return t.detach().cpu().numpy()


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
            assert_close(_np(phi), _np(ref_phi), TOL[precision], (s.N, "phi"))
            assert_close(_np(g), _np(ref_g), TOL[precision], (s.N, "grad"))
    finally:
        pc.close()


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_noalloc_holds_its_stated_limit(precision):
    # the header promises N = 32768 charges for p = 16 and M = 800 in either precision: the
    # scratch of that evaluation fits the fixed array (else PSUM_ERR_ARG) and the results
    # match psum_eval
    s = W.uniform_gauss(N=32768, d=(1.0, 1.5, 2.0), p=16, M=800, seed=11)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision)
    try:
        x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
        q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
        ref_phi, ref_g = pc(x, q)
        phi = torch.full_like(ref_phi, float("nan"))
        g = torch.full_like(ref_g, float("nan"))
        B.psum_eval_noalloc(pc.plan, x, q, phi, g, check=True)
        assert_close(_np(phi), _np(ref_phi), TOL[precision], "phi")
        assert_close(_np(g), _np(ref_g), TOL[precision], "grad")
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
