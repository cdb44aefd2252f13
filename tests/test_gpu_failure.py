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


@pytest.mark.parametrize("call", ["eval", "graph", "backward"])
def test_forced_allocation_failure_is_reported_and_the_plan_recovers(call):
    # the test hook makes the next scratch growth fail as an out-of-memory cudaMalloc would:
    # the call returns PSUM_ERR_NOMEM and queues nothing; the plan then grows its scratch again
    # and evaluates exactly as a fresh plan
    s = W.config(1)
    small = W.uniform_pm1(N=300, p=8, M=200, seed=3)
    ref = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c")
    try:
        x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
        q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
        phi0, g0 = ref(x, q)
        pc(torch.as_tensor(small.x, device="cuda"), torch.as_tensor(small.q, device="cuda"))   # a smaller scratch
        B.psum_debug_fail_allocs(pc.plan, 1)
        phi = torch.full_like(q, 7.0)
        grad = torch.full_like(x, 7.0)
        with pytest.raises(B.PsumError) as e:
            if call == "eval":
                B.psum_eval(pc.plan, x, q, phi, grad)
            elif call == "graph":
                B.psum_eval_graph(pc.plan, x, q, phi, grad)
            else:
                B.psum_energy_backward(pc.plan, x, q, phi0, g0, None, phi, grad)
        assert e.value.status == B.PSUM_ERR_NOMEM
        torch.cuda.synchronize()
        assert bool((phi == 7.0).all()) and bool((grad == 7.0).all())     # nothing was queued
        assert B.psum_sync(pc.plan) == B.PSUM_OK
        phi1, g1 = pc(x, q)
        assert torch.equal(phi1, phi0) and torch.equal(g1, g0)
    finally:
        pc.close()
        ref.close()


_DEBUG_SCRIPT = r"""
import json, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W
out = {"checks": B.psum_debug_checks(), "cases": []}
s = W.config(1)
x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
for precision, pairs in (("fp32c", "one-sided"), ("fp32c", "symmetric"), ("fp64", "symmetric")):
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=precision, pairs=pairs)
    phi0, g0 = pc(x, q)
    ok0 = B.psum_sync(pc.plan)
    B.psum_debug_bounds_limit(pc.plan, 256)     # below one partial slot: every write is refused
    phi = torch.empty_like(q)
    g = torch.empty_like(x)
    B.psum_eval(pc.plan, x, q, phi, g)
    st = B.psum_sync(pc.plan)
    nan = bool(torch.isnan(phi).all() and torch.isnan(g).all())
    B.psum_debug_bounds_limit(pc.plan, 0)
    phi1, g1 = pc(x, q)
    out["cases"].append([precision, pairs, ok0, st, nan, bool(torch.equal(phi1, phi0) and torch.equal(g1, g0))])
    pc.close()
print(json.dumps(out))
"""


def test_debug_build_bounds_checks_report_instead_of_faulting():
    # The debug library range-checks the pair kernels' partial sums.  Its test hook makes the
    # checks see a buffer smaller than one slot, so every write is refused inside the real
    # buffer: the evaluation reports PSUM_ERR_INTERNAL with NaN outputs, and the next one on the
    # same context is exact.  Run in a child process, which loads the debug library.
    import json
    import os
    import subprocess
    import sys

    from paper_1310_4374_gb300 import build as _b
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = _b.build(debug=True)
    env = dict(os.environ, PSUM_LIB=lib)
    r = subprocess.run([sys.executable, "-c", _DEBUG_SCRIPT, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checks"] is True
    for precision, pairs, ok0, st, nan, same in out["cases"]:
        assert ok0 == B.PSUM_OK, (precision, pairs)
        assert st == B.PSUM_ERR_INTERNAL and nan and same, (precision, pairs, st, nan, same)
