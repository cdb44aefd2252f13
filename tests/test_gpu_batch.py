"""Batched evaluation of many independent systems (one persistent pair-sum launch, CUDA
graph replay, autotuned kernel variant) against the oracle and the single-system path."""
import numpy as np
import pytest

from oracle import psum_oracle as O
from parity_check import assert_close
from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32c": 1e-6}


def _cat(systems):
    x = np.concatenate([s.x for s in systems])
    q = np.concatenate([s.q for s in systems])
    return (torch.as_tensor(x, dtype=torch.float64, device="cuda"),
            torch.as_tensor(q, dtype=torch.float64, device="cuda"))


_REF = {}


def _oracle(s):
    if s.name not in _REF:
        _REF[s.name] = O.periodic_sum(s.x, s.q, s.d, s.p, s.M, K=s.K, parts=True)
    return _REF[s.name]


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle_per_system(precision, use_graph):
    systems = W.config(4, small=True)
    pb = B.PeriodicBatch(systems, precision=precision)
    try:
        x, q = _cat(systems)
        phi, g = pb(x, q, use_graph=use_graph)
        phi = phi.cpu().numpy()
        g = g.cpu().numpy()
        for b, s in enumerate(systems):
            sl = slice(pb.offsets[b], pb.offsets[b + 1])
            ref = _oracle(s)
            assert_close(phi[sl], ref["phi"], TOL[precision], (b, s.name, "phi"))
            assert_close(g[sl], ref["grad"], TOL[precision], (b, s.name, "grad"))
            C = B.psum_batch_get_coeffs(pb.batch, b, pb.P[b])
            assert np.max(np.abs(C - ref["C"])) < (1e-9 if precision == "fp64" else 1e-4) * np.abs(ref["C"]).max()
        info = B.psum_batch_get_info(pb.batch)
        assert info["B"] == len(systems) and info["variant"] >= 0 and info["ctas"] >= 1
    finally:
        pb.close()


@pytest.mark.parametrize("pairs", ["one-sided", "symmetric"])
def test_batch_agrees_with_single_evaluations(pairs):
    # the plans' pair_kernel option steers the autotuner: symmetric plans force the
    # symmetric kernel, one-sided plans exclude it
    systems = W.config(4, small=True)
    pb = B.PeriodicBatch(systems, precision="fp32c", pairs=pairs)
    try:
        x, q = _cat(systems)
        phi, g = pb(x, q)
        v = B.psum_batch_get_info(pb.batch)["variant"]
        assert (v == 2) if pairs == "symmetric" else (v in (0, 1))
        for b, s in enumerate(systems):
            pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c", K=s.K, pairs=pairs)
            try:
                p1, g1 = pc(torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.q, device="cuda"))
            finally:
                pc.close()
            sl = slice(pb.offsets[b], pb.offsets[b + 1])
            assert_close(phi[sl].cpu().numpy(), p1.cpu().numpy(), 1e-7)
            assert_close(g[sl].cpu().numpy(), g1.cpu().numpy(), 1e-7)
    finally:
        pb.close()


def test_graph_replay_follows_new_inputs_in_the_same_buffers():
    systems = W.config(4, small=True)
    pb = B.PeriodicBatch(systems, precision="fp32c")
    try:
        x, q = _cat(systems)
        phi = torch.empty_like(q)
        g = torch.empty_like(x)
        pb(x, q, phi, g, use_graph=True)
        first = phi.clone()
        pb(x, q, phi, g, use_graph=True)                 # replay
        assert torch.equal(first, phi)
        q.mul_(-2.0)                                     # new charges, same buffer
        pb(x, q, phi, g, use_graph=True)
        assert torch.allclose(phi, -2.0 * first, rtol=1e-6, atol=1e-9 * float(first.abs().max()))
        plain_phi, _ = pb(x, q, use_graph=False)
        assert torch.equal(plain_phi, phi)
    finally:
        pb.close()


def test_batch_reports_status_per_system():
    systems = W.config(4, small=True)
    pb = B.PeriodicBatch(systems, precision="fp32c")
    try:
        x, q = _cat(systems)
        q[pb.offsets[2]] += 0.25                         # system 2 no longer neutral
        phi = torch.empty_like(q)
        B.psum_batch_eval(pb.batch, x, q, phi, None)
        first, st = B.psum_batch_sync(pb.batch, pb.B)
        assert first == B.PSUM_ERR_NONNEUTRAL
        assert st[2] == B.PSUM_ERR_NONNEUTRAL and all(v == 0 for k, v in enumerate(st) if k != 2)
        sl = slice(pb.offsets[2], pb.offsets[3])
        assert torch.isnan(phi[sl]).all() and torch.isfinite(phi[:pb.offsets[2]]).all()
    finally:
        pb.close()


def _many(B, seed):
    """B small neutral +-1 systems (p = 8, M = 200), boxes (1, U[1,2], U[1,2]) with the batch
    workload's near-block rule."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        N = 2 * int(rng.integers(30, 400))
        d = (1.0, float(rng.uniform(1.0, 2.0)), float(rng.uniform(1.0, 2.0)))
        x = rng.uniform(-0.5, 0.5, size=(N, 3)) * np.asarray(d)
        q = np.concatenate([np.ones(N // 2), -np.ones(N // 2)])
        rng.shuffle(q)
        out.append(W.System(x, q, d, 8, 200, name=f"many{seed}_{b}_N{N}", K=W.batch_near_block(d)))
    return out


@pytest.mark.parametrize("precision,nsys", [("fp32c", 1024), ("ff", 300)])
def test_batches_beyond_256_systems(precision, nsys):
    # more than 256 systems sort by the Hilbert key, then stably by the system: every system's
    # result equals its own evaluation on the same plan (to the kernels' rounding) and, on a
    # sample of systems, the oracle
    systems = _many(nsys, seed=nsys)
    pb = B.PeriodicBatch(systems, precision=precision)
    try:
        x, q = _cat(systems)
        phi, g = pb(x, q, use_graph=True)
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
        tol = TOL["fp64"] if precision == "ff" else TOL["fp32c"]
        for b, s in enumerate(systems):
            p1 = torch.empty(s.N, dtype=torch.float64, device="cuda")
            g1 = torch.empty((s.N, 3), dtype=torch.float64, device="cuda")
            B.psum_eval(pb.plans[b], torch.as_tensor(s.x, device="cuda"), torch.as_tensor(s.q, device="cuda"), p1, g1,
                        check=True)
            sl = slice(pb.offsets[b], pb.offsets[b + 1])
            assert_close(phi[sl], p1.cpu().numpy(), tol, (b, s.name, "phi"))
            assert_close(g[sl], g1.cpu().numpy(), tol, (b, s.name, "grad"))
        rng = np.random.default_rng(nsys + 1)
        for b in list(rng.choice(nsys, size=6, replace=False)) + [0, nsys - 1]:
            s = systems[b]
            ref = _oracle(s)
            sl = slice(pb.offsets[b], pb.offsets[b + 1])
            assert_close(phi[sl], ref["phi"], tol, (b, s.name, "phi vs oracle"))
            assert_close(g[sl], ref["grad"], tol, (b, s.name, "grad vs oracle"))
    finally:
        pb.close()
