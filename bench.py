#!/usr/bin/env python3
"""Benchmark of the periodic Coulomb sum on one GB300 (or N replicas).

One step = one pass of the whole hot path (psum_eval: validation, spatial sort,
near-field pair sum at the charges and the check points, least-squares fit,
zero-mean constant, far field, combination) over 100,000 charges in the
(1, 1.5, 2) box with p = 16 and M = 800, FP32C pair arithmetic.  Inputs are
resident in device memory; L2 is flushed (a 256 MiB write) before every timed
step, outside the timed events.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "periodic Coulomb pair-interactions/s (pot+force) at 1e-6 rel err, FP32 vs FP64"
UNIT = "pairs/s"
N_MAIN, D_MAIN, P_MAIN, M_MAIN, SEED_MAIN = 100_000, (1.0, 1.5, 2.0), 16, 800, 2
# Algorithmic work of one potential+gradient pair (the contract's count): the minimal
# instruction stream of one (target, source, image) term -- 3 offset subtractions, 1 multiply
# and 2 fused multiply-adds for r^2, 1 select for K(0) = 0, q/r, the potential add, 1/r^2,
# q/r^3 and 3 fused multiply-adds for the field: 14 FP32-pipe operations (and one MUFU rsqrt).
FP32_OPS_PAIR_ALG = 14
FP32_OPS_PAIR_GRAD = 13    # FP32-pipe lane operations per potential+gradient pair, one-sided kernel
                           # (3 sub, 3 r^2, 4 phi/weight, 3 grad)
# symmetric kernel: per step a lane pairs its 4 targets with two sources (16 ordered pairs,
# both directions) in 76 packed f32x2 operations (152 lane operations: per target 3 sub,
# 3 r^2, 1 1/r^2, 6 action and 5-6 reaction operations, and the block of 4 targets' potential
# reactions added to the running sum)
FP32_OPS_PAIR_SYM = 152 / 16
FP32_OPS_PAIR_PHI = 7      # potential only (3 sub, 3 r^2, 1 fma)
FP64_OPS_PAIR = 19         # float64 kernel, one-sided
FP64_OPS_PAIR_SYM = 12     # float64 kernel, symmetric


def workload_name(N=N_MAIN):
    return f"uniform Gaussian charges, N={N}, box d=(1,1.5,2), p=16, M=800, 3x3x3 near images, fp32c"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="psum", choices=["psum", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the trimmed / RBF / Gauss-grid leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU budget of the oracle sample")
    ap.add_argument("--n", type=int, default=N_MAIN, help="charges (smaller cases are for profiling only)")
    ap.add_argument("--pairs", default="auto", choices=["auto", "one-sided", "symmetric"],
                    help="pair kernel of the charge sums (auto: symmetric from 12 tiles of 512 charges)")
    ap.add_argument("--terms", default="fast", choices=["fast", "refined"],
                    help="float32 pair terms of the main workload (refined: float-float offsets and 1/r fused "
                         "into the sums, for strongly cancelling systems)")
    ap.add_argument("--checks", default="auto", choices=["auto", "points", "layers"],
                    help="form of the check-point sums (auto: the two image layers at the M points)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [s for s, p in zip(sm, power)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "samples": len(rows), "power_w_max": max(power) if power else None, "reasons": reasons}


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest value over all ranks (every rank gets it); the value itself without a group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pairs_per_rank_step: int, world: int, steps: int, total_ms_max: float) -> float:
    """Whole-job pairs/s: every rank evaluates its own system (weak scaling), timed by the
    slowest rank."""
    return pairs_per_rank_step * world * steps / (total_ms_max * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def near_code_hash():
    """First 16 hex digits of the SHA-256 of the symmetric charge kernel's code
    (near_common.cuh and near_sym.cu): comments removed and whitespace collapsed, so that
    a comment edit keeps the recorded counters valid."""
    import re
    src = ""
    for name in ("near_common.cuh", "near_sym.cu"):
        with open(os.path.join(ROOT, "paper_1310_4374_gb300", "csrc", name)) as f:
            src += f.read() + "\n"
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256(" ".join(src.split()).encode()).hexdigest()[:16]


def near_kernel_traffic(n_points, kernel, image_groups, terms="fast"):
    """DRAM bytes per launch of the charge near-field kernel from the committed ncu
    summary of a smaller case: the read of the packed sources (which stay in L2) scales
    with the number of points; the write of the partial sums scales with the number of
    partial slots (symmetric kernel: tiles^2 x image groups, 16 KiB each).  None if the
    record is for the other kernel or the kernel source has changed since the counters
    were taken."""
    path = os.path.join(ROOT, "profiles", "near32_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if (rec.get("near_code_sha256_16") != near_code_hash() or rec.get("pair_kernel") != kernel
                or rec.get("terms", "fast") != terms):
            return None
        read = rec["dram_read_bytes"] * n_points / rec["n_points"]
        if kernel == "symmetric":
            tiles = (n_points + 511) // 512
            slots, slots_rec = tiles * tiles * image_groups, rec["n_tiles"] ** 2 * rec["image_groups"]
            return read + rec["dram_write_bytes"] * slots / slots_rec
        return read + rec["dram_write_bytes"]
    except Exception:
        return None


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_psum(args):
    import numpy as np
    import torch

    from paper_1310_4374_gb300 import binding as B
    from paper_1310_4374_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()

    # every rank evaluates its own replica of the system (weak scaling, no exchange)
    s = W.uniform_gauss(N=args.n, d=D_MAIN, p=P_MAIN, M=M_MAIN, seed=SEED_MAIN + rank)
    pairs_step = 27 * s.N * (s.N + 2 * s.M)
    pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c", pairs=args.pairs, checks=args.checks,
                           terms=args.terms)
    pair_kernel, image_groups = B.psum_pair_kernel(pc.plan, s.N)
    check_form = B.psum_check_form(pc.plan)
    # interactions the kernels evaluate: the charge sums, and the check sums as 27 images at
    # the 2M points, or as the two 9-image layers at the M points (same right-hand side)
    pairs_evaluated = 27 * s.N * s.N + (18 * s.N * s.M if check_form == "layers" else 27 * s.N * 2 * s.M)
    B.psum_profile(pc.plan, True)
    x = torch.as_tensor(s.x, dtype=torch.float64, device=dev)
    q = torch.as_tensor(s.q, dtype=torch.float64, device=dev)
    phi = torch.empty(s.N, dtype=torch.float64, device=dev)
    grad = torch.empty((s.N, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        B.psum_eval(pc.plan, x, q, phi, grad, stream=stream)

    for _ in range(max(args.warmup, 0)):
        step()
    st = B.psum_sync(pc.plan, stream)
    if st != B.PSUM_OK:
        raise B.PsumError(st, "warm-up")
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = B.psum_launch_count(pc.plan)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_ms = []
    torch.cuda.synchronize()
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        stage_ms.append(B.psum_last_timings(pc.plan, stream))     # waits for the stream
    torch.cuda.synchronize()
    barrier()
    launches = B.psum_launch_count(pc.plan) - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = B.psum_sync(pc.plan, stream)
    if st != B.PSUM_OK:
        raise B.PsumError(st, "timed steps")
    total_ms = max_over_ranks(sum(step_ms), dist, device=dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(pairs_step, world, args.steps, total_ms)

    # dominant kernel: the near-field sum at the charges (potential + gradient)
    near_ms = statistics.mean(t["near_charges"] for t in stage_ms)
    near_pairs = 27 * s.N * s.N
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * sm_max * 1e6
    sym = pair_kernel == "symmetric"
    ops_exec = FP32_OPS_PAIR_SYM if sym else FP32_OPS_PAIR_GRAD
    pair_rate = near_pairs / (near_ms * 1e-3)
    # achieved = algorithmic operations (14 per pair) x pairs of one launch / its duration
    achieved = FP32_OPS_PAIR_ALG * pair_rate
    traffic = near_kernel_traffic(s.N, pair_kernel, image_groups, args.terms)
    roofline = {"bound": "alu", "kernel": "k_near32s (symmetric pairs)" if sym else "k_near32<grad>",
                "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "T FP32-pipe ops/s", "frac": achieved / peak_ops, "traffic": traffic,
                "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz "
                               "(sm_max_mhz of MEASURED_PEAKS.json, measured)",
                "ops_per_pair": FP32_OPS_PAIR_ALG,
                "ops_per_pair_note": "algorithmic count of one pot+grad pair (14 FP32-pipe operations + 1 MUFU)",
                "pairs_per_launch": near_pairs, "pair_rate": pair_rate, "kernel_ms": near_ms,
                # the share of the FP32 pipe the kernel's own instruction stream keeps busy
                "issue_frac": ops_exec * pair_rate / peak_ops, "executed_ops_per_pair": ops_exec,
                # x, q in and phi, grad phi out, float64: 64 bytes per charge
                "algorithmic_bytes_per_launch": 64 * s.N}
    if sym:
        roofline["image_groups"] = image_groups
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = achieved / (props.multi_processor_count * 128 * clk["sm_mhz"] * 1e6)

    value_evaluated = pairs_evaluated * world * args.steps / (total_ms * 1e-3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "value_counts": "nominal pairs 27 N (N + 2M): the 3x3x3 image sum at the N charges and at the "
                           "2M check points; value_evaluated counts the pairs the kernels evaluate "
                           "(27 N^2 + 18 N M with the check sums as two image layers)",
           "value_evaluated": value_evaluated,
           "step_ms": step_ms,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_name(s.N), "N": s.N, "p": s.p, "M": s.M, "box": list(s.d),
                      "near_images": 27, "pairs_per_step": pairs_step,
                      "check_form": check_form + (" (phi_near(y~) - phi_near(y) as the image layer beyond "
                                                  "the partner's face minus the opposite layer, 18 images at "
                                                  "the M points)" if check_form == "layers" else ""),
                      "pairs_evaluated_per_step": pairs_evaluated,
                      "terms": args.terms,
                      "precision": "fp32c: f32 pair arithmetic on group-relative coordinates, two-sum "
                                   "compensated accumulation; f64 sort keys, fit, mean and far field",
                      "l2": "flushed before every timed step (256 MiB write, outside the events)",
                      "pair_kernel": pair_kernel + (" (each mirror pair (i,j,p)/(j,i,-p) shares one offset "
                                                    "and one 1/r)" if sym else ""),
                      "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
           "solves_per_s": world * args.steps / (total_ms * 1e-3),
           "stages_ms": {k: statistics.mean(t[k] for t in stage_ms) for k in stage_ms[0]},
           "roofline": roofline, "gpu_launches": launches, "clocks": clk,
           "paper_context": "no GPU throughput published; the paper's brute-force periodic sum on a Tesla C2050 "
                            "(Fermi, FP64) ran up to ~100x a 4-core Intel QX6780 and was faster than the CPU FMM "
                            "up to N~40k (Sec. 4.3, Fig. 5); its practical GPU ceiling was N~1e5"}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(pc, s, args)
    if rank == 0 and not args.no_fp64:
        out["fp64"] = fp64_leg(args)
    if rank == 0 and not args.no_batch:
        out["batch"] = batch_leg(args)
    if rank == 0 and not args.no_backward:
        out["backward"] = backward_leg(args)
    if rank == 0 and not args.no_variants:
        out["variants"] = variants_leg(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_leg(s, phi, grad, args)
    pc.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def e2e_leg(pc, s, args):
    """The same metric through psum_eval_host: host buffers, copies inside the timed region."""
    import numpy as np
    import torch

    from paper_1310_4374_gb300 import binding as B

    x = torch.as_tensor(s.x, dtype=torch.float64).pin_memory()
    q = torch.as_tensor(s.q, dtype=torch.float64).pin_memory()
    phi = torch.empty(s.N, dtype=torch.float64).pin_memory()
    grad = torch.empty((s.N, 3), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    B.psum_profile(pc.plan, False)
    st = B.psum_eval_host(pc.plan, x, q, phi, grad, stream=stream)     # warm-up
    if st != B.PSUM_OK:
        raise B.PsumError(st, "e2e warm-up")
    times = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        st = B.psum_eval_host(pc.plan, x, q, phi, grad, stream=stream)
        times.append(time.perf_counter() - t0)
        if st != B.PSUM_OK:
            raise B.PsumError(st, "e2e")
    clk = clocks.stop()
    B.psum_profile(pc.plan, True)
    pairs = 27 * s.N * (s.N + 2 * s.M)
    t = statistics.mean(times)
    return {"value": pairs / t, "unit": UNIT, "h2d_bytes_per_step": int(x.numel() * 8 + q.numel() * 8),
            "d2h_bytes_per_step": int(phi.numel() * 8 + grad.numel() * 8), "ms_per_step": t * 1e3,
            "step_ms": [v * 1e3 for v in times], "clocks": clk,
            "api": "psum_eval_host (pinned host buffers; copies and final synchronisation timed)"}


def fp64_leg(args):
    """The FP64 pair kernel against FP32C (and float-float) on the headline workload itself:
    100k uniform Gaussian charges in the (1, 1.5, 2) box, p = 16, M = 800.  One warm-up and
    `reps` timed evaluations per precision (an FP64 evaluation takes about 6 s)."""
    import torch

    from paper_1310_4374_gb300 import binding as B
    from paper_1310_4374_gb300 import workloads as W

    s = W.uniform_gauss(N=args.n, d=D_MAIN, p=P_MAIN, M=M_MAIN, seed=SEED_MAIN)
    x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
    q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
    res = {}
    outs = {}
    for prec, reps in (("fp64", 1), ("ff", 2), ("fp32c", 3)):
        pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision=prec)
        B.psum_profile(pc.plan, True)
        phi, g = pc(x, q)                       # warm-up
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        near = []
        ev0.record()
        for _ in range(reps):
            phi, g = pc(x, q, check=False)
            near.append(B.psum_last_timings(pc.plan)["near_charges"])
        ev1.record()
        torch.cuda.synchronize()
        st = B.psum_sync(pc.plan)
        if st != B.PSUM_OK:
            raise B.PsumError(st, "fp64 leg")
        ms = ev0.elapsed_time(ev1) / reps
        near_ms = statistics.mean(near)
        kernel = B.psum_pair_kernel(pc.plan, s.N)[0]
        pc.close()
        pairs = 27 * s.N * (s.N + 2 * s.M)
        near_rate = 27 * s.N * s.N / (near_ms * 1e-3)
        res[prec] = {"pairs_per_s": pairs / (ms * 1e-3), "ms_per_step": ms, "timed_steps": reps,
                     "near_charges_pairs_per_s": near_rate, "near_charges_ms": near_ms, "pair_kernel": kernel}
        if prec == "fp64":
            # float64 lane operations per ordered pair: one-sided 3 offset, 3 r^2, 5 rsqrt
            # refinement, 1 q/r, 1 sum, 2 weight, 3 field; symmetric per mirror pair 3 + 3 + 5
            # + 1 (1/r^2) shared and 6 per direction, 24 for two ordered pairs
            ops = FP64_OPS_PAIR_SYM if kernel == "symmetric" else FP64_OPS_PAIR
            props = torch.cuda.get_device_properties(x.device)
            peak = props.multi_processor_count * 2 * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6
            res[prec]["roofline"] = {"bound": "alu", "kernel": "k_near64s" if kernel == "symmetric" else "k_near64",
                                     "ops_per_pair": FP32_OPS_PAIR_ALG,
                                     "achieved": FP32_OPS_PAIR_ALG * near_rate / 1e12, "peak": peak / 1e12,
                                     "unit": "T FP64-pipe ops/s", "frac": FP32_OPS_PAIR_ALG * near_rate / peak,
                                     "issue_frac": ops * near_rate / peak, "executed_ops_per_pair": ops,
                                     "peak_source": "SMs x 2 FP64 lanes x sm_max_mhz (nominal 1.25 TFLOP/s FP64; "
                                                    "1.90 DFMA/clk/SM measured)"}
        outs[prec] = (phi.cpu().numpy(), g.cpu().numpy())
    import numpy as np

    def rel(a, b):
        return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))

    def mx(a, b):
        return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(b ** 2)))
    res["workload"] = workload_name(s.N).replace("fp32c", "fp64, ff and fp32c")
    res["speedup_fp32c_over_fp64"] = res["fp32c"]["pairs_per_s"] / res["fp64"]["pairs_per_s"]
    res["speedup_ff_over_fp64"] = res["ff"]["pairs_per_s"] / res["fp64"]["pairs_per_s"]
    for a in ("fp32c", "ff"):
        res[f"eps2_{a}_vs_fp64"] = {"phi": rel(outs[a][0], outs["fp64"][0]), "grad": rel(outs[a][1], outs["fp64"][1]),
                                    "phi_max_over_rms": mx(outs[a][0], outs["fp64"][0]),
                                    "grad_max_over_rms": mx(outs[a][1], outs["fp64"][1])}
    return res


def batch_leg(args):
    """256 independent +-1 systems (N log-uniform in [500, 20000], boxes (1, U[1,2], U[1,2]),
    p in {8, 12, 16}) in one batched evaluation replayed from a CUDA graph."""
    import numpy as np
    import torch

    from paper_1310_4374_gb300 import binding as B
    from paper_1310_4374_gb300 import workloads as W

    systems = W.config(4)
    t0 = time.perf_counter()
    pb = B.PeriodicBatch(systems, precision="fp32c", checks=args.checks)
    t_plans = time.perf_counter() - t0
    check_forms = sorted({B.psum_check_form(p) for p in pb.plans})
    try:
        x = torch.as_tensor(np.concatenate([s.x for s in systems]), dtype=torch.float64, device="cuda")
        q = torch.as_tensor(np.concatenate([s.q for s in systems]), dtype=torch.float64, device="cuda")
        phi = torch.empty_like(q)
        grad = torch.empty_like(x)
        for _ in range(max(args.warmup, 1)):
            pb(x, q, phi, grad, use_graph=True)
        info = B.psum_batch_get_info(pb.batch)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            B.psum_batch_eval(pb.batch, x, q, phi, grad, use_graph=True)
        ev1.record()
        torch.cuda.synchronize()
        first, _ = B.psum_batch_sync(pb.batch, pb.B)
        if first != B.PSUM_OK:
            raise B.PsumError(first, "batch leg")
        ms = ev0.elapsed_time(ev1) / reps
    finally:
        pb.close()
    wide = sum(1 for s in systems if tuple(s.K) != (1, 1, 1))
    return {"workload": f"{len(systems)} systems, N log-uniform in [500, 20000] (total {info['N_total']}), "
                        "d = (1, U[1,2], U[1,2]), p in {8,12,16}, +-1 charges, fp32c, CUDA graph; "
                        f"{wide} flat boxes with a widened near block (K = (2,1,1))",
            "pairs_per_s": info["pairs"] / (ms * 1e-3), "systems_per_s": len(systems) / (ms * 1e-3),
            "ms_per_step": ms, "pairs_per_step": info["pairs"], "ctas": info["ctas"],
            "autotuned_variant": info["variant"], "plan_setup_s": t_plans, "check_form": "/".join(check_forms)}


def backward_leg(args):
    """Energy, forces and dE/dq of 100k tight dipoles (200k charges) in the (1, 1, 2) box,
    p = 16, M = 800, fp32c: forward psum_eval + psum_energy + psum_energy_backward.  The
    potential of this system cancels strongly (about 20x below the root-sum-square of its
    terms), so it runs the refined float32 terms that meet the 1e-6 bound; the fast terms'
    forward is timed beside it."""
    import torch

    from paper_1310_4374_gb300 import binding as B
    from paper_1310_4374_gb300 import workloads as W

    s = W.config(5)
    x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
    q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
    phi = torch.empty_like(q)
    grad = torch.empty_like(x)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    dEdq = torch.empty_like(q)
    dEdx = torch.empty_like(x)
    res = {}
    for terms in ("refined", "fast"):
        pc = B.PeriodicCoulomb(s.d, s.p, s.M, precision="fp32c", terms=terms)
        try:
            def step():
                B.psum_eval(pc.plan, x, q, phi, grad)
                B.psum_energy(pc.plan, q, phi, E)
                B.psum_energy_backward(pc.plan, x, q, phi, grad, None, dEdq, dEdx)

            step()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            B.psum_eval(pc.plan, x, q, phi, grad)
            B.psum_energy(pc.plan, q, phi, E)
            ev[1].record()
            B.psum_energy_backward(pc.plan, x, q, phi, grad, None, dEdq, dEdx)
            ev[2].record()
            torch.cuda.synchronize()
            st = B.psum_sync(pc.plan)
            if st != B.PSUM_OK:
                raise B.PsumError(st, "backward leg")
            res[terms] = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), B.psum_scratch_bytes(pc.plan, s.N))
        finally:
            pc.close()
    fwd, bwd, (nbytes, bands) = res["refined"]
    pairs_f = 27 * s.N * (s.N + 2 * s.M)
    pairs_b = 27 * s.N * 2 * s.M
    return {"workload": "100k dipole pairs (200k charges, +-0.8, separation 0.01), d = (1,1,2), p = 16, M = 800, "
                        "fp32c with refined terms",
            "forward_ms": fwd, "backward_ms": bwd, "pairs_per_s": (pairs_f + pairs_b) / ((fwd + bwd) * 1e-3),
            "pairs_forward": pairs_f, "pairs_backward": pairs_b, "scratch_bytes": nbytes, "bands": bands,
            "fast_terms": {"forward_ms": res["fast"][0], "backward_ms": res["fast"][1],
                           "note": "eps2(phi) 1.33e-6 on this system, above the 1e-6 bound"}}


def variants_leg(args):
    """The options of Secs. 2-3 on one cube workload (100k uniform Gaussian charges in the
    unit cube, p = 16, fp32c): the 3x3x3 block with the spherical basis and Fibonacci check
    points, the near set trimmed to the ball at lambda = sqrt(3) (get step 2; the block's own
    lambda_eff on a cube), the RBF basis of Eq. 5, and the Gauss spherical grid.  Each is
    timed (CUDA events, mean of 2 evaluations after a warm-up) and compared with the block."""
    import numpy as np
    import torch

    from paper_1310_4374_gb300 import binding as B
    from paper_1310_4374_gb300 import workloads as W

    s = W.uniform_gauss(N=N_MAIN, d=(1.0, 1.0, 1.0), p=P_MAIN, M=M_MAIN, seed=SEED_MAIN + 200)
    x = torch.as_tensor(s.x, dtype=torch.float64, device="cuda")
    q = torch.as_tensor(s.q, dtype=torch.float64, device="cuda")
    cases = [("block", dict()),
             ("ball_sqrt3", dict(lam=3 ** 0.5)),
             ("rbf256", dict(basis="rbf")),
             ("gauss_grid", dict(points="gauss"))]
    res, ref = {}, None
    for name, kw in cases:
        M = 0 if kw.get("points") == "gauss" else s.M
        pc = B.PeriodicCoulomb(s.d, s.p, M, precision="fp32c", **kw)
        try:
            B.psum_profile(pc.plan, True)
            phi, g = pc(x, q)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(2):
                phi, g = pc(x, q, check=False)
            ev1.record()
            torch.cuda.synchronize()
            st = B.psum_sync(pc.plan)
            if st != B.PSUM_OK:
                raise B.PsumError(st, "variants leg")
            info = pc.info
            r = {"ms_per_step": ev0.elapsed_time(ev1) / 2,
                 "stages_ms": B.psum_last_timings(pc.plan),
                 "M": info["M"], "P": info["P"], "images": info["n_images"], "lambda_eff": info["lambda_eff"]}
        finally:
            pc.close()
        phi, g = phi.cpu().numpy(), g.cpu().numpy()
        if ref is None:
            ref = (phi, g)
        else:
            r["eps2_vs_block"] = {"phi": float(np.sqrt(np.mean((phi - ref[0]) ** 2) / np.mean(ref[0] ** 2))),
                                  "grad": float(np.sqrt(np.mean((g - ref[1]) ** 2) / np.mean(ref[1] ** 2)))}
            r["speedup_vs_block"] = res["block"]["ms_per_step"] / r["ms_per_step"]
        res[name] = r
    res["workload"] = (f"uniform Gaussian charges, N={s.N}, unit cube, p={s.p}, fp32c; "
                       "block: 27 images, Fibonacci M=800; ball: lambda=sqrt(3); rbf: 256 centres on S_b; "
                       "gauss: M=(p+1)(2p+1)")
    return res


def cpu_baseline_leg(s, phi_gpu, grad_gpu, args):
    """The oracle on the host cores on a bounded sample: the 2M check-point rows plus a
    seeded sample of targets, with the fit, mean and far field; also the GPU's error there."""
    import numpy as np

    from oracle import psum_oracle as O

    pl = O.Plan(s.d, s.p, s.M)
    rng = np.random.default_rng(1234)
    # size the target sample from a short calibration run
    n_probe = max(64, 8 * O.num_threads())
    probe = s.x[:n_probe]
    t0 = time.perf_counter()
    O.near_sum(probe, s.x, s.q, s.d, grad=True)
    rate = 27 * s.N * n_probe / (time.perf_counter() - t0)      # pairs/s on all host cores
    n_check_pairs = 27 * s.N * 2 * s.M
    n_t = int(max(64, min(16384, (args.cpu_seconds * rate - n_check_pairs) / (27 * s.N))))
    sample = np.sort(rng.choice(s.N, size=n_t, replace=False))
    t0 = time.perf_counter()
    ref = pl.evaluate(s.x, s.q, targets=s.x[sample])
    dt = time.perf_counter() - t0
    pairs = 27 * s.N * (2 * s.M + n_t)
    phi = phi_gpu.cpu().numpy()[sample]
    g = grad_gpu.cpu().numpy()[sample]
    return {"value": pairs / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"near sums at the {2 * s.M} check points and {n_t} seeded charges of the same "
                      f"{s.N}-charge system, plus the fit, mean and far field ({pairs:.3e} pairs, {dt:.1f} s)",
            "gpu_eps2_on_sample": {"phi": O.relative_l2(phi, ref["phi"]), "grad": O.relative_l2(g, ref["grad"])}}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    from oracle import psum_oracle as O
    from paper_1310_4374_gb300 import workloads as W

    s = W.uniform_gauss(N=N_MAIN, d=D_MAIN, p=P_MAIN, M=M_MAIN, seed=SEED_MAIN)
    pl = O.Plan(s.d, s.p, s.M)
    rng = np.random.default_rng(4321)
    n_t = 64
    pairs = 27 * s.N * (2 * s.M + n_t)

    def step():
        sample = np.sort(rng.choice(s.N, size=n_t, replace=False))
        pl.evaluate(s.x, s.q, targets=s.x[sample])

    for _ in range(max(args.warmup, 0)):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = pairs * args.steps / dt
    sample = (f"per step: near sums at the {2 * s.M} check points and {n_t} seeded charges of the "
              f"{s.N}-charge system, plus the fit, mean and far field ({pairs:.3e} pairs)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name().replace("fp32c", "CPU oracle f64"),
                                            "sampled": True},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_psum(args)


if __name__ == "__main__":
    main()
