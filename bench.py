"""FastPFP throughput benchmark: pair-solves/s at n = n' = 1000.

One step = one batch of synthetic attributed graph pairs (n = n' = 1000,
p = 0.1, U(0,1) weights, edge noise 0.05, 16-dim attributes, lambda = 1,
alpha = 0.5, eps_1 = eps_2 = 1e-6, I_0 = 100, I_1 = 1000) solved end to end
(affinity, gradient products, projection, blend/normalise, loop control,
greedy discretisation, objective) through fastpfp_match_batched, inputs
resident in HBM.  L2 is flushed between steps.  The whole-job value is the
pairs all ranks solved divided by the slowest rank's summed step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Under torchrun (N > 1) every rank solves its own pairs (weak scaling); the
only collectives are the timing barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fastpfp_pair_solves_per_s_n1000"
UNIT = "pair-solves/s"
WORKLOAD = dict(workload="attributed_1000", n=1000, n2=1000, p=0.1, sigma=0.05, k=16,
                attr_sigma=0.05, lam=1.0, alpha=0.5, tol_outer=1e-6, tol_inner=1e-6,
                max_outer=100, max_inner=1000)
# The dominant kernel of a batched step: the wave projection kernel.
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pdb_kernel_attributed_1000.md")
PD_SOURCE = os.path.join(ROOT, "paper_1207_1114_gb300", "csrc", "projection_batched.cu")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def pd_source_hash() -> str:
    with open(PD_SOURCE, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic_per_launch():
    """DRAM bytes of one projection launch from the committed ncu summary, or
    None when the projection kernel changed since the counters were taken."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    h = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+-]+)", text)
    if not h or not t or h.group(1) != pd_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def make_pairs(rank: int, batch: int):
    from paper_1207_1114_gb300 import synth
    return [synth.attributed_1000(seed=rank * 1000 + b) for b in range(batch)]


def params(F, profile=0, precision="fp32"):
    """The workload's parameters.  bf16: tensor-core products until
    max|dX| < 1e-3, then FP32 iterations (at most 30) to convergence."""
    w = WORKLOAD
    extra = dict(precision=F.BF16, refine_iters=30, switch_tol=1e-3) if precision == "bf16" else {}
    return F.default_params(lam=w["lam"], alpha=w["alpha"], tol_outer=w["tol_outer"],
                            tol_inner=w["tol_inner"], max_outer=w["max_outer"],
                            max_inner=w["max_inner"], profile=profile, **extra)


def cpu_oracle_sample(g, outer_per_pair, inner_per_pair, budget_s=12.0):
    """Times the oracle on one gradient, one blend and a bounded number of
    projection rounds of one pair, and extrapolates to one whole solve with
    the given per-pair iteration counts."""
    import oracle
    A = g.A.astype(np.float64)
    A2 = g.A2.astype(np.float64)
    K = oracle.affinity(g.B, g.B2)
    N = A.shape[0]
    X = np.full((N, N), 1.0 / (N * N))
    t0 = time.perf_counter()
    G = oracle.gradient(A, X, A2, K, g.lam)
    t_grad = time.perf_counter() - t0
    Y = G
    t0 = time.perf_counter()
    Y, _, _ = oracle.pd(Y, fixed_iters=2)
    t_round = (time.perf_counter() - t0) / 2
    rounds = int(max(2, min(400, (budget_s - t_grad) / max(t_round, 1e-6))))
    t0 = time.perf_counter()
    Y, _, _ = oracle.pd(Y, fixed_iters=rounds)
    t_round = (time.perf_counter() - t0) / rounds
    t0 = time.perf_counter()
    oracle.blend(X, np.pad(G, ((0, 0), (0, 0))), 0.5, True)
    t_blend = time.perf_counter() - t0
    t_solve = outer_per_pair * (t_grad + t_blend) + inner_per_pair * t_round
    sample = (f"1 pair of the n=1000 workload: 1 gradient ({t_grad:.2f}s) + {rounds} projection "
              f"rounds ({t_round * 1e3:.2f} ms/round) + 1 blend, extrapolated to "
              f"{outer_per_pair:.1f} outer / {inner_per_pair:.0f} inner iterations per pair")
    return 1.0 / t_solve, sample, t_grad + rounds * t_round + t_blend


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle as it stands, on the host cores."""
    import oracle
    if rank != 0:
        return
    golden = os.path.join(ROOT, "tests", "golden", "attributed_1000_seed0.json")
    with open(golden) as f:
        gold = json.load(f)
    outer = gold["outer_iters"]
    inner = sum(gold["inner"])
    g = make_pairs(0, 1)[0]
    vals, samples = [], []
    for i in range(args.warmup + args.steps):
        v, sample, _ = cpu_oracle_sample(g, outer, inner, budget_s=args.ref_budget)
        if i >= args.warmup:
            vals.append(v)
            samples.append(sample)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD, pairs_per_step=1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": samples[-1] +
                         f"; iteration counts are the oracle's own full solve of seed 0 "
                         f"({outer} outer, {inner} inner)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=7, help="pairs per step and rank")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-budget", type=float, default=10.0, dest="ref_budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="gradient products: plain FP32, or BF16 tensor cores + FP32 refinement")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_1207_1114_gb300 import build as fbuild
    fbuild.build()
    from paper_1207_1114_gb300 import fastpfp as F

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    pairs = make_pairs(rank, args.batch)
    n = WORKLOAD["n"]
    dpairs = [(torch.as_tensor(g.A, device=dev), torch.as_tensor(g.A2, device=dev),
               torch.as_tensor(g.B, device=dev), torch.as_tensor(g.B2, device=dev)) for g in pairs]
    solver = F.Solver(max_n=n, max_batch=args.batch, device=local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    p_plain = params(F, precision=args.precision)
    p_prof = params(F, profile=1, precision=args.precision)
    for _ in range(args.warmup):
        solver.match_batched(dpairs, params=p_plain)
    # timed region: per-step CUDA events, L2 flushed (untimed) before every step
    step_ms, stats_all = [], []
    barrier()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = solver.match_batched(dpairs, params=p_prof)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            stats_all.append([o.stats for o in outs])
            accs = [float((o.perm.cpu().numpy() == g.gt).mean()) for o, g in zip(outs, pairs)]
        barrier()
    total_ms = float(sum(step_ms))
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    pairs_done = args.batch * args.steps * world
    value = pairs_done / (total_ms / 1e3)

    # roofline of the dominant kernel (projection): algorithmic bytes of all
    # its launches / their summed CUDA-event time
    flat = [s for step in stats_all for s in step]
    outer = sum(s.outer_iters for s in flat)
    inner = sum(s.inner_iters_total for s in flat)
    ms_proj = sum(s.ms_proj for s in flat)
    ms_gemm = sum(s.ms_gemm for s in flat)
    ms_disc = sum(s.ms_disc for s in flat)
    bytes_round = 8.0 * n * n              # read + write the FP32 N x N slacked matrix
    bytes_blend = 12.0 * n * n             # read X, read Y[:, :m], write X
    alg_bytes = inner * bytes_round + outer * bytes_blend
    achieved = alg_bytes / (ms_proj / 1e3) / 1e9 if ms_proj > 0 else None
    peak, peak_kind = peaks()
    traffic = ncu_traffic_per_launch()
    launches = sum(s.launches for s in flat)
    # one projection launch per outer iteration of a wave (a step is one wave)
    proj_launches = sum(max(s.outer_iters for s in step) for step in stats_all)

    # end to end through the public host-memory batch entry point: every step
    # copies its pairs from pinned host memory and reads the permutations back
    e2e_value = None
    h2d = d2h = 0
    host = [tuple(torch.as_tensor(a).pin_memory() for a in (g.A, g.A2, g.B, g.B2)) for g in pairs]
    for hp in host:
        h2d += sum(x.numel() * x.element_size() for x in hp)
    d2h = args.batch * n * 4
    solver.match_batched_host(host, params=p_plain)   # warm
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.match_batched_host(host, params=p_plain)
    barrier()
    e2e_s = time.perf_counter() - t0
    tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_value = args.batch * e2e_steps * world / float(tt.item())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        v, sample, _ = cpu_oracle_sample(pairs[0], outer / len(flat), inner / len(flat))
        cpu = {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "bf16+f32", "data": "synthetic",
            "config": dict(WORKLOAD, pairs_per_step=args.batch, precision=args.precision,
                           l2="flushed (512 MB write) before every timed step",
                           parallelism=f"pairs sharded over {world} rank(s)"),
            "accuracy": float(np.mean(accs)),
            "iterations": {"outer_per_pair": outer / len(flat), "inner_per_pair": inner / len(flat)},
            "phase_ms": {"gemm": ms_gemm, "projection": ms_proj, "discretize": ms_disc},
            "roofline": {"kernel": "pdb_kernel (wave projection rounds + blend)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic,
                         "alg_bytes_per_launch": alg_bytes / max(proj_launches, 1)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
