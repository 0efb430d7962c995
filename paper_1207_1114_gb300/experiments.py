"""The paper's synthetic experiments, run through the library on one GPU.

* ``e1``: Section 5.1 — unweighted random graphs with 50 % connectivity, n
  from 100 to 1500, matched in four cases (isomorphic; n edge editions; 10 %
  node deletion; both).  Each row records the runtime of one solve and the
  matching error ||A - X A' X^T||_F^2 - ||A - X_GT A' X_GT^T||_F^2 of the
  discrete result, for FastPFP (alpha = 0.5), the projected gradient
  method of Eq. (pg) (step 1 / L, L = ||A||_2 ||A'||_2) and FastGA
  (Appendix; fixed beta on Q / max|Q|, default 100), the paper's three
  O(n^3) methods.
* ``alpha``: Section 6's step-size sensitivity — FastPFP on attributed
  n = 1000 pairs for alpha from 0.1 to 1: outer iterations, runtime,
  accuracy and objective.
* ``compare``: FastPFP, PG and FastGA on the same single pairs of the
  synthetic workloads (plain weighted n = 300 and 1000, attributed n = 1000,
  partial 1000 into 1200): time per solve, outer iterations, accuracy —
  the paper's runtime comparisons (Sections 5.1-5.4) on synthetic inputs.
* ``wave``: one wave of attributed pairs (one batched call, outer loop
  enqueued by the host so every kernel is a plain launch): the small,
  fixed case the kernel profiles are captured on.

Usage::

    python -m paper_1207_1114_gb300.experiments e1 [--sizes 100,300,...] [--json out.json]
    python -m paper_1207_1114_gb300.experiments alpha [--seeds 0,1,2] [--json out.json]
    python -m paper_1207_1114_gb300.experiments compare [--seeds 0,1,2] [--json out.json]
    python -m paper_1207_1114_gb300.experiments wave [--pairs 17] [--n 1000] [--max-outer 1]

Every solve runs on the CUDA path (``Solver.match``); the host only draws
the inputs (``synth``) and scores the discrete results.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import fastpfp as F
from . import synth

E1_SIZES = (100, 300, 500, 700, 900, 1100, 1300, 1500)
ALPHAS = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0)


def matching_error(A: np.ndarray, A2: np.ndarray, perm: np.ndarray) -> float:
    """||A - X A' X^T||_F^2 for the partial permutation X with
    X[i, perm[i]] = 1 (rows with perm[i] < 0 are zero), in float64."""
    A = A.astype(np.float64)
    A2 = A2.astype(np.float64)
    n = A.shape[0]
    idx = np.where(perm >= 0)[0]
    M = np.zeros((n, n))
    M[np.ix_(idx, idx)] = A2[np.ix_(perm[idx], perm[idx])]
    return float(((A - M) ** 2).sum())


def lipschitz_step(A: np.ndarray, A2: np.ndarray, iters: int = 60) -> float:
    """1 / (||A||_2 ||A'||_2), the projected gradient method's step (power
    iteration for the spectral norms)."""
    def norm2(a):
        v = np.ones(a.shape[0]) / np.sqrt(a.shape[0])
        for _ in range(iters):
            w = a @ v
            nw = np.linalg.norm(w)
            if nw == 0.0:
                return 0.0
            v = w / nw
        return float(np.linalg.norm(a @ v))
    L = norm2(A.astype(np.float64)) * norm2(A2.astype(np.float64))
    return 1.0 / L if L > 0 else 1.0


def _solve_timed(solver, g, params, dev, want_X=False):
    import torch
    A = torch.as_tensor(g.A, device=dev)
    A2 = torch.as_tensor(g.A2, device=dev)
    B = torch.as_tensor(g.B, device=dev) if g.k else None
    B2 = torch.as_tensor(g.B2, device=dev) if g.k else None
    solver.match(A, A2, B, B2, params=params)          # warm-up (graph capture, caches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = solver.match(A, A2, B, B2, params=params, want_X=want_X)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def e1_sweep(sizes=E1_SIZES, cases="abcd", seeds=(0,), algorithms=("fastpfp", "pg", "fastga"), device: int = 0,
             max_outer: int = 100, max_inner: int = 1000, detail: bool = False, beta: float = 100.0):
    """Rows of the Section 5.1 sweep (one per size, case, seed, algorithm).
    detail: each row also carries the solve's permutation, its inner-count
    trace, its soft assignment X and its parameters (for checking against
    the oracle)."""
    import torch
    dev = torch.device("cuda", device)
    solver = F.Solver(max_n=max(sizes), max_batch=1, device=device)
    rows = []
    try:
        for n in sizes:
            for case in cases:
                for seed in seeds:
                    g = synth.e1_pair(n, case, seed=seed)
                    err_gt = matching_error(g.A, g.A2, g.gt)
                    for alg in algorithms:
                        if alg == "pg":
                            alpha = lipschitz_step(g.A, g.A2)
                            p = F.default_params(lam=0.0, alpha=alpha, algorithm=F.ALG_PG, normalize_max=0,
                                                 max_outer=max_outer, max_inner=max_inner)
                        elif alg == "fastga":
                            alpha = float("nan")   # no step size: the soft-assignment replaces X
                            p = F.default_params(lam=0.0, algorithm=F.ALG_FASTGA, beta=beta,
                                                 max_outer=max_outer, max_inner=max_inner)
                        else:
                            alpha = 0.5
                            p = F.default_params(lam=0.0, alpha=alpha, max_outer=max_outer, max_inner=max_inner)
                        r, sec = _solve_timed(solver, g, p, dev, want_X=detail)
                        perm = r.perm.cpu().numpy()
                        inl = g.gt >= 0
                        rows.append(dict(n=n, case=case, seed=seed, algorithm=alg, alpha=alpha,
                                         seconds=sec, outer=int(r.stats.outer_iters),
                                         converged=bool(r.stats.converged),
                                         error=matching_error(g.A, g.A2, perm) - err_gt,
                                         accuracy=float((perm[inl] == g.gt[inl]).mean())))
                        if detail:
                            rows[-1].update(perm=perm, inner=solver.last_trace()[0], X=r.X.cpu().numpy(),
                                            objective=float(r.stats.objective),
                                            max_outer=max_outer, max_inner=max_inner)
    finally:
        solver.close()
    return rows


def alpha_sweep(alphas=ALPHAS, seeds=(0, 1, 2), device: int = 0, n: int = 1000, detail: bool = False):
    """Rows of the step-size sweep on attributed n-node pairs (one per alpha
    and seed).  detail: each row also carries the permutation, the
    inner-count trace and the soft assignment X."""
    import torch
    dev = torch.device("cuda", device)
    solver = F.Solver(max_n=n, max_batch=1, device=device)
    rows = []
    try:
        for seed in seeds:
            g = synth.attributed_1000(seed=seed, n=n)
            for a in alphas:
                p = F.default_params(lam=g.lam, alpha=float(a))
                r, sec = _solve_timed(solver, g, p, dev, want_X=detail)
                perm = r.perm.cpu().numpy()
                rows.append(dict(alpha=float(a), seed=seed, seconds=sec, outer=int(r.stats.outer_iters),
                                 converged=bool(r.stats.converged), objective=float(r.stats.objective),
                                 accuracy=float((perm == g.gt).mean())))
                if detail:
                    rows[-1].update(perm=perm, inner=solver.last_trace()[0], X=r.X.cpu().numpy())
    finally:
        solver.close()
    return rows


COMPARE_CASES = (
    ("plain_300", lambda seed: synth.graph_pair(300, p=0.3, sigma=0.02, k=0, seed=seed)),
    ("plain_1000", lambda seed: synth.graph_pair(1000, p=0.1, sigma=0.02, k=0, seed=seed)),
    ("attributed_1000", lambda seed: synth.attributed_1000(seed=seed)),
    ("partial_1000_1200", lambda seed: synth.partial_1000_1200(seed=seed)),
)


def compare(seeds=(0,), device: int = 0, beta: float = 100.0, cases=COMPARE_CASES):
    """Rows of the method comparison: one per case, seed and method (FastPFP
    alpha = 0.5, PG with step 1/L, FastGA with the fixed beta), each a timed
    single-pair solve after an untimed one."""
    import torch
    dev = torch.device("cuda", device)
    solver = F.Solver(max_n=1200, max_batch=1, device=device)
    rows = []
    try:
        for name, make in cases:
            for seed in seeds:
                g = make(seed)
                for alg in ("fastpfp", "pg", "fastga"):
                    if alg == "pg":
                        p = F.default_params(lam=g.lam, alpha=lipschitz_step(g.A, g.A2), algorithm=F.ALG_PG,
                                             normalize_max=0)
                    elif alg == "fastga":
                        p = F.default_params(lam=g.lam, algorithm=F.ALG_FASTGA, beta=beta)
                    else:
                        p = F.default_params(lam=g.lam)
                    r, sec = _solve_timed(solver, g, p, dev)
                    perm = r.perm.cpu().numpy()
                    inl = g.gt >= 0
                    rows.append(dict(case=name, seed=seed, algorithm=alg, seconds=sec,
                                     outer=int(r.stats.outer_iters), inner=int(r.stats.inner_iters_total),
                                     converged=bool(r.stats.converged), objective=float(r.stats.objective),
                                     accuracy=float((perm[inl] == g.gt[inl]).mean())))
    finally:
        solver.close()
    return rows


def wave(pairs: int = 17, n: int = 1000, max_outer: int = 1, precision: str = "fp32", device: int = 0):
    """One batched solve of `pairs` attributed n-node pairs (seeds 0..) with
    the host-enqueued outer loop and at most max_outer outer iterations;
    returns (seconds, stats of pair 0)."""
    import torch
    dev = torch.device("cuda", device)
    prec = {"fp32": F.FP32, "bf16": F.BF16, "fp8": F.FP8, "fp32_simt": F.FP32_SIMT}[precision]
    solver = F.Solver(max_n=n, max_batch=pairs, device=device)
    try:
        gs = [synth.attributed_1000(seed=i, n=n) for i in range(pairs)]
        d = [tuple(torch.as_tensor(a, device=dev) for a in (g.A, g.A2, g.B, g.B2)) for g in gs]
        p = F.default_params(lam=gs[0].lam, max_outer=max_outer, loop_mode=1, precision=prec)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = solver.match_batched(d, params=p)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, out[0].stats
    finally:
        solver.close()


def _table(rows, keys):
    out = ["| " + " | ".join(keys) + " |", "|" + "---|" * len(keys)]
    for r in rows:
        out.append("| " + " | ".join(f"{r[k]:.4g}" if isinstance(r[k], float) else str(r[k]) for k in keys) + " |")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("which", choices=["e1", "alpha", "wave", "compare"])
    ap.add_argument("--pairs", type=int, default=17)
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--max-outer", type=int, default=1, dest="max_outer")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp8", "fp32_simt"])
    ap.add_argument("--sizes", default=",".join(map(str, E1_SIZES)))
    ap.add_argument("--cases", default="abcd")
    ap.add_argument("--seeds", default="0")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--json", default=None, help="also write the rows to this file")
    a = ap.parse_args(argv)
    seeds = tuple(int(s) for s in a.seeds.split(","))
    if a.which == "wave":
        sec, st = wave(a.pairs, a.n, a.max_outer, a.precision, device=a.device)
        print(f"wave of {a.pairs} pairs of n = {a.n}: {sec * 1e3:.1f} ms, outer {st.outer_iters}, "
              f"inner {st.inner_iters_total}, wave_pairs {st.wave_pairs}")
        return
    if a.which == "compare":
        rows = compare(seeds=seeds, device=a.device)
        print(_table(rows, ["case", "seed", "algorithm", "seconds", "outer", "inner", "converged", "accuracy"]))
        if a.json:
            with open(a.json, "w") as f:
                json.dump(rows, f, indent=1)
        return
    if a.which == "e1":
        rows = e1_sweep(tuple(int(s) for s in a.sizes.split(",")), a.cases, seeds, device=a.device)
        print(_table(rows, ["n", "case", "algorithm", "seconds", "outer", "converged", "error", "accuracy"]))
    else:
        rows = alpha_sweep(seeds=seeds, device=a.device)
        print(_table(rows, ["alpha", "seed", "seconds", "outer", "converged", "objective", "accuracy"]))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
