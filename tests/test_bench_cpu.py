"""Host-side pieces of bench.py: the parameters each mode passes to the
library, the kernel-code hash behind the ncu traffic field, and the oracle
baseline's unit costs.  CPU only."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1207_1114_gb300 import fastpfp as F  # noqa: E402
from paper_1207_1114_gb300 import synth  # noqa: E402


def test_code_hash_ignores_comments_but_not_code():
    a = "int f(int x) { // double it\n  return 2 * x; /* fast */ }\n"
    b = "int f(int x) {\n  return 2 * x;\n}\n// another note\n"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_hash(a) == bench.code_hash(b)
    assert bench.code_hash(a) != bench.code_hash(c)
    # a comment marker inside a string literal is code
    assert bench.code_hash('const char* s = "//x";') != bench.code_hash('const char* s = "";')


def test_profile_traffic_needs_a_matching_code_hash(tmp_path, monkeypatch):
    """The traffic field is read from a summary only while its recorded hash
    is the kernel's current code hash (and the round count matches)."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.source_hash("pdb_kernel")
    (prof / "pdb_kernel_attributed_1000.md").write_text(
        f"source_sha256_16: {h}\ndram_bytes_per_launch: 1234\nrounds_per_launch: 1000\n")
    (prof / "pdb_kernel_large_4000.md").write_text(
        "source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 1234\nrounds_per_launch: 1000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic_per_launch("pdb_kernel", "attributed_1000", 1000) == 1234
    assert bench.ncu_traffic_per_launch("pdb_kernel", "attributed_1000", 500) is None
    assert bench.ncu_traffic_per_launch("pdb_kernel", "large_4000", 1000) is None


def test_params_per_mode():
    p = bench.params(F, 1.0)
    assert p.precision == F.FP32 and p.algorithm == F.ALG_FASTPFP and p.alpha == 0.5
    p = bench.params(F, 1.0, precision="fp8")
    assert p.precision == F.FP8 and p.refine_iters == 30 and p.switch_tol == 1e-3
    p = bench.params(F, 1.0, pg_alpha=0.01)
    assert p.algorithm == F.ALG_PG and p.normalize_max == 0 and abs(p.alpha - 0.01) < 1e-9


def test_params_override_and_switch_point():
    """The parameters of the X-at-the-switch rerun: the same mode with no
    refinement and I_0 cut to the low-precision iteration count."""
    p = bench.params(F, 1.0, precision="bf16", refine_iters=0, max_outer=7)
    assert p.precision == F.BF16 and p.refine_iters == 0 and p.max_outer == 7
    assert p.switch_tol == 1e-3 and p.max_inner == 1000


def test_oracle_timed_solves_are_whole_solves():
    """The cpu_baseline's oracle timing: whole solves, at least one pair, in
    order, stopping once the budget is spent."""
    pairs = [synth.graph_pair(20, p=0.3, sigma=0.02, k=2, lam=0.5, seed=s) for s in range(3)]
    done, spent = bench.oracle_timed_solves(pairs, 0.0)
    assert done == 1 and spent > 0
    done, spent = bench.oracle_timed_solves(pairs, 1e9)
    assert done == 3
    kw = bench.oracle_solve_kwargs(0.5, pg_alpha=0.1)
    assert kw["algorithm"] == "pg" and kw["alpha"] == 0.1 and kw["normalize_max"] is False


def test_rank_shares_split_the_job_by_cost():
    """Under torchrun every rank takes its share of the whole job's
    world x batch pairs from shard.partition: the shares are disjoint and
    complete, equal-size pairs split evenly, and one rank's share is the
    job's first pairs (the same pairs as before the split existed)."""
    world, batch = 2, 6
    shapes = bench.global_shapes("batch_mixed_512", world * batch)
    shares = [bench.rank_share("batch_mixed_512", r, world, batch)[0] for r in range(world)]
    assert sorted(shares[0] + shares[1]) == list(range(world * batch))
    from paper_1207_1114_gb300 import shard
    cost = [sum(shard.pair_cost(*shapes[i]) for i in sh) for sh in shares]
    assert max(cost) <= 1.5 * min(cost)
    idx, pairs = bench.rank_share("batch_mixed_512", 1, world, batch)
    for i, g in zip(idx, pairs):
        assert (g.A.shape[0], g.A2.shape[0]) == shapes[i]
    eq = [bench.rank_share("attributed_1000", r, 2, 2)[0] for r in range(2)]
    assert sorted(eq[0] + eq[1]) == [0, 1, 2, 3] and len(eq[0]) == len(eq[1]) == 2
    assert bench.rank_share("attributed_1000", 0, 1, 3)[0] == [0, 1, 2]


def test_pg_step_is_one_over_the_lipschitz_constant():
    g = synth.graph_pair(30, p=0.3, sigma=0.0, seed=1)
    L = np.linalg.norm(g.A.astype(np.float64), 2) * np.linalg.norm(g.A2.astype(np.float64), 2)
    assert bench.pg_step([g]) == pytest.approx(1.0 / L, rel=1e-6)


def test_single_thread_oracle_units_are_positive():
    g = synth.graph_pair(40, p=0.3, sigma=0.02, k=2, seed=2)
    u = bench.oracle_single_thread_units(g, rounds=2)
    assert all(v > 0 for v in u.values())
    assert isinstance(bench.cpu_model(), str)
