"""The N > 1 host logic on CPU: gloo process groups of world size 2.

Independent pairs shard across ranks with no exchange on the data path
(paper_1207_1114_gb300/shard.py); the only collectives are the final gather
of results and, in bench.py, the barrier and the max over ranks of the timed
region.  Here each rank "solves" its share with the FP64 oracle (a stand-in
for the GPU solver; the sharding logic does not care which solver runs)."""
import itertools
import os
import pickle
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1207_1114_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Out:
    def __init__(self, perm, stats):
        self.perm = perm
        self.stats = stats


def _oracle_solver(pairs):
    outs = []
    for g in pairs:
        r = oracle.solve(g.A, g.A2, g.B if g.k else None, g.B2 if g.k else None, lam=g.lam,
                         max_outer=10, max_inner=60)
        outs.append(_Out(np.asarray(r["perm"], dtype=np.int32),
                         {"outer_iters": int(r["outer_iters"])}))
    return outs


def _pairs():
    return synth.batch_mixed(count=7, seed=5, n_lo=6, n_hi=18, out_hi=4)


def _worker(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ.setdefault("GLOO_SOCKET_IFNAME", "lo")   # the host name need not resolve
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_num_threads(1)   # two processes share the cores; tiny problems
    try:
        pairs = _pairs()
        shapes = [(g.A.shape[0], g.A2.shape[0]) for g in pairs]
        res = shard.solve_sharded(_oracle_solver, pairs, shapes, rank, world,
                                  gather=shard.torch_gather)
        import bench
        dev = torch.device("cpu")
        out = {"shard": [(r.index, r.rank, r.perm.tolist(), r.stats) for r in res],
               "timing": (bench.max_over_ranks(1.5 + rank, dev),
                          bench.whole_job_rate(10, 2.0 + 2.0 * rank, dev))}
        with open(os.path.join(outdir, f"r{rank}.pkl"), "wb") as f:
            pickle.dump(out, f)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks():
    """Both ranks' results of one world-size-2 gloo run."""
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        res = []
        for r in range(world):
            with open(os.path.join(d, f"r{r}.pkl"), "rb") as f:
                res.append(pickle.load(f))
    return res


def test_partition_covers_every_pair_once_and_is_deterministic():
    rng = np.random.default_rng(0)
    costs = rng.uniform(1, 100, 37)
    for world in (1, 2, 3, 8, 50):
        sh = shard.partition(costs, world)
        assert len(sh) == world
        assert sorted(i for s in sh for i in s) == list(range(len(costs)))
        assert sh == shard.partition(costs, world)


@pytest.mark.parametrize("world", [2, 3])
def test_partition_meets_the_lpt_bound(world):
    """Graham's bound for longest-processing-time scheduling: the makespan is
    at most (4/3 - 1/(3 w)) times the optimum, here found by brute force."""
    rng = np.random.default_rng(world)
    for _ in range(20):
        costs = rng.uniform(1, 10, 8)
        sh = shard.partition(costs, world)
        lpt = max(sum(costs[i] for i in s) for s in sh)
        opt = min(max(sum(c for c, a in zip(costs, assign) if a == r) for r in range(world))
                  for assign in itertools.product(range(world), repeat=len(costs)))
        assert lpt <= (4 / 3 - 1 / (3 * world)) * opt + 1e-9


def test_pair_cost_grows_with_size_and_is_orientation_free():
    assert shard.pair_cost(100, 120) == shard.pair_cost(120, 100)
    assert shard.pair_cost(50, 50) < shard.pair_cost(60, 50) < shard.pair_cost(60, 60)


def test_sharded_solve_over_two_gloo_ranks_equals_one_process(two_ranks):
    one = shard.solve_sharded(_oracle_solver, _pairs(),
                              [(g.A.shape[0], g.A2.shape[0]) for g in _pairs()], 0, 1)
    res = [r["shard"] for r in two_ranks]
    assert res[0] == res[1]                         # every rank holds every result
    ranks = {r[1] for r in res[0]}
    assert ranks == {0, 1}                          # both ranks did work
    for (idx, _, perm, stats), ref in zip(res[0], one):
        assert idx == ref.index
        assert perm == ref.perm.tolist()
        assert stats == ref.stats


def test_bench_timing_takes_the_slowest_rank(two_ranks):
    for mx, rate in (r["timing"] for r in two_ranks):
        assert mx == 2.5
        assert rate == pytest.approx(10 * 2 / 4.0)


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched as the driver launches it for N > 1
    (torchrun, two ranks): rank 0 alone times the oracle and prints one JSON
    line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert "nothing extrapolated" in line["cpu_baseline"]["sample"]
    assert line["ms_per_step"] == pytest.approx(1e3 / line["value"])
    assert line["e2e"]["h2d_bytes_per_step"] == 0
