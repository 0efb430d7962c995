"""GPU parity of whole solves in the configurations the benchmark runs, and
run-to-run reproducibility, all through the C ABI against the FP64 oracle.

  * Reproducibility: the projection's cross-CTA sums are exact (every
    contribution rounded to a power-of-two quantum before its atomic add), so
    two runs of one solve or batch give bit-identical X, permutations,
    iteration counts and objectives.
  * Precision policy: the X the BF16 or E4M3 phase reached is taken from the
    same solve stopped at the switch (bit-identical to the first lowp_iters
    iterations of the full solve, by the above); the oracle runs the FP32
    refinement from it, replaying the GPU's inner counts: X max-abs 1e-4,
    objective relative 1e-5, permutation bit-exact (Eq. fastPFP, Section 5).
  * n = 4000 (the large workload): one pair held on chip by the wave kernel
    (tensor memory + shared memory), a few outer iterations replayed.
  * n = 1000 free run: the GPU's own stopping decisions against the oracle's
    free run stored in tests/golden/attributed_1000_seed0.json.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1207_1114_gb300 import fastpfp as F
from paper_1207_1114_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def dev_pair(g):
    return (cu(g.A), cu(g.A2), cu(g.B) if g.k else None, cu(g.B2) if g.k else None)


@pytest.fixture(scope="module")
def solver():
    s = F.Solver(max_n=1000, max_batch=40)
    yield s
    s.close()


def _canon(g):
    if g.A.shape[0] >= g.A2.shape[0]:
        return g.A, g.A2, g.B, g.B2, False
    return g.A2, g.A, g.B2, g.B, True


def _greedy_objective(g, Xg, lam):
    """Greedy of Section 4.5 on the GPU's X (oracle, FP64) and Eq. (3) at it."""
    A, A2, Bc, B2c, tr = _canon(g)
    roc = oracle.greedy_sorted((Xg.T if tr else Xg).astype(np.float64))
    K = oracle.affinity(Bc, B2c) if g.k and lam else None
    return roc, oracle.qap_objective(A, A2, roc, K, lam), tr


def _same_bits(a, b):
    """Two runs of one solve: identical permutation, counts, objective and X."""
    np.testing.assert_array_equal(a.perm.cpu().numpy(), b.perm.cpu().numpy())
    for f in ("outer_iters", "inner_iters_total", "inner_iters_max", "lowp_iters", "converged"):
        assert getattr(a.stats, f) == getattr(b.stats, f), f
    assert a.stats.objective == b.stats.objective
    assert a.stats.final_delta == b.stats.final_delta
    assert torch.equal(a.X, b.X)


# ------------------------------------------------------------ reproducibility

@pytest.mark.parametrize("precision", [F.FP32, F.BF16])
def test_lone_pair_is_bit_reproducible(solver, precision):
    g = synth.attributed_1000(seed=0)
    args = dev_pair(g)
    p = F.default_params(lam=1.0, precision=precision, refine_iters=30)
    runs = [solver.match(*args, params=p, want_X=True) for _ in range(2)]
    _same_bits(*runs)
    assert runs[0].stats.wave_pairs == 1   # the wave kernel (a wave of one)


def test_wave_and_streamed_batch_are_bit_reproducible(solver):
    """A single wave (six mixed pairs) and a streamed batch (24 pairs of
    850..1000 nodes, more than one wave holds) run twice."""
    pairs = synth.batch_mixed(count=6, seed=5, n_lo=60, n_hi=400, out_hi=50)
    dev = [dev_pair(g) for g in pairs]
    p = F.default_params(lam=0.5, max_outer=30, max_inner=300)
    a = solver.match_batched(dev, params=p, want_X=True)
    b = solver.match_batched(dev, params=p, want_X=True)
    for x, y in zip(a, b):
        _same_bits(x, y)
    rng = np.random.default_rng(44)
    big = [synth.graph_pair(int(rng.integers(850, 1001)), p=0.1, sigma=0.05, k=8, lam=0.5, seed=800 + i)
           for i in range(24)]
    dev = [dev_pair(g) for g in big]
    p = F.default_params(lam=0.5, max_outer=10, max_inner=60, tol_outer=1e-3)
    a = solver.match_batched(dev, params=p, want_X=True)
    ta = [solver.last_trace(pair=i)[0] for i in range(len(big))]
    assert max(o.stats.wave_pairs for o in a) < len(big)
    b = solver.match_batched(dev, params=p, want_X=True)
    for i, (x, y) in enumerate(zip(a, b)):
        _same_bits(x, y)
        np.testing.assert_array_equal(ta[i], solver.last_trace(pair=i)[0])


def test_projection_is_bit_reproducible(solver):
    """fastpfp_project (the single-pair kernel) twice on the same input."""
    rng = np.random.default_rng(12)
    Y = (rng.random((700, 700)) * 4.0 - 1.0).astype(np.float32)
    outs = []
    for _ in range(2):
        Yg = cu(Y)
        it, d = solver.project(Yg, tol=0.0, max_iter=50)
        outs.append((Yg, it, d))
    assert outs[0][1] == outs[1][1] == 50 and outs[0][2] == outs[1][2]
    assert torch.equal(outs[0][0], outs[1][0])
    ref, _, _ = oracle.pd(Y, fixed_iters=50)
    assert np.abs(outs[0][0].cpu().numpy() - ref).max() <= 2e-5


# ------------------------------------------------------- precision policy

def _switch_x(solver, dev, pair, precision, lowp_iters, lam, **kw):
    """X of pair `pair` when its low-precision phase ended: the same batch
    stopped after lowp_iters outer iterations, with no refinement left, so
    the phase ends exactly there (and not earlier: the other switch rules
    see the same iterates as in the full solve)."""
    p = F.default_params(lam=lam, precision=precision, refine_iters=0, max_outer=lowp_iters, **kw)
    outs = solver.match_batched(dev, params=p, want_X=True)
    inner, _ = solver.last_trace(pair=pair)
    st = outs[pair].stats
    assert st.status == 0 and st.outer_iters == lowp_iters and st.lowp_iters == lowp_iters
    return outs[pair].X.cpu().numpy(), inner


def _check_lowp_batch(solver, pairs, precision, lam, **kw):
    """Every pair of a batched low-precision solve: the oracle's FP32
    refinement from the X at the switch, replaying the GPU's inner counts."""
    dev = [dev_pair(g) for g in pairs]
    p = F.default_params(lam=lam, precision=precision, refine_iters=40, **kw)
    outs = solver.match_batched(dev, params=p, want_X=True)
    # every pair's trace now: the reruns at the switch points replace them
    traces = [solver.last_trace(pair=i)[0] for i in range(len(pairs))]
    errs = []
    for i, (g, o) in enumerate(zip(pairs, outs)):
        inner = traces[i]
        st = o.stats
        L, T = st.lowp_iters, st.outer_iters
        assert st.status == 0 and 1 <= L < T and st.converged == 1
        Xs, inner_s = _switch_x(solver, dev, i, precision, L, lam, **kw)
        np.testing.assert_array_equal(inner_s, inner[:L])
        ref = oracle.solve(g.A, g.A2, g.B, g.B2, lam=lam, X0=Xs, replay_inner=inner[L:],
                           replay_outer=T - L, **kw)
        Xg = o.X.cpu().numpy()
        err = float(np.abs(Xg - ref["X"]).max())
        assert err <= 1e-4, (i, err)
        roc, obj, tr = _greedy_objective(g, Xg, lam)
        perm = o.perm.cpu().numpy()
        if tr:
            np.testing.assert_array_equal(perm, roc)
        else:
            want = -np.ones(g.A.shape[0], dtype=np.int32)
            want[roc] = np.arange(len(roc), dtype=np.int32)
            np.testing.assert_array_equal(perm, want)
        assert abs(st.objective - obj) <= 1e-5 * abs(obj)
        assert abs(st.objective - ref["objective"]) <= 1e-5 * abs(ref["objective"])
        errs.append(err)
    return errs


@pytest.mark.parametrize("precision", [F.BF16, F.FP8])
def test_lowp_phase_then_fp32_refinement_matches_oracle_replay(solver, precision):
    """One n = 1000 attributed pair (the headline workload) with BF16 or E4M3
    products, then the FP32 refinement, against the oracle's refinement from
    the X at the switch."""
    g = synth.attributed_1000(seed=1)
    _check_lowp_batch(solver, [g], precision, 1.0)


@pytest.mark.parametrize("precision", [F.BF16, F.FP8])
def test_lowp_wave_matches_oracle_replay(solver, precision):
    """A wave of four equal-size pairs (n = n': no slack columns carried from
    the low-precision phase) with different switch points."""
    pairs = [synth.graph_pair(n, p=0.15, sigma=0.03, k=8, lam=0.5, seed=90 + n) for n in (150, 220, 300, 260)]
    _check_lowp_batch(solver, pairs, precision, 0.5, max_inner=300)


# ------------------------------------------------------- n = 4000 on chip

def test_large_4000_wave_kernel_matches_oracle():
    """The large workload's launch configuration: one 4000-node pair is a
    wave of one, its 64 MB slacked matrix held on chip (tensor memory plus
    shared memory) for every round.  Two outer iterations of 20 rounds each,
    replayed by the oracle."""
    g = synth.large_4000(seed=0)
    kw = dict(max_outer=2, max_inner=20, tol_inner=0.0)
    with F.Solver(max_n=4000) as s:
        res = s.match(*dev_pair(g), params=F.default_params(lam=0.5, **kw), want_X=True)
        inner, _ = s.last_trace()
    st = res.stats
    assert st.status == 0 and st.outer_iters == 2 and list(inner) == [20, 20]
    assert st.wave_pairs == 1
    ref = oracle.solve(g.A, g.A2, g.B, g.B2, lam=0.5, replay_inner=inner, replay_outer=2, **kw)
    Xg = res.X.cpu().numpy()
    assert np.abs(Xg - ref["X"]).max() <= 1e-4
    roc, obj, _ = _greedy_objective(g, Xg, 0.5)
    np.testing.assert_array_equal(np.argsort(roc), res.perm.cpu().numpy())
    assert abs(st.objective - obj) <= 1e-5 * abs(obj)


# ------------------------------------------------------- n = 1000 free run

def test_attributed_1000_free_run_matches_stored_oracle_solve(solver):
    """The headline pair solved with the GPU's own stopping decisions against
    the oracle's free run (stored by tests/golden/make_golden.py): the same
    permutation, the objective to 1e-5, the outer count within one (the last
    max|dX| sits near eps_1 = 1e-6, where FP32 and FP64 may stop one
    iteration apart), and the same max|dX| trace up to FP32 noise."""
    with open(os.path.join(GOLDEN, "attributed_1000_seed0.json")) as f:
        gold = json.load(f)
    g = synth.attributed_1000(seed=0)
    res = solver.match(*dev_pair(g), params=F.default_params(lam=1.0), want_X=True)
    _, deltas = solver.last_trace()
    st = res.stats
    assert st.status == 0 and st.converged == 1
    np.testing.assert_array_equal(res.perm.cpu().numpy(), np.asarray(gold["perm"], dtype=np.int32))
    assert abs(st.objective - gold["objective"]) <= 1e-5 * abs(gold["objective"])
    assert gold["outer_iters"] <= st.outer_iters <= gold["outer_iters"] + 1
    for t, d in enumerate(gold["delta"][:5]):   # well above the FP32 noise floor
        assert abs(deltas[t] - d) <= 1e-3 * d + 1e-6, (t, deltas[t], d)


# ------------------------------------------- a streamed batch in one graph

def _pairs_24():
    rng = np.random.default_rng(46)
    return [synth.graph_pair(int(rng.integers(850, 1001)), p=0.1, sigma=0.05, k=8, lam=0.5, seed=900 + i)
            for i in range(24)]


def test_graph_streamed_batch_equals_host_streamed_batch(solver):
    """A batch larger than one wave with the graph loop (loop_mode 0) runs as
    one CUDA graph whose planner kernel chooses every wave on the device; with
    loop_mode 1 the host plans the same waves between outer iterations.  The
    two give the same bits, and the graph form synchronises the host once."""
    pairs = _pairs_24()
    dev = [dev_pair(g) for g in pairs]
    kw = dict(lam=0.5, max_outer=12, max_inner=80, tol_outer=1e-3)
    g = solver.match_batched(dev, params=F.default_params(loop_mode=0, **kw), want_X=True)
    tg = [solver.last_trace(pair=i)[0] for i in range(len(pairs))]
    h = solver.match_batched(dev, params=F.default_params(loop_mode=1, **kw), want_X=True)
    assert 0 < max(o.stats.wave_pairs for o in g) < len(pairs)
    assert len({o.stats.outer_iters for o in g}) > 1        # pairs left at different times
    assert all(o.stats.host_syncs == 1 for o in g)
    assert all(o.stats.host_syncs > 1 for o in h)
    for i, (a, b) in enumerate(zip(g, h)):
        _same_bits(a, b)
        assert a.stats.wave_pairs == b.stats.wave_pairs
        np.testing.assert_array_equal(tg[i], solver.last_trace(pair=i)[0])


def test_graph_streamed_batch_matches_oracle(solver):
    """Every pair of the graph-streamed batch against the oracle replaying
    its own inner counts (X max-abs 1e-4, greedy bit-exact, objective)."""
    pairs = _pairs_24()
    dev = [dev_pair(g) for g in pairs]
    kw = dict(max_outer=12, max_inner=80, tol_outer=1e-3)
    outs = solver.match_batched(dev, params=F.default_params(lam=0.5, **kw), want_X=True)
    for i, (g, o) in enumerate(zip(pairs, outs)):
        inner, _ = solver.last_trace(pair=i)
        assert o.stats.status == 0 and len(inner) == o.stats.outer_iters
        ref = oracle.solve(g.A, g.A2, g.B, g.B2, lam=0.5, replay_inner=inner,
                           replay_outer=o.stats.outer_iters, **kw)
        Xg = o.X.cpu().numpy()
        assert np.abs(Xg - ref["X"]).max() <= 1e-4
        roc, obj, _ = _greedy_objective(g, Xg, 0.5)
        np.testing.assert_array_equal(np.argsort(roc), o.perm.cpu().numpy())
        assert abs(o.stats.objective - obj) <= 1e-5 * abs(obj)


def test_graph_streamed_bf16_batch_of_uneven_pairs(solver):
    """A mixed batch of 40 uneven pairs (outliers on either side) with the
    BF16 phase, streamed in one graph: identical to the host-planned stream,
    and every pair ends at the plain FP32 solve's objective."""
    pairs = synth.batch_mixed(count=40, seed=47, n_lo=300, n_hi=900, out_hi=100)
    dev = [dev_pair(g) for g in pairs]
    kw = dict(lam=0.5, precision=F.BF16, refine_iters=30, max_inner=200)
    g = solver.match_batched(dev, params=F.default_params(loop_mode=0, **kw), want_X=True)
    h = solver.match_batched(dev, params=F.default_params(loop_mode=1, **kw), want_X=True)
    assert max(o.stats.wave_pairs for o in g) < len(pairs) and g[0].stats.host_syncs == 1
    p32 = solver.match_batched(dev, params=F.default_params(lam=0.5, max_inner=200))
    for a, b, c in zip(g, h, p32):
        _same_bits(a, b)
        assert a.stats.status == 0 and a.stats.lowp_iters >= 1
        assert abs(a.stats.objective - c.stats.objective) <= 1e-4 * abs(c.stats.objective)


def test_fp32_products_on_tensor_cores_match_the_simt_solve(solver):
    """The FP32 solve with its products on the tensor cores (split TF32)
    and on the FMA pipes: the same permutation, iteration counts within one
    and X within 1e-5 when the counts agree; each against the oracle's
    replay of its own counts."""
    g = synth.attributed_1000(seed=3)
    args = dev_pair(g)
    outs = {}
    for prec in (F.FP32, F.FP32_SIMT):
        r = solver.match(*args, params=F.default_params(lam=1.0, precision=prec), want_X=True)
        inner, _ = solver.last_trace()
        ref = oracle.solve(g.A, g.A2, g.B, g.B2, lam=1.0, replay_inner=inner, replay_outer=r.stats.outer_iters)
        assert r.stats.status == 0 and np.abs(r.X.cpu().numpy() - ref["X"]).max() <= 1e-4
        outs[prec] = r
    a, b = outs[F.FP32], outs[F.FP32_SIMT]
    np.testing.assert_array_equal(a.perm.cpu().numpy(), b.perm.cpu().numpy())
    assert abs(a.stats.outer_iters - b.stats.outer_iters) <= 1 and a.stats.lowp_iters == 0
    if a.stats.outer_iters == b.stats.outer_iters:
        assert (a.X - b.X).abs().max().item() <= 1e-5


# ------------------------------------------- the outer stop's max|dX| exactly
def _tiny_start(n, seed):
    """A start whose entries sit ~2^-40 below the iterate's: every change
    |X(1) - X(0)| then needs more than FP64's 53 bits, so its FP64 rounding
    (the oracle's max|dX|) differs from a rounding through FP32."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(1.0, 2.0, (n, n)) * 2.0 ** -40).astype(np.float32)


def _exact_delta(X1, X0):
    return float(np.abs(X1.astype(np.float64) - X0.astype(np.float64)).max())


@pytest.mark.parametrize("algorithm", [F.ALG_FASTPFP, F.ALG_FASTGA])
def test_outer_delta_is_the_fp64_max_change_in_a_wave(solver, algorithm):
    """max|dX| of Algorithm 1's outer stop, taken per element in FP32 (exact
    TwoSum pairs) and rounded to FP64 once, equals the FP64 maximum of the
    changes of X the solve returns, bit for bit; wave kernel (three pairs in
    one wave) and FastGA's kernel."""
    gs = [synth.graph_pair(n, p=0.2, sigma=0.02, k=0, seed=40 + n) for n in (90, 150, 61)]
    X0s = [_tiny_start(g.n, g.n) for g in gs]
    prm = F.default_params(algorithm=algorithm, beta=100.0, max_outer=1, max_inner=30)
    res = solver.match_batched([dev_pair(g)[:2] + (None, None, cu(X0)) for g, X0 in zip(gs, X0s)],
                               params=prm, want_X=True)
    for i, (r, X0) in enumerate(zip(res, X0s)):
        _, deltas = solver.last_trace(pair=i)
        want = _exact_delta(r.X.cpu().numpy(), X0)
        assert float(np.float32(want)) != want   # the case needs the exact low part
        assert deltas[0] == want, (i, deltas[0], want)


def test_outer_delta_is_the_fp64_max_change_alone():
    """The same bit-exact max|dX| from pd_kernel, which runs a pair too wide
    for any wave (N > 4096) alone."""
    n = 4100
    g = synth.graph_pair(n, p=0.01, sigma=0.0, k=0, seed=2)
    X0 = _tiny_start(n, 5)
    with F.Solver(max_n=n) as s:
        r = s.match(cu(g.A), cu(g.A2), X0=cu(X0), params=F.default_params(max_outer=1, max_inner=10),
                    want_X=True)
        _, deltas = s.last_trace()
    assert r.stats.wave_pairs == 0
    want = _exact_delta(r.X.cpu().numpy(), X0)
    assert float(np.float32(want)) != want
    assert deltas[0] == want
