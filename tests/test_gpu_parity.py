"""GPU parity: every CUDA step and the whole solve against the FP64 oracle,
called through the C ABI (libfastpfp.so) on the same seeded inputs.

Tolerances (FP32 kernels against the FP64 oracle):
  * gradient entries: |err| <= 1e-5 * (|A| |X| |A'| + lambda |K|) entrywise, the
    FP32 dot-product bound for sums of <= ~1e4 terms;
  * P_D after a replayed number of rounds: max-abs 2e-5 (entries of order 1);
  * final X of a replayed solve: max-abs 1e-4; objective relative 1e-5;
  * discretisation: bit-exact (both sides compare the same FP32 values).
"""
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


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


@pytest.fixture(scope="module")
def solver():
    s = F.Solver(max_n=1200, max_batch=8)
    yield s
    s.close()


def _canon(g):
    """Canonical orientation: larger graph on the rows."""
    if g.A.shape[0] >= g.A2.shape[0]:
        return g.A, g.A2, g.B, g.B2, False
    return g.A2, g.A, g.B2, g.B, True


# --------------------------------------------------------------- single steps

@pytest.mark.parametrize("N,m,k", [(1, 1, 1), (7, 5, 3), (130, 97, 16), (1000, 1000, 16)])
def test_affinity_matches_oracle(solver, N, m, k):
    rng = np.random.default_rng(N + m)
    B = rng.normal(size=(N, k)).astype(np.float32)
    B2 = rng.normal(size=(m, k)).astype(np.float32)
    K = solver.affinity(cu(B), cu(B2)).cpu().numpy()
    ref = oracle.affinity(B, B2)
    bound = np.abs(B).astype(np.float64) @ np.abs(B2).astype(np.float64).T
    assert (np.abs(K - ref) <= 1e-6 * bound + 1e-30).all()


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
@pytest.mark.parametrize("N,m", [(1, 1), (5, 3), (129, 100), (300, 300), (1200, 1000)])
def test_gradient_matches_oracle(solver, N, m, precision):
    """The FP32 products, on the tensor cores (split TF32) and on the FMA
    pipes, against the oracle.

    FMA pipes: round-to-nearest FP32 sums, well inside 1e-5 * |A||X||A'|.
    Split TF32: each product term loses at most 3 * 2^-22 of itself (the
    dropped lo*lo and the remainders read as TF32), and each tcgen05.mma's
    addition into its FP32 accumulator may drop up to one unit in the last
    place of the running sum (2^-23 of it, at most the bound) -- one such
    addition per 8 terms of K, ceil(N / 8) in A*X and ceil(m / 8) in T*A'.
    The correction terms accumulate apart (2^-11 smaller), so
    |err| <= ((ceil(N/8) + ceil(m/8)) * 2^-23 + 6 * 2^-22 + 2^-23) * bound."""
    rng = np.random.default_rng(N * 3 + m)
    A = synth.random_graph(rng, N, 0.2).astype(np.float32)
    A2 = synth.random_graph(rng, m, 0.2).astype(np.float32)
    X = rng.random((N, m)).astype(np.float32)
    K = rng.normal(size=(N, m)).astype(np.float32)
    lam = 0.7
    prec = F.FP32 if precision == "fp32" else F.FP32_SIMT
    G = solver.gradient(cu(A), cu(X), cu(A2), cu(K), lam, precision=prec).cpu().numpy()
    ref = oracle.gradient(A, X, A2, K, lam)
    bound = np.abs(A) @ np.abs(X).astype(np.float64) @ np.abs(A2) + lam * np.abs(K)
    if precision == "fp32":
        tol = (-(-N // 8) - (-m // 8)) * 2.0**-23 + 6 * 2.0**-22 + 2.0**-23
    else:
        tol = 1e-5
    err = np.abs(G - ref) / (bound + 1e-30)
    assert err.max() <= tol, (err.max(), tol, float(np.mean((G - ref) / (bound + 1e-30))))


def _bf16(a):
    """Round to bfloat16 (nearest even) and back, as the tensor-core path does."""
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("N,m", [(5, 3), (129, 100), (300, 300), (1000, 1000), (1200, 1000)])
def test_gradient_bf16_tensor_cores_matches_oracle(solver, N, m):
    """tcgen05 BF16 products: A, X, A' and T are rounded to BF16 (unit roundoff
    2^-9), accumulation is FP32.  Against the oracle on the same BF16-rounded
    operands only T's rounding remains: |err| <= 3e-3 * |A||X||A'| (+ the FP32
    term); against the unrounded oracle four roundings: 1e-2 * the bound."""
    rng = np.random.default_rng(N * 5 + m)
    A = synth.random_graph(rng, N, 0.2).astype(np.float32)
    A2 = synth.random_graph(rng, m, 0.2).astype(np.float32)
    X = rng.random((N, m)).astype(np.float32)
    K = rng.normal(size=(N, m)).astype(np.float32)
    lam = 0.7
    G = solver.gradient(cu(A), cu(X), cu(A2), cu(K), lam, precision=F.BF16).cpu().numpy()
    bound = np.abs(A) @ np.abs(X).astype(np.float64) @ np.abs(A2) + lam * np.abs(K)
    ref = oracle.gradient(A, X, A2, K, lam)
    assert (np.abs(G - ref) <= 1e-2 * bound + 1e-30).all()
    ref16 = oracle.gradient(_bf16(A), _bf16(X), _bf16(A2), K, lam)
    assert (np.abs(G - ref16) <= 3e-3 * bound + 1e-30).all()


@pytest.mark.parametrize("N", [1, 2, 3, 7, 64, 100, 129, 333, 1000, 1200])
def test_projection_matches_oracle_fixed_rounds(solver, N):
    rng = np.random.default_rng(N)
    Y = (rng.random((N, N)) * 5.0).astype(np.float32)
    Yg = cu(Y)
    it, _ = solver.project(Yg, tol=0.0, max_iter=40)
    assert it == 40
    ref, _, _ = oracle.pd(Y, fixed_iters=40)
    assert np.abs(Yg.cpu().numpy() - ref).max() <= 2e-5
    assert (Yg.cpu().numpy() >= 0).all()


@pytest.mark.parametrize("N", [50, 257, 1000])
def test_projection_tolerance_stop_replays(solver, N):
    rng = np.random.default_rng(7 * N)
    Y = (rng.random((N, N)) * rng.random((N, 1)) * 20).astype(np.float32)
    Yg = cu(Y)
    it, d = solver.project(Yg, tol=1e-5, max_iter=2000)
    assert 1 <= it <= 2000
    assert it == 2000 or d < 1e-5
    ref, _, _ = oracle.pd(Y, fixed_iters=it)
    assert np.abs(Yg.cpu().numpy() - ref).max() <= 2e-5


def test_projection_streamed_band_large_n():
    """N = 4000: a CTA's band no longer fits in shared memory, the kernel
    streams it from global memory."""
    with F.Solver(max_n=4000) as s:
        rng = np.random.default_rng(4000)
        Y = (rng.random((4000, 4000)) * 3.0).astype(np.float32)
        Yg = cu(Y)
        it, _ = s.project(Yg, tol=0.0, max_iter=6)
        assert it == 6
        ref, _, _ = oracle.pd(Y, fixed_iters=6)
        assert np.abs(Yg.cpu().numpy() - ref).max() <= 2e-5


@pytest.mark.parametrize("shape", [(1, 1), (2, 1), (9, 9), (100, 37), (257, 256), (1200, 1000)])
@pytest.mark.parametrize("levels", [0, 4])
def test_discretize_bit_exact(solver, shape, levels):
    rng = np.random.default_rng(shape[0] * 11 + shape[1] + levels)
    X = rng.random(shape).astype(np.float32)
    if levels:
        X = (np.floor(X * levels) / levels).astype(np.float32)   # heavy ties
    got = solver.discretize(cu(X)).cpu().numpy()
    ref = oracle.greedy_sorted(X.astype(np.float64))
    np.testing.assert_array_equal(got, ref)


# ---------------------------------------------------------------- whole solve

def _check_against_replay(g, res, solver, lam, **kw):
    """X of the GPU solve against the oracle replaying the GPU's iteration counts."""
    inner, _ = solver.last_trace()
    st = res.stats
    assert st.status == 0 and len(inner) == st.outer_iters
    r = oracle.solve(g.A, g.A2, g.B, g.B2, lam=lam, replay_inner=inner,
                     replay_outer=st.outer_iters, **kw)
    Xg = res.X.cpu().numpy()
    assert np.abs(Xg - r["X"]).max() <= 1e-4
    # discretisation of the GPU's X is bit-exact with the oracle's greedy
    A, A2, _, _, tr = _canon(g)
    Xc = Xg.T if tr else Xg
    roc = oracle.greedy_sorted(Xc.astype(np.float64))
    perm = res.perm.cpu().numpy()
    if tr:
        np.testing.assert_array_equal(perm, roc)
    else:
        want = -np.ones(A.shape[0], dtype=np.int32)
        want[roc] = np.arange(len(roc), dtype=np.int32)
        np.testing.assert_array_equal(perm, want)
    # objective (Eq. 3) of the GPU's permutation, FP64 on both sides
    Bc, B2c = (g.B2, g.B) if tr else (g.B, g.B2)
    K = oracle.affinity(Bc, B2c) if g.k and lam else None
    obj = oracle.qap_objective(A, A2, roc, K, lam)
    assert abs(st.objective - obj) <= 1e-5 * abs(obj)
    return r


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plain_100_matches_oracle(solver, seed):
    g = synth.plain_100(seed)
    res = solver.match(cu(g.A), cu(g.A2), params=F.default_params(), want_X=True)
    _check_against_replay(g, res, solver, 0.0)
    assert (res.perm.cpu().numpy() == g.gt).mean() >= 0.99


@pytest.mark.parametrize("n_a,n_b", [(60, 75), (75, 60), (17, 13), (13, 17), (1, 1), (2, 1),
                                     (1, 3)])
def test_partial_and_transposed_match_oracle(solver, n_a, n_b):
    n, n_out = min(n_a, n_b), abs(n_a - n_b)
    g = synth.graph_pair(n, p=0.3, sigma=0.03, k=4, n_out=n_out, lam=0.5, seed=n_a * 100 + n_b)
    if n_a > n_b:   # graph 1 is the larger one
        g = synth.GraphPair(g.A2, g.A, g.B2, g.B, np.argsort(g.gt).astype(np.int32)[:n], g.lam)
    p = F.default_params(lam=0.5, max_outer=30, max_inner=300)
    res = solver.match(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2), params=p, want_X=True)
    assert res.stats.transposed == int(n_a < n_b)
    _check_against_replay(g, res, solver, 0.5, max_outer=30, max_inner=300)


def test_slack_reset_policy_matches_oracle(solver):
    g = synth.graph_pair(40, p=0.3, sigma=0.03, k=3, n_out=12, lam=0.5, seed=9)
    p = F.default_params(lam=0.5, max_outer=20, max_inner=200, slack_policy=1)
    res = solver.match(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2), params=p, want_X=True)
    _check_against_replay(g, res, solver, 0.5, max_outer=20, max_inner=200, slack_policy=1)


def test_no_normalisation_matches_oracle(solver):
    g = synth.graph_pair(50, p=0.3, sigma=0.02, seed=10)
    p = F.default_params(max_outer=15, max_inner=200, normalize_max=0)
    res = solver.match(cu(g.A), cu(g.A2), params=p, want_X=True)
    _check_against_replay(g, res, solver, 0.0, max_outer=15, max_inner=200, normalize_max=False)


def test_warm_start_x0_matches_oracle(solver):
    g = synth.graph_pair(64, p=0.3, sigma=0.02, n_out=8, seed=11)
    rng = np.random.default_rng(0)
    X0 = rng.random((g.n, g.n2)).astype(np.float32)
    p = F.default_params(max_outer=20, max_inner=200)
    res = solver.match(cu(g.A), cu(g.A2), params=p, X0=cu(X0), want_X=True)
    _check_against_replay(g, res, solver, 0.0, max_outer=20, max_inner=200, X0=X0)


def _same_solve(a, b, Xa, Xb):
    """Two runs of one solve (different entry points or loop control) give
    the same bits: the projection's cross-CTA sums are exact, so the order in
    which the atomics land does not matter.  Same permutation, iteration
    counts, objective and X."""
    np.testing.assert_array_equal(a.perm.cpu().numpy() if hasattr(a.perm, "cpu") else a.perm,
                                  b.perm.cpu().numpy() if hasattr(b.perm, "cpu") else b.perm)
    assert a.stats.objective == b.stats.objective
    assert a.stats.outer_iters == b.stats.outer_iters
    assert a.stats.inner_iters_total == b.stats.inner_iters_total
    assert a.stats.lowp_iters == b.stats.lowp_iters
    np.testing.assert_array_equal(np.asarray(Xa), np.asarray(Xb))


def test_host_entry_point_equals_device_entry_point(solver):
    g = synth.graph_pair(90, p=0.2, sigma=0.03, k=5, n_out=10, lam=0.5, seed=12)
    p = F.default_params(lam=0.5, max_outer=25, max_inner=300)
    d = solver.match(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2), params=p, want_X=True)
    h = solver.match_host(g.A, g.A2, g.B, g.B2, params=p, want_X=True)
    _same_solve(d, h, d.X.cpu().numpy(), h.X)


def test_batched_host_entry_point_equals_device_batch(solver):
    """fastpfp_match_batched_host stages every wave from host memory; it must
    give what fastpfp_match_batched gives on device copies of the same pairs."""
    pairs = synth.batch_mixed(count=6, seed=21, n_lo=40, n_hi=200, out_hi=30)
    p = F.default_params(lam=0.5, max_outer=25, max_inner=250)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    d = solver.match_batched(dev, params=p, want_X=True)
    h = solver.match_batched_host([(g.A, g.A2, g.B, g.B2) for g in pairs], params=p, want_X=True)
    for a, b in zip(d, h):
        _same_solve(a, b, a.X.cpu().numpy(), b.X)


@pytest.mark.parametrize("count", [3, 24])
def test_pinned_host_inputs_gathered_by_one_kernel_equal_device_batch(count):
    """Pinned host inputs are read in place by one gather kernel (pageable
    ones are copied as before); a batch mixing both — one wave (3 pairs) and
    a streamed batch (24 pairs, the graph path) — gives what the device entry
    point gives on the same pairs, bit for bit, including odd sizes whose
    byte counts are not multiples of 16."""
    pairs = synth.batch_mixed(count=count, seed=31 + count, n_lo=41, n_hi=333, out_hi=17)
    p = F.default_params(lam=0.5, max_outer=12, max_inner=200)
    solver = F.Solver(max_n=350, max_batch=count)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    d = solver.match_batched(dev, params=p, want_X=True)
    host = []
    for i, g in enumerate(pairs):
        arrs = (g.A, g.A2, g.B, g.B2)
        if i % 3 != 2:   # two of every three pairs pinned, the third pageable
            arrs = tuple(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).pin_memory() for a in arrs)
        host.append(arrs)
    h = solver.match_batched_host(host, params=p, want_X=True)
    solver.close()
    for a, b in zip(d, h):
        _same_solve(a, b, a.X.cpu().numpy(), b.X)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_graph_loop_equals_host_loop_single(solver, precision):
    """Algorithm 1's repeat loop as a CUDA-graph while node (loop_mode 0)
    and as host-polled chunks (loop_mode 1) run the same kernels: the same
    solve up to FP32 reduction order (_same_solve)."""
    g = synth.graph_pair(300, p=0.1, sigma=0.03, k=8, n_out=20, lam=0.5, seed=31)
    prec = F.BF16 if precision == "bf16" else F.FP32
    args = (cu(g.A), cu(g.A2), cu(g.B), cu(g.B2))
    out = []
    for mode in (0, 1):
        p = F.default_params(lam=0.5, loop_mode=mode, precision=prec, refine_iters=10)
        out.append(solver.match(*args, params=p, want_X=True))
    a, b = out
    _same_solve(a, b, a.X.cpu().numpy(), b.X.cpu().numpy())
    # the graph loop adds one condition kernel per iteration but runs no
    # product or projection launch after the stop; the host loop may
    assert 0 < a.stats.launches <= b.stats.launches + a.stats.outer_iters + 1


def test_graph_loop_equals_host_loop_batched(solver):
    pairs = synth.batch_mixed(count=8, seed=32, n_lo=30, n_hi=250, out_hi=40)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    res = [solver.match_batched(dev, params=F.default_params(lam=0.5, loop_mode=mode), want_X=True)
           for mode in (0, 1)]
    for a, b in zip(*res):
        _same_solve(a, b, a.X.cpu().numpy(), b.X.cpu().numpy())


@pytest.mark.parametrize("max_outer", [1, 2, 5])
def test_graph_loop_stops_at_the_outer_cap(solver, max_outer):
    """The while node ends after exactly I_0 iterations when X has not
    converged (a normal stop: converged = 0)."""
    g = synth.plain_100(1)
    for batched in (False, True):
        p = F.default_params(max_outer=max_outer, loop_mode=0)
        if batched:
            outs = solver.match_batched([(cu(g.A), cu(g.A2), None, None)] * 2, params=p)
        else:
            outs = [solver.match(cu(g.A), cu(g.A2), params=p)]
        for o in outs:
            assert o.stats.outer_iters == max_outer and o.stats.converged == 0
            assert o.stats.status == 0


def _check_batch(solver, pairs, lam, **kw):
    """Every pair of one wave against the oracle replaying that pair's trace."""
    p = F.default_params(lam=lam, **kw)
    dev = [(cu(g.A), cu(g.A2), cu(g.B) if g.k else None, cu(g.B2) if g.k else None) for g in pairs]
    outs = solver.match_batched(dev, params=p, want_X=True)
    for i, (g, o) in enumerate(zip(pairs, outs)):
        inner, _ = solver.last_trace(pair=i)
        assert o.stats.status == 0 and len(inner) == o.stats.outer_iters
        r = oracle.solve(g.A, g.A2, g.B, g.B2, lam=lam, replay_inner=inner,
                         replay_outer=o.stats.outer_iters, **kw)
        Xg = o.X.cpu().numpy()
        assert np.abs(Xg - r["X"]).max() <= 1e-4
        A, A2, Bc, B2c, tr = _canon(g)
        roc = oracle.greedy_sorted((Xg.T if tr else Xg).astype(np.float64))
        K = oracle.affinity(Bc, B2c) if g.k and lam else None
        obj = oracle.qap_objective(A, A2, roc, K, lam)
        assert abs(o.stats.objective - obj) <= 1e-5 * abs(obj)
    return outs


def test_batched_wave_of_uneven_pairs_matches_oracle(solver):
    """Six pairs of uneven sizes (outliers on either side) share one wave."""
    pairs = synth.batch_mixed(count=6, seed=3, n_lo=20, n_hi=160, out_hi=25)
    pairs[1] = synth.GraphPair(pairs[1].A2, pairs[1].A, pairs[1].B2, pairs[1].B, pairs[1].gt, 0.5)
    _check_batch(solver, pairs, 0.5, max_outer=25, max_inner=250)


def test_batched_wave_at_full_size_matches_oracle(solver):
    """Three n = 1000 attributed pairs in one wave, a few outer iterations."""
    pairs = [synth.attributed_1000(seed=s) for s in range(3)]
    _check_batch(solver, pairs, 1.0, max_outer=3, max_inner=150)


def test_batched_wave_with_two_quads_per_thread_matches_oracle(solver):
    """1000-into-1200 pairs: a 1200-wide row is covered by three row groups
    of 160 threads with two column quads each (TMEM rows of eight columns)."""
    pairs = [synth.partial_1000_1200(seed=s) for s in range(3)]
    _check_batch(solver, pairs, 0.5, max_outer=3, max_inner=100)


def test_batched_wave_of_wide_rows_matches_oracle(stream_solver_wide):
    """Rows of 2100 nodes: one row group of 288 threads with two quads each."""
    pairs = [synth.graph_pair(2100, p=0.05, sigma=0.05, k=8, lam=0.5, seed=70 + s) for s in range(2)]
    outs = _check_batch(stream_solver_wide, pairs, 0.5, max_outer=2, max_inner=30)
    assert all(o.stats.wave_pairs == 2 for o in outs)


@pytest.fixture(scope="module")
def stream_solver_wide():
    s = F.Solver(max_n=2100, max_batch=2)
    yield s
    s.close()


def test_bf16_phase_then_fp32_refinement(solver):
    """Precision policy: BF16 tensor-core products until max|dX| < switch_tol,
    then FP32 iterations.  The refined result matches the plain FP32 solve's
    permutation and objective, and its X the plain solve's to 1e-3 (the
    oracle replay of the refinement is in test_gpu_solve_parity.py)."""
    g = synth.attributed_1000(seed=1)
    A, A2, B, B2 = cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)
    p32 = F.default_params(lam=1.0)
    r32 = solver.match(A, A2, B, B2, params=p32, want_X=True)
    p16 = F.default_params(lam=1.0, precision=F.BF16, refine_iters=30, switch_tol=1e-3)
    r16 = solver.match(A, A2, B, B2, params=p16, want_X=True)
    st = r16.stats
    assert st.status == 0 and st.lowp_iters >= 1 and st.outer_iters > st.lowp_iters
    assert st.converged == 1
    np.testing.assert_array_equal(r16.perm.cpu().numpy(), r32.perm.cpu().numpy())
    assert abs(st.objective - r32.stats.objective) <= 1e-5 * abs(r32.stats.objective)
    assert np.abs(r16.X.cpu().numpy() - r32.X.cpu().numpy()).max() <= 1e-3


def test_bf16_batched_wave(solver):
    """A wave of pairs with the BF16 phase: every pair converges in FP32 and
    recovers the ground truth like the FP32 solve."""
    pairs = synth.batch_mixed(count=5, seed=11, n_lo=100, n_hi=400, out_hi=40)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    p16 = F.default_params(lam=0.5, precision=F.BF16, refine_iters=30)
    p32 = F.default_params(lam=0.5)
    o16 = solver.match_batched(dev, params=p16)
    o32 = solver.match_batched(dev, params=p32)
    for a, b in zip(o16, o32):
        assert a.stats.status == 0 and a.stats.lowp_iters >= 1
        assert abs(a.stats.objective - b.stats.objective) <= 1e-4 * abs(b.stats.objective)


def test_batched_mixed_small_pairs_plain(solver):
    """Pairs without attributes and exact-size matches in one wave."""
    pairs = [synth.plain_100(seed=s) for s in range(4)] + [synth.graph_pair(7, p=0.5, sigma=0.0,
                                                                             seed=9)]
    outs = _check_batch(solver, pairs, 0.0, max_outer=40, max_inner=400)
    for g, o in zip(pairs[:4], outs):
        assert (o.perm.cpu().numpy() == g.gt).mean() >= 0.99


# ------------------------------------------------- streamed (continuous) batches

@pytest.fixture(scope="module")
def stream_solver():
    s = F.Solver(max_n=1000, max_batch=128)
    yield s
    s.close()


def _replay_check(solver, g, o, i, lam, **kw):
    inner, _ = solver.last_trace(pair=i)
    assert o.stats.status == 0 and len(inner) == o.stats.outer_iters
    r = oracle.solve(g.A, g.A2, g.B, g.B2, lam=lam, replay_inner=inner,
                     replay_outer=o.stats.outer_iters, **kw)
    Xg = o.X.cpu().numpy()
    assert np.abs(Xg - r["X"]).max() <= 1e-4
    A, A2, Bc, B2c, tr = _canon(g)
    roc = oracle.greedy_sorted((Xg.T if tr else Xg).astype(np.float64))
    K = oracle.affinity(Bc, B2c) if g.k and lam else None
    obj = oracle.qap_objective(A, A2, roc, K, lam)
    assert abs(o.stats.objective - obj) <= 1e-5 * abs(obj)


def test_streamed_batch_refills_waves_and_matches_oracle(stream_solver):
    """Twenty-four pairs of 850..1000 nodes do not fit in one wave (on-chip
    storage):
    the batch is streamed, finished pairs leaving and waiting pairs entering
    between outer iterations.  A loose outer tolerance makes the pairs stop
    at different iterations.  Every pair matches the oracle replaying its
    own inner counts."""
    rng = np.random.default_rng(40)
    pairs = [synth.graph_pair(int(rng.integers(850, 1001)), p=0.1, sigma=0.05, k=8, lam=0.5,
                              seed=400 + i) for i in range(24)]
    kw = dict(max_outer=12, max_inner=80, tol_outer=1e-3)
    p = F.default_params(lam=0.5, **kw)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    outs = stream_solver.match_batched(dev, params=p, want_X=True)
    waves = [o.stats.wave_pairs for o in outs]
    assert 0 < max(waves) < len(pairs)
    assert len({o.stats.outer_iters for o in outs}) > 1   # pairs left at different times
    for i in (0, 5, 11, 17, 19, 21, 22, 23):   # first and last admitted pairs among them
        _replay_check(stream_solver, pairs[i], outs[i], i, 0.5, **kw)


def test_streamed_host_batch_equals_device_batch(stream_solver):
    rng = np.random.default_rng(41)
    pairs = [synth.graph_pair(int(rng.integers(850, 1001)), p=0.1, sigma=0.05, k=8, lam=0.5,
                              seed=500 + i) for i in range(22)]
    p = F.default_params(lam=0.5, max_outer=8, max_inner=60, tol_outer=1e-3)
    d = stream_solver.match_batched([(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs], params=p,
                                    want_X=True)
    assert max(o.stats.wave_pairs for o in d) < len(pairs)
    h = stream_solver.match_batched_host([(g.A, g.A2, g.B, g.B2) for g in pairs], params=p, want_X=True)
    for a, b in zip(d, h):
        _same_solve(a, b, a.X.cpu().numpy(), b.X)


def test_streamed_mixed_batch_of_120(stream_solver):
    """120 mixed pairs (n in 200..600, up to 100 outliers): more than one
    wave holds on chip.  Every pair returns a valid partial permutation;
    sampled pairs match the oracle replay."""
    pairs = synth.batch_mixed(count=120, seed=7, n_lo=200, n_hi=600, out_hi=100)
    kw = dict(max_outer=30, max_inner=200)
    p = F.default_params(lam=0.5, **kw)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    outs = stream_solver.match_batched(dev, params=p, want_X=True)
    assert max(o.stats.wave_pairs for o in outs) < len(pairs)
    for g, o in zip(pairs, outs):
        assert o.stats.status == 0
        perm = o.perm.cpu().numpy()
        n_a, n_b = g.A.shape[0], g.A2.shape[0]
        used = perm[perm >= 0]
        assert len(np.unique(used)) == len(used) and (used < n_b).all()
        assert len(used) == min(n_a, n_b)
    for i in (0, 57, 119):
        _replay_check(stream_solver, pairs[i], outs[i], i, 0.5, **kw)


def test_bandwidth_probe_orders_the_memory_levels():
    """The probe behind the roofline denominators: tensor memory (all SMs)
    is faster than shared memory, which is faster than L2, which is faster
    than HBM; all are plausible for one GB300 (HBM within the measured copy
    figure's ballpark)."""
    tmem = F.bandwidth_probe(3, sweeps=2000)
    smem = F.bandwidth_probe(0, sweeps=2000)
    l2 = F.bandwidth_probe(1, sweeps=200)
    hbm = F.bandwidth_probe(2, sweeps=5)
    assert tmem > smem > l2 > hbm > 1000.0
    assert hbm < 10000.0
    with pytest.raises(F.FastPFPError):
        F.bandwidth_probe(4)


# ------------------------------------------------------------ errors / faults

def test_nonfinite_input_is_reported(solver):
    g = synth.plain_100(0)
    A = g.A.copy()
    A[3, 5] = A[5, 3] = np.nan
    with pytest.raises(F.FastPFPError) as e:
        solver.match(cu(A), cu(g.A2))
    assert e.value.code == F.FASTPFP_ERR_NONFINITE
    solver.match(cu(g.A), cu(g.A2))     # the handle stays usable


def test_argument_errors(solver):
    g = synth.plain_100(0)
    with pytest.raises(F.FastPFPError) as e:
        solver.match(cu(g.A), cu(g.A2), params=F.default_params(alpha=1.5))
    assert e.value.code == F.FASTPFP_ERR_ARG
    big = torch.zeros((1300, 1300), device=DEV)
    with pytest.raises(F.FastPFPError) as e:
        solver.match(big, cu(g.A2))
    assert e.value.code == F.FASTPFP_ERR_SIZE


@pytest.mark.parametrize("loop_mode", [0, 1])
def test_barrier_timeout_is_reported_and_handle_recovers(solver, loop_mode):
    """A lost barrier arrival (test-only flag) makes every wait run out after
    timeout_ms; the call returns ERR_TIMEOUT (the graph loop's condition sees
    the error word and ends) and the context stays usable."""
    g = synth.plain_100(0)
    p = F.default_params(timeout_ms=200, debug_flags=1, max_outer=3, loop_mode=loop_mode)
    with pytest.raises(F.FastPFPError) as e:
        solver.match(cu(g.A), cu(g.A2), params=p)
    assert e.value.code == F.FASTPFP_ERR_TIMEOUT
    res = solver.match(cu(g.A), cu(g.A2))
    assert res.stats.status == 0 and (res.perm.cpu().numpy() == g.gt).mean() >= 0.99


# ------------------------------------------------------ full-size workloads

def test_attributed_1000_full_size_properties(solver):
    """n = n' = 1000 attributed pair at the benchmark's launch configuration:
    the oracle cannot replay the whole solve in seconds, so check what holds
    at any size and sample one gradient step."""
    g = synth.attributed_1000(0)
    p = F.default_params(lam=1.0)
    A, A2, B, B2 = cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)
    res = solver.match(A, A2, B, B2, params=p, want_X=True)
    st = res.stats
    assert st.status == 0 and 1 <= st.outer_iters <= 100
    Xg = res.X.cpu().numpy()
    assert Xg.min() >= 0 and Xg.max() == 1.0
    perm = res.perm.cpu().numpy()
    assert sorted(perm.tolist()) == list(range(1000))
    roc = oracle.greedy_sorted(Xg.astype(np.float64))
    np.testing.assert_array_equal(np.argsort(roc), perm)
    K = oracle.affinity(g.B, g.B2)
    obj = oracle.qap_objective(g.A, g.A2, roc, K, 1.0)
    assert abs(st.objective - obj) <= 1e-5 * abs(obj)
    assert (perm == g.gt).mean() >= 0.98
    # one gradient step at the final X on sampled rows
    G = solver.gradient(A, res.X, A2, solver.affinity(B, B2), 1.0).cpu().numpy()
    rows = np.arange(0, 1000, 97)
    T = g.A[rows].astype(np.float64) @ Xg.astype(np.float64)
    ref = T @ g.A2.astype(np.float64) + K[rows]
    bound = np.abs(g.A[rows]) @ np.abs(Xg).astype(np.float64) @ np.abs(g.A2) + np.abs(K[rows])
    assert (np.abs(G[rows] - ref) <= 1e-5 * bound).all()


# ------------------------------------------------------------ tile shapes

@pytest.mark.parametrize("N,m", [(129, 100), (1000, 900), (1200, 1000)])
def test_gradient_tiles_give_identical_products(solver, N, m):
    """Both CTA tiles of each product accumulate every output in the same
    order: FP32 tile 64 equals tile 128 bit for bit; the BF16 128-column tile
    matches the 256-column one to FP32 rounding and the oracle to the BF16
    bound."""
    rng = np.random.default_rng(N + 17 * m)
    A = synth.random_graph(rng, N, 0.2).astype(np.float32)
    A2 = synth.random_graph(rng, m, 0.2).astype(np.float32)
    X = rng.random((N, m)).astype(np.float32)
    K = rng.normal(size=(N, m)).astype(np.float32)
    lam = 0.7
    bound = np.abs(A) @ np.abs(X).astype(np.float64) @ np.abs(A2) + lam * np.abs(K)
    args = (cu(A), cu(X), cu(A2), cu(K), lam)
    try:
        assert solver.get_tiles(N, 1) == (128, 256)
        g128 = solver.gradient(*args, precision=F.FP32_SIMT).cpu().numpy()
        t256 = solver.gradient(*args, precision=F.BF16).cpu().numpy()
        s256 = solver.gradient(*args).cpu().numpy()
        solver.set_tiles(64, 128, n=N, count=1)
        assert solver.get_tiles(N, 1) == (64, 128)
        g64 = solver.gradient(*args, precision=F.FP32_SIMT).cpu().numpy()
        t128 = solver.gradient(*args, precision=F.BF16).cpu().numpy()
        s128 = solver.gradient(*args).cpu().numpy()
    finally:
        solver.set_tiles(128, 256)
    np.testing.assert_array_equal(g64, g128)
    assert (np.abs(t128 - t256) <= 1e-6 * bound + 1e-30).all()
    assert (np.abs(s128 - s256) <= 1e-6 * bound + 1e-30).all()
    ref16 = oracle.gradient(_bf16(A), _bf16(X), _bf16(A2), K, lam)
    assert (np.abs(t128 - ref16) <= 3e-3 * bound + 1e-30).all()


def test_batched_wave_with_small_tiles_matches_oracle(solver):
    """A wave whose grouped products run on the small tiles (FP32 64 rows,
    BF16 128 columns) against the oracle's replay, and its BF16 phase
    against the FP32 solve."""
    pairs = synth.batch_mixed(count=5, seed=21, n_lo=100, n_hi=400, out_hi=40)
    try:
        solver.set_tiles(64, 128)
        _check_batch(solver, pairs, 0.5, max_outer=20, max_inner=200)
        dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
        o16 = solver.match_batched(dev, params=F.default_params(lam=0.5, precision=F.BF16, refine_iters=30))
    finally:
        solver.set_tiles(128, 256)
    o32 = solver.match_batched(dev, params=F.default_params(lam=0.5))
    for a, b in zip(o16, o32):
        assert a.stats.status == 0 and a.stats.lowp_iters >= 1
        assert abs(a.stats.objective - b.stats.objective) <= 1e-4 * abs(b.stats.objective)


def test_autotune_fills_the_table_for_every_reachable_class():
    s = F.Solver(max_n=1000, max_batch=32)
    try:
        t = s.autotune(reps=2)
        assert t.shape == (F.TUNE_SIZES, F.TUNE_COUNTS, 4)
        # size classes up to N = 1000 (0..3) and every count class are timed
        assert (t[:4] > 0).all() and (t[4:] == 0).all()
        for n in (50, 200, 400, 1000):
            for c in (1, 3, 10, 32):
                f, b = s.get_tiles(n, c)
                assert f in (64, 128) and b in (128, 256)
                sc = {50: 0, 200: 1, 400: 2, 1000: 3}[n]
                cc = {1: 0, 3: 1, 10: 2, 32: 3}[c]
                assert f == (64 if t[sc, cc, 1] < t[sc, cc, 0] else 128)
                assert b == (128 if t[sc, cc, 3] < t[sc, cc, 2] else 256)
        pairs = synth.batch_mixed(count=4, seed=23, n_lo=60, n_hi=300, out_hi=30)
        _check_batch(s, pairs, 0.5, max_outer=15, max_inner=200)
        with pytest.raises(F.FastPFPError):
            s.set_tiles(96, 256)
        with pytest.raises(F.FastPFPError):
            s.autotune(reps=0)
    finally:
        s.close()


# ------------------------------------------------------------ FP8 products

def _e4m3_rows(a):
    """Per-row power-of-two scaling and E4M3 rounding as the FP8 products do
    (the largest e with max|row| * 2^e <= 448, round to nearest even), then
    back to float64: the operand the tensor cores effectively multiply."""
    a = np.asarray(a, dtype=np.float32)
    mx = np.abs(a).max(axis=1).astype(np.float64)
    e = np.zeros(len(a), dtype=np.int64)
    nz = mx > 0
    fr, ex = np.frexp(mx[nz])
    e[nz] = np.where(fr <= 0.875, 9, 8) - ex
    up = np.ldexp(1.0, e)[:, None]
    q = torch.as_tensor((a * up).astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    return q.astype(np.float64) / up


def test_e4m3_emulation_rounds_like_the_format():
    """The test-side emulation itself: E4M3 keeps 3 mantissa bits (relative
    spacing 2^-3), so after scaling every normal value is within 2^-4 of
    itself, the row maximum lands in (224, 448], and exact grid points
    survive unchanged."""
    rng = np.random.default_rng(3)
    a = rng.random((7, 50)).astype(np.float32) * np.logspace(-3, 3, 7, dtype=np.float32)[:, None]
    q = _e4m3_rows(a)
    assert (np.abs(q - a) <= 2.0 ** -4 * np.abs(a) + 1e-12).all()
    grid = np.array([[0.0, 1.0, 1.125, 448.0, 0.015625]], dtype=np.float32)
    np.testing.assert_array_equal(_e4m3_rows(grid), grid.astype(np.float64))


@pytest.mark.parametrize("N,m", [(5, 3), (129, 100), (300, 300), (1000, 1000), (1200, 1000)])
def test_gradient_fp8_tensor_cores_matches_oracle(solver, N, m):
    """tcgen05 E4M3 products with per-row scales.  Against the oracle on the
    operands as the kernels quantise them (A and A' per row from FP32, X per
    column through its BF16 copy) only T's quantisation remains: E4M3 after
    BF16, |err| <= (2^-4 + 2^-8) |A||X||A'| (+ FP32 terms); against the
    unquantised oracle four E4M3 roundings: 0.3 * the bound."""
    rng = np.random.default_rng(N * 7 + m)
    A = synth.random_graph(rng, N, 0.2).astype(np.float32)
    A2 = synth.random_graph(rng, m, 0.2).astype(np.float32)
    X = rng.random((N, m)).astype(np.float32)
    K = rng.normal(size=(N, m)).astype(np.float32)
    lam = 0.7
    G = solver.gradient(cu(A), cu(X), cu(A2), cu(K), lam, precision=F.FP8).cpu().numpy()
    bound = np.abs(A) @ np.abs(X).astype(np.float64) @ np.abs(A2) + lam * np.abs(K)
    ref = oracle.gradient(A, X, A2, K, lam)
    assert (np.abs(G - ref) <= 0.3 * bound + 1e-30).all()
    Aq, A2q = _e4m3_rows(A), _e4m3_rows(A2).T
    Xq = _e4m3_rows(_bf16(X).T).T
    ref8 = oracle.gradient(Aq, Xq, A2q, K, lam)
    bound8 = np.abs(Aq) @ np.abs(Xq) @ np.abs(A2q) + lam * np.abs(K)
    assert (np.abs(G - ref8) <= (2.0 ** -4 + 2.0 ** -8) * bound8 + 1e-5 * bound8 + 1e-30).all()


def test_fp8_phase_then_fp32_refinement(solver):
    """The precision policy with E4M3 products: the FP8 phase runs until
    max|dX| < switch_tol, then FP32 iterations; the refined result matches
    the plain FP32 solve's permutation and objective."""
    g = synth.attributed_1000(seed=2)
    A, A2, B, B2 = cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)
    r32 = solver.match(A, A2, B, B2, params=F.default_params(lam=1.0), want_X=True)
    p8 = F.default_params(lam=1.0, precision=F.FP8, refine_iters=30, switch_tol=1e-3)
    r8 = solver.match(A, A2, B, B2, params=p8, want_X=True)
    st = r8.stats
    assert st.status == 0 and st.lowp_iters >= 1 and st.outer_iters > st.lowp_iters
    assert st.converged == 1
    np.testing.assert_array_equal(r8.perm.cpu().numpy(), r32.perm.cpu().numpy())
    assert abs(st.objective - r32.stats.objective) <= 1e-5 * abs(r32.stats.objective)
    assert np.abs(r8.X.cpu().numpy() - r32.X.cpu().numpy()).max() <= 1e-3


def test_fp8_batched_wave(solver):
    """A wave of uneven pairs with the FP8 phase: every pair ends in FP32 at
    the plain solve's objective."""
    pairs = synth.batch_mixed(count=5, seed=13, n_lo=100, n_hi=400, out_hi=40)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    o8 = solver.match_batched(dev, params=F.default_params(lam=0.5, precision=F.FP8, refine_iters=30))
    o32 = solver.match_batched(dev, params=F.default_params(lam=0.5))
    for a, b in zip(o8, o32):
        assert a.stats.status == 0 and a.stats.lowp_iters >= 1
        assert abs(a.stats.objective - b.stats.objective) <= 1e-4 * abs(b.stats.objective)


def test_gemm_probe_orders_the_product_kernels():
    """The GEMM throughput probe behind the bench's product fractions: every
    kernel does real work (FP32 well above 1 TFLOP/s), the tensor cores beat
    the SIMT kernel, and nothing exceeds its nominal dense peak (FP32 80.5,
    split TF32 375, BF16 2250, FP8 4500 TFLOP/s)."""
    f32 = F.gemm_probe(F.FP32_SIMT, n=2048, reps=3)
    tf32 = F.gemm_probe(F.FP32, n=2048, reps=3)
    bf16 = F.gemm_probe(F.BF16, n=2048, reps=3)
    fp8 = F.gemm_probe(F.FP8, n=2048, reps=3)
    assert 1.0 < f32 < 80.5
    assert f32 < tf32 < 1125.0 / 3      # three TF32 MMAs per product term, TF32 at half the BF16 rate
    assert f32 < bf16 < 2250.0
    assert 1.0 < fp8 < 4500.0
    with pytest.raises(F.FastPFPError):
        F.gemm_probe(F.BF16, n=1000)


# ------------------------------------------- projected gradient, Eq. (pg)

def _check_pg(solver, pairs, lam, alpha, **kw):
    """Every pair of one batched PG solve against the oracle replaying that
    pair's inner counts (X max-abs 1e-4, objective relative 1e-5)."""
    p = F.default_params(lam=lam, alpha=alpha, algorithm=F.ALG_PG, **kw)
    dev = [(cu(g.A), cu(g.A2), cu(g.B) if g.k else None, cu(g.B2) if g.k else None) for g in pairs]
    outs = solver.match_batched(dev, params=p, want_X=True)
    for i, (g, o) in enumerate(zip(pairs, outs)):
        inner, _ = solver.last_trace(pair=i)
        assert o.stats.status == 0 and len(inner) == o.stats.outer_iters
        r = oracle.solve(g.A, g.A2, g.B, g.B2, lam=lam, alpha=alpha, replay_inner=inner,
                         replay_outer=o.stats.outer_iters, algorithm="pg", **kw)
        assert np.abs(o.X.cpu().numpy() - r["X"]).max() <= 1e-4
        assert abs(o.stats.objective - r["objective"]) <= 1e-5 * abs(r["objective"])
    return outs


def test_pg_single_pair_matches_oracle(solver):
    """Eq. (pg) on one attributed pair with outliers: the gradient epilogue
    forms X + alpha (A X A' + lambda K), the projection keeps P_d of it."""
    g = synth.graph_pair(60, p=0.3, sigma=0.02, k=3, n_out=8, lam=0.5, seed=5)
    outs = _check_pg(solver, [g], 0.5, 0.05, normalize_max=False, max_outer=40, max_inner=300)
    assert outs[0].stats.converged == 1


def test_pg_wave_of_uneven_pairs_matches_oracle(solver):
    pairs = synth.batch_mixed(count=5, seed=17, n_lo=20, n_hi=150, out_hi=20)
    _check_pg(solver, pairs, 0.5, 0.05, normalize_max=False, max_outer=25, max_inner=250)


def test_pg_bf16_phase_then_fp32_refinement(solver):
    """PG with the BF16 tensor-core products (the epilogue adds X in FP32)
    and FP32 refinement ends at the plain FP32 PG solve's objective."""
    pairs = synth.batch_mixed(count=4, seed=19, n_lo=100, n_hi=300, out_hi=30)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    kw = dict(lam=0.5, alpha=0.01, algorithm=F.ALG_PG, normalize_max=0)
    o16 = solver.match_batched(dev, params=F.default_params(precision=F.BF16, refine_iters=40, **kw))
    o32 = solver.match_batched(dev, params=F.default_params(**kw))
    for a, b in zip(o16, o32):
        assert a.stats.status == 0 and a.stats.lowp_iters >= 1
        assert abs(a.stats.objective - b.stats.objective) <= 1e-4 * abs(b.stats.objective)


def test_e1_sweep_recovers_isomorphisms():
    """The Section 5.1 driver on small graphs (FastPFP, PG and FastGA):
    FastPFP and FastGA find the hidden isomorphism (case a: zero error,
    accuracy 1) and every row is complete."""
    from paper_1207_1114_gb300 import experiments
    rows = experiments.e1_sweep(sizes=(60,), cases="abcd", max_outer=60, max_inner=400)
    assert len(rows) == 12
    for alg in ("fastpfp", "fastga"):
        a = [r for r in rows if r["case"] == "a" and r["algorithm"] == alg][0]
        assert a["error"] == 0.0 and a["accuracy"] == 1.0
    for r in rows:
        assert r["seconds"] > 0 and r["outer"] >= 1


def test_fp8_transposed_partial_pair(solver):
    """E4M3 products on a pair whose first graph is the smaller one (the
    canonical swap transposes every operand) with outliers: the FP8 phase and
    the FP32 refinement end at the plain FP32 solve's objective."""
    g = synth.graph_pair(300, p=0.15, sigma=0.03, k=8, n_out=60, lam=0.5, seed=27)
    A, A2, B, B2 = cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)       # graph 1 (300) is the smaller
    r32 = solver.match(A, A2, B, B2, params=F.default_params(lam=0.5))
    r8 = solver.match(A, A2, B, B2, params=F.default_params(lam=0.5, precision=F.FP8, refine_iters=30))
    assert r8.stats.status == 0 and r8.stats.transposed == 1 and r8.stats.lowp_iters >= 1
    assert abs(r8.stats.objective - r32.stats.objective) <= 1e-4 * abs(r32.stats.objective)
    perm = r8.perm.cpu().numpy()
    assert (perm >= 0).all() and len(np.unique(perm)) == len(perm)


def test_pg_fp8_phase_then_fp32_refinement(solver):
    """The projected gradient step formed in the E4M3 products' epilogue
    (X + alpha (scaled accumulator) + alpha lambda K) ends, after FP32
    refinement, at the plain FP32 PG solve's objective."""
    pairs = synth.batch_mixed(count=3, seed=29, n_lo=100, n_hi=300, out_hi=30)
    dev = [(cu(g.A), cu(g.A2), cu(g.B), cu(g.B2)) for g in pairs]
    kw = dict(lam=0.5, alpha=0.01, algorithm=F.ALG_PG, normalize_max=0)
    o8 = solver.match_batched(dev, params=F.default_params(precision=F.FP8, refine_iters=40, **kw))
    o32 = solver.match_batched(dev, params=F.default_params(**kw))
    for a, b in zip(o8, o32):
        assert a.stats.status == 0 and a.stats.lowp_iters >= 1
        assert abs(a.stats.objective - b.stats.objective) <= 1e-4 * abs(b.stats.objective)


def test_autotune_on_a_tiny_handle():
    """Tile timing on the smallest shapes (N = 40: one partial tile, TMA boxes
    larger than the matrices) and a solve on whatever it picked, against the
    oracle replay."""
    s = F.Solver(max_n=40, max_batch=3)
    try:
        t = s.autotune(reps=1)
        assert (t[0, :2] > 0).all() and (t[1:] == 0).all()
        pairs = [synth.graph_pair(n, p=0.4, sigma=0.02, k=3, lam=0.5, seed=60 + n) for n in (12, 25, 33)]
        _check_batch(s, pairs, 0.5, max_outer=20, max_inner=200)
    finally:
        s.close()
