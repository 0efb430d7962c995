"""Pins for the FP64 oracle: each test checks an oracle function against
something other than itself -- a closed form solved a different way, an
identity from the paper's Appendix, finite differences, brute force, a
library routine on a special case, or a theorem's bound.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1207_1114_gb300 import synth


def _sym(rng, n, scale=1.0):
    a = rng.random((n, n)) * scale
    a = np.triu(a, 1)
    return a + a.T


# ---------------------------------------------------------------- P1, Eq. (P1)

def _kkt_affine_projection(Y):
    """Euclidean projection of Y onto {D : D1 = 1, D^T 1 = 1}, solved as a
    constrained least-squares problem (pseudo-inverse of the constraint Gram
    matrix), independent of the closed form of Eq. (P1)."""
    n = Y.shape[0]
    C = np.zeros((2 * n, n * n))
    for i in range(n):
        C[i, i * n:(i + 1) * n] = 1.0           # row sums
        C[n + i, i::n] = 1.0                    # column sums
    y = Y.reshape(-1)
    mu = np.linalg.pinv(C @ C.T) @ (C @ y - 1.0)
    return (y - C.T @ mu).reshape(n, n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13])
def test_p1_equals_kkt_projection(n):
    rng = np.random.default_rng(n)
    Y = rng.normal(size=(n, n)) * 3.0
    np.testing.assert_allclose(oracle.p1(Y), _kkt_affine_projection(Y), atol=1e-11, rtol=0)


def test_p1_sums_are_one_and_idempotent():
    rng = np.random.default_rng(1)
    Y = rng.normal(size=(60, 60)) * 10
    Z = oracle.p1(Y)
    assert np.abs(Z.sum(0) - 1).max() < 1e-12
    assert np.abs(Z.sum(1) - 1).max() < 1e-12
    np.testing.assert_allclose(oracle.p1(Z), Z, atol=1e-13)


# ---------------------------------------------------------------- P2, Eq. (P2)

def test_p2_is_nearest_nonnegative():
    rng = np.random.default_rng(2)
    Y = rng.normal(size=(17, 17))
    Z = oracle.p2(Y)
    assert (Z >= 0).all()
    assert (Z[Y >= 0] == Y[Y >= 0]).all()
    assert (Z[Y < 0] == 0).all()


# ---------------------------------------------------------- P_D, Sec. 4.3

def test_pd_single_step_when_p1_is_nonnegative():
    """If P1(Y) >= 0 the alternation stops at P1(Y): the second P1 changes
    nothing (sums already 1) and P2 changes nothing (already >= 0)."""
    rng = np.random.default_rng(3)
    n = 20
    Y = np.full((n, n), 1.0 / n) + rng.normal(0, 1e-3, (n, n))
    P1 = _kkt_affine_projection(Y)
    assert (P1 > 0).all()
    out, it, last = oracle.pd(Y, tol=1e-9, max_iter=100)
    assert it == 2 and last < 1e-12
    np.testing.assert_allclose(out, P1, atol=1e-12)


def _birkhoff(rng, n, terms=6):
    w = rng.random(terms)
    w /= w.sum()
    D = np.zeros((n, n))
    for t in range(terms):
        D[np.arange(n), rng.permutation(n)] += w[t]
    return D


def test_pd_fixes_doubly_stochastic_input():
    rng = np.random.default_rng(4)
    D = _birkhoff(rng, 12)
    out, it, last = oracle.pd(D, tol=1e-9, max_iter=100)
    assert it == 1 and last < 1e-14
    np.testing.assert_allclose(out, D, atol=1e-14)


@pytest.mark.parametrize("n", [7, 40])
def test_pd_output_is_doubly_stochastic(n):
    rng = np.random.default_rng(n)
    Y = rng.random((n, n)) * rng.random((n, 1)) * 50.0   # gradient-like, uneven scale
    out, it, last = oracle.pd(Y, tol=1e-12, max_iter=200000)
    assert last < 1e-12
    assert (out >= 0).all()
    assert np.abs(out.sum(1) - 1).max() < 1e-9
    assert np.abs(out.sum(0) - 1).max() < 1e-9


def test_pd_partial_block_sums():
    """Section 4.3: with slack columns, X = P_D(Y)[:, :m] has unit column sums
    and row sums <= 1."""
    rng = np.random.default_rng(5)
    N, m = 30, 22
    Y = np.zeros((N, N))
    Y[:, :m] = rng.random((N, m)) * 5
    out, _, last = oracle.pd(Y, tol=1e-12, max_iter=200000)
    X = out[:, :m]
    assert np.abs(X.sum(0) - 1).max() < 1e-9
    assert (X.sum(1) <= 1 + 1e-9).all()


def test_pd_fixed_iterations_is_nonexpansive():
    """A fixed number of (P1, P2) rounds composes projections onto convex
    sets, so it is nonexpansive (Lemma 1's ingredient)."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        Y1 = rng.normal(size=(9, 9))
        Y2 = Y1 + rng.normal(size=(9, 9)) * rng.random()
        a, _, _ = oracle.pd(Y1, fixed_iters=7)
        b, _, _ = oracle.pd(Y2, fixed_iters=7)
        assert np.linalg.norm(a - b) <= np.linalg.norm(Y1 - Y2) * (1 + 1e-12)


# ----------------------------------------------------- gradient, Sec. 4.1

def test_gradient_matches_finite_differences_of_f():
    rng = np.random.default_rng(7)
    N, m, k, lam = 7, 5, 3, 0.7
    A, A2 = _sym(rng, N), _sym(rng, m)
    B, B2 = rng.normal(size=(N, k)), rng.normal(size=(m, k))
    K = oracle.affinity(B, B2)
    X = rng.random((N, m))

    def f(Z):  # Section 4.1: f = 1/2 tr(Z^T A Z A') + lambda tr(Z^T B B'^T)
        return 0.5 * np.trace(Z.T @ A @ Z @ A2) + lam * np.trace(Z.T @ B @ B2.T)

    G = oracle.gradient(A, X, A2, K, lam)
    h = 1e-6
    num = np.zeros_like(X)
    for i in range(N):
        for j in range(m):
            E = np.zeros_like(X)
            E[i, j] = h
            num[i, j] = (f(X + E) - f(X - E)) / (2 * h)
    np.testing.assert_allclose(G, num, rtol=1e-7, atol=1e-7)
    assert abs(oracle.relaxed_objective(A, A2, X, K, lam) - f(X)) < 1e-10


# --------------------------------------- objectives, Sec. 3 and Appendix

def _perm_matrix(row_of_col, N):
    m = len(row_of_col)
    P = np.zeros((N, m))
    P[row_of_col, np.arange(m)] = 1.0
    return P


@pytest.mark.parametrize("N,m", [(5, 5), (6, 4)])
def test_error_objective_matches_definition_and_appendix_identity(N, m):
    """Eq. (1) by its definition with an explicit P, and the Appendix identity
    Eq. (1) = const - 2 * Eq. (3) for every partial permutation."""
    rng = np.random.default_rng(N * 10 + m)
    k, lam = 3, 0.4
    A, A2 = _sym(rng, N), _sym(rng, m)
    B, B2 = rng.normal(size=(N, k)), rng.normal(size=(m, k))
    K = oracle.affinity(B, B2)
    const = 0.5 * (np.sum(A * A) + np.sum(A2 * A2)) + lam * (np.sum(B * B) + np.sum(B2 * B2))
    for rows in itertools.permutations(range(N), m):
        r = np.array(rows, dtype=np.int32)
        P = _perm_matrix(r, N)
        direct = 0.5 * np.linalg.norm(A - P @ A2 @ P.T) ** 2 + lam * np.linalg.norm(B - P @ B2) ** 2
        e = oracle.error_objective(A, A2, r, B, B2, lam)
        q = oracle.qap_objective(A, A2, r, K, lam)
        assert abs(e - direct) < 1e-9
        assert abs(e - (const - 2.0 * q)) < 1e-9


# ----------------------------------------------------- greedy, Sec. 4.5

def _greedy_python(X):
    """Steps 1-3 of Section 4.5 with Python sets (tiny inputs only)."""
    N, m = X.shape
    L = {(i, j) for i in range(N) for j in range(m)}
    out = -np.ones(m, dtype=np.int32)
    while L:
        best = max(L, key=lambda ij: (X[ij], -(ij[0] * m + ij[1])))
        out[best[1]] = best[0]
        L = {(i, j) for (i, j) in L if i != best[0] and j != best[1]}
    return out


@pytest.mark.parametrize("shape", [(1, 1), (4, 4), (7, 3), (9, 9)])
@pytest.mark.parametrize("levels", [0, 3])
def test_greedy_literal_sorted_and_python_agree(shape, levels):
    rng = np.random.default_rng(shape[0] * 7 + shape[1] + levels)
    for _ in range(10):
        X = rng.random(shape)
        if levels:
            X = np.floor(X * levels) / levels   # many exact ties
        a = oracle.greedy_literal(X)
        b = oracle.greedy_sorted(X)
        c = _greedy_python(X)
        assert (a == b).all() and (a == c).all()


def test_greedy_equals_hungarian_on_dominant_matrices():
    """When every row's maximum is a distinct column and dominates its column,
    greedy and optimal assignment coincide."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(8)
    for n in (5, 50, 300):
        p = rng.permutation(n)
        X = rng.random((n, n)) * 0.1
        X[np.arange(n), p] += 1.0
        r = oracle.greedy_sorted(X)
        rows, cols = linear_sum_assignment(-X)
        ref = np.empty(n, dtype=np.int32)
        ref[cols] = rows
        assert (r == ref).all()
        assert (oracle.greedy_literal(X) == ref).all()


# --------------------------------------- blend / closure / Theorem 1

def test_closure_under_convex_combination():
    """Section 4.1: with normalisation off, a partial-DS X stays partial-DS
    when blended with a DS P_D output."""
    rng = np.random.default_rng(9)
    N = m = 10
    X = _birkhoff(rng, N)
    Y = _birkhoff(rng, N)
    Xn, d = oracle.blend(X, Y, alpha=0.3, normalize=False)
    assert (Xn >= 0).all()
    assert np.abs(Xn.sum(0) - 1).max() < 1e-14 and np.abs(Xn.sum(1) - 1).max() < 1e-14
    np.testing.assert_allclose(Xn, 0.7 * X + 0.3 * Y, atol=1e-15)
    assert d == pytest.approx(np.abs(0.3 * (Y - X)).max(), abs=1e-15)


def test_normalisation_divides_by_max():
    rng = np.random.default_rng(10)
    X = rng.random((6, 4))
    Y = np.zeros((6, 6))
    Y[:, :4] = rng.random((6, 4)) * 3
    Xn, _ = oracle.blend(X, Y, alpha=0.5, normalize=True)
    assert Xn.max() == 1.0
    raw = 0.5 * X + 0.5 * Y[:, :4]
    np.testing.assert_allclose(Xn * raw.max(), raw, rtol=1e-15)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.9])
def test_theorem1_linear_rate(alpha):
    """Theorem 1: with ||A (x) A'||_2 < eps and no normalisation, successive
    differences contract at rate 1 - alpha + alpha*eps.  The inner loop runs
    a fixed number of rounds so the projection map is one fixed
    nonexpansive map."""
    rng = np.random.default_rng(11)
    n, lam = 9, 0.5
    A, A2 = _sym(rng, n), _sym(rng, n)
    eps = 0.6
    s = np.sqrt(eps / (np.linalg.norm(A, 2) * np.linalg.norm(A2, 2)))
    A, A2 = A * s, A2 * s
    K = oracle.affinity(rng.normal(size=(n, 4)), rng.normal(size=(n, 4)))
    X = rng.random((n, n))
    prev = None
    rate = 1 - alpha + alpha * eps
    ratios = []
    for _ in range(12):
        G = oracle.gradient(A, X, A2, K, lam)
        Y, _, _ = oracle.pd(G, fixed_iters=25)
        Xn, _ = oracle.blend(X, Y, alpha=alpha, normalize=False)
        diff = np.linalg.norm(Xn - X)
        if prev is not None and prev > 1e-13:
            ratios.append(diff / prev)
        prev, X = diff, Xn
    assert max(ratios) <= rate + 1e-9


# ------------------------------------------------ whole method, Alg. 1

def test_exact_recovery_of_noiseless_copy():
    """Section 5.1 (graph isomorphism): a permuted noiseless copy is matched
    to the ground truth."""
    g = synth.graph_pair(80, p=0.3, sigma=0.0, seed=3)
    r = oracle.solve(g.A, g.A2)
    assert (r["perm"] == g.gt).all()
    assert r["error"] < 1e-8


def test_attributed_recovery_and_ground_truth_objective():
    g = synth.graph_pair(120, p=0.1, sigma=0.05, k=16, lam=1.0, seed=4)
    r = oracle.solve(g.A, g.A2, g.B, g.B2, lam=1.0)
    assert (r["perm"] == g.gt).mean() >= 0.99
    gt_rows = np.argsort(g.gt).astype(np.int32)   # graph-1 row matched to each graph-2 column
    K = oracle.affinity(g.B, g.B2)
    gt_obj = oracle.qap_objective(g.A, g.A2, gt_rows, K, 1.0)
    assert r["objective"] >= gt_obj - 1e-6 * abs(gt_obj)


@pytest.mark.parametrize("n", [4, 5, 6])
def test_brute_force_optimum_on_tiny_isomorphic_graphs(n):
    """Brute force over all n! permutations: on a noiseless copy FastPFP's
    discrete objective reaches the optimum; the brute-force optimum itself
    is the ground truth's."""
    for seed in range(4):
        g = synth.graph_pair(n, p=0.6, sigma=0.0, seed=100 + seed)
        A, A2 = g.A.astype(np.float64), g.A2.astype(np.float64)
        best = max(oracle.qap_objective(A, A2, np.array(p, dtype=np.int32))
                   for p in itertools.permutations(range(n)))
        gt_rows = np.argsort(g.gt).astype(np.int32)
        assert abs(oracle.qap_objective(A, A2, gt_rows) - best) < 1e-9
        r = oracle.solve(A, A2)
        assert r["objective"] <= best + 1e-9


def test_swapped_graph_order_gives_transposed_result():
    """Section 3 assumes n >= n'; solving (A', A) must give the transpose."""
    g = synth.graph_pair(30, p=0.3, sigma=0.02, k=4, n_out=6, lam=0.5, seed=5)
    r1 = oracle.solve(g.A, g.A2, g.B, g.B2, lam=0.5)
    r2 = oracle.solve(g.A2, g.A, g.B2, g.B, lam=0.5)
    assert r1["transposed"] and not r2["transposed"]
    np.testing.assert_array_equal(r1["X"], r2["X"].T)
    for i, j in enumerate(r1["perm"]):
        assert r2["perm"][j] == i
    assert r1["objective"] == r2["objective"]


def test_replay_reproduces_free_run():
    g = synth.plain_100(seed=1)
    r = oracle.solve(g.A, g.A2, max_outer=30)
    rr = oracle.solve(g.A, g.A2, max_outer=30, replay_inner=r["inner"], replay_outer=r["outer_iters"])
    np.testing.assert_array_equal(r["X"], rr["X"])
    np.testing.assert_array_equal(r["perm"], rr["perm"])


def test_thread_count_does_not_change_results():
    g = synth.graph_pair(60, p=0.2, sigma=0.02, k=3, n_out=7, lam=0.3, seed=6)
    n0 = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        a = oracle.solve(g.A, g.A2, g.B, g.B2, lam=0.3, max_outer=8)
        oracle.set_num_threads(max(2, n0))
        b = oracle.solve(g.A, g.A2, g.B, g.B2, lam=0.3, max_outer=8)
    finally:
        oracle.set_num_threads(n0)
    np.testing.assert_array_equal(a["X"], b["X"])


# ------------------------------------ projected gradient, Eq. (pg)

def _random_doubly_stochastic(rng, n, terms=4):
    """A convex combination of permutation matrices (Birkhoff)."""
    w = rng.random(terms)
    w /= w.sum()
    X = np.zeros((n, n))
    for c in w:
        X[np.arange(n), rng.permutation(n)] += c
    return X


def test_pg_zero_step_keeps_a_feasible_point():
    """Eq. (pg) with alpha = 0 is X <- P_d(X): a doubly stochastic X is its
    own projection, so the first iterate equals X(0) (a method that dropped
    the X term would return the uniform matrix instead)."""
    rng = np.random.default_rng(31)
    n = 6
    A, A2 = _sym(rng, n), _sym(rng, n)
    X0 = _random_doubly_stochastic(rng, n)
    r = oracle.solve(A, A2, alpha=0.0, X0=X0, normalize_max=False, max_outer=1, tol_inner=1e-13,
                     max_inner=50, algorithm="pg")
    np.testing.assert_allclose(r["X"], X0, atol=1e-12)
    assert r["delta"][0] <= 1e-12


@pytest.mark.parametrize("N,m", [(7, 7), (9, 6)])
def test_pg_on_a_linear_objective_reaches_the_assignment_optimum(N, m):
    """With A = A' = 0 the objective is lambda tr(X^T K) and Eq. (pg) is
    projected gradient ascent of a linear function: its iterates settle on
    the optimal vertex, the linear assignment maximum (scipy), as a 0/1
    matrix — FastPFP's blend of the same gradient would settle on the soft
    projection P_d(lambda K) instead."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(N * 10 + m)
    B, B2 = rng.normal(size=(N, 4)), rng.normal(size=(m, 4))
    K = B @ B2.T
    r = oracle.solve(np.zeros((N, N)), np.zeros((m, m)), B, B2, lam=1.0, alpha=1.0, normalize_max=False,
                     max_outer=300, tol_outer=1e-12, tol_inner=1e-12, max_inner=2000, algorithm="pg")
    rows, cols = linear_sum_assignment(K, maximize=True)
    P = np.zeros((N, m))
    P[rows, cols] = 1.0
    assert np.abs(r["X"] - P).max() < 1e-6
    expect = np.full(N, -1, dtype=np.int32)
    expect[rows] = cols
    assert (r["perm"] == expect).all()


def test_pg_is_equivariant_under_relabelling():
    """Relabelling graph 2's nodes by q (A2 -> A2[q][:, q], B2 -> B2[q])
    relabels the columns of every PG iterate the same way (the uniform start
    is invariant): catches a transposed operand or a mixed-up index."""
    rng = np.random.default_rng(33)
    n = 9
    g = synth.graph_pair(n, p=0.4, sigma=0.05, k=3, lam=0.5, seed=4)
    q = rng.permutation(n)
    kw = dict(lam=0.5, alpha=0.02, normalize_max=False, max_outer=6, tol_outer=0.0, tol_inner=1e-12,
              max_inner=400, algorithm="pg")
    r = oracle.solve(g.A, g.A2, g.B, g.B2, **kw)
    rq = oracle.solve(g.A, g.A2[q][:, q], g.B, g.B2[q], **kw)
    np.testing.assert_allclose(rq["X"], r["X"][:, q], atol=1e-10)
    np.testing.assert_allclose(rq["delta"], r["delta"], rtol=1e-8, atol=1e-12)


def test_replay_rejects_a_trace_shorter_than_the_replay():
    """A replay needs one positive inner count per outer iteration it runs;
    a shorter or zero trace is an error, not a read past its end."""
    g = synth.plain_100(0)
    with pytest.raises(ValueError):
        oracle.solve(g.A, g.A2, replay_inner=[3, 3], replay_outer=3)
    with pytest.raises(ValueError):
        oracle.solve(g.A, g.A2, replay_inner=[3, 0, 3], replay_outer=3)
    r = oracle.solve(g.A, g.A2, replay_inner=[3, 3, 3, 9], replay_outer=3)
    assert list(r["inner"]) == [3, 3, 3]
