"""Pins of the FastGA oracle (oracle/fastga.py) to what the paper and the
mathematics fix, independent of the oracle itself:

  * Eq. (GAO4) with C_aibj = A_ij A'_ab, summed index by index, equals the
    product of Eq. (GAO3) (the Appendix's O(n^4) -> O(n^3) step);
  * the normalisation loop is Sinkhorn scaling: its fixed point is doubly
    stochastic and keeps the cross ratios of exp(beta Q / max|Q|), and a
    per-row constant added to Q does not change it;
  * beta acts on Q / max|Q|: scaling A (so Q) by any positive factor leaves
    the soft-assignment, hence the whole run, unchanged;
  * closed forms: with nothing to match (A = 0, lambda = 0) every iterate
    is the uniform doubly stochastic matrix;
  * a noiseless permuted copy is recovered (the ground truth is known), in
    either orientation, and a partial match assigns every node of the
    smaller graph exactly once (unit column sums of X);
  * replaying a run's own inner counts reproduces it."""
import numpy as np
import pytest

from oracle import fastga as ga
from oracle import gradient
from paper_1207_1114_gb300 import synth


def test_gao4_index_sum_equals_the_gao3_product():
    rng = np.random.default_rng(1)
    n, n2 = 5, 4
    A = synth.random_graph(rng, n, 0.6)
    A2 = synth.random_graph(rng, n2, 0.6)
    X = rng.random((n, n2))
    # Q_ia = sum_j sum_b X_jb C_aibj, C_aibj = A_ij A'_ab (i, j: graph 1; a, b: graph 2)
    Q4 = np.zeros((n, n2))
    for i in range(n):
        for a in range(n2):
            for j in range(n):
                for b in range(n2):
                    Q4[i, a] += X[j, b] * A[i, j] * A2[a, b]
    np.testing.assert_allclose(gradient(A, X, A2), Q4, rtol=1e-13, atol=1e-13)


def test_normalisation_is_sinkhorn_scaling():
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(7, 7))
    Y, k, d = ga.normalise(ga.soft_assign(Q, 0.7), tol=1e-14, max_iter=20000)
    assert d < 1e-14 and k < 20000
    np.testing.assert_allclose(Y.sum(0), 1.0, atol=1e-12)
    np.testing.assert_allclose(Y.sum(1), 1.0, atol=1e-12)
    E = np.exp(0.7 * Q / np.abs(Q).max())
    r1 = Y[0, 0] * Y[2, 3] / (Y[0, 3] * Y[2, 0])
    r2 = E[0, 0] * E[2, 3] / (E[0, 3] * E[2, 0])
    assert r1 == pytest.approx(r2, rel=1e-10)
    # a constant per row of the scaled Q is divided out by the first row normalisation
    c = rng.normal(size=(7, 1)) * 0.3
    s = np.abs(Q).max()
    Y2, _, _ = ga.normalise(np.maximum(np.exp(0.7 * (Q / s + c)), ga.FLOOR), tol=1e-14, max_iter=20000)
    np.testing.assert_allclose(Y2, Y, rtol=1e-9, atol=1e-12)


def test_beta_acts_on_q_scaled_by_its_largest_magnitude():
    g = synth.graph_pair(24, p=0.3, sigma=0.05, k=3, n_out=4, lam=0.5, seed=9)
    r = ga.solve(g.A, g.A2, g.B, g.B2, lam=0.5, max_outer=6, max_inner=200)
    # A, A' and B, B' doubled: both terms of Q = A X A' + lambda B B'^T scale by 4
    r2 = ga.solve(2.0 * g.A, 2.0 * g.A2, 2.0 * g.B, 2.0 * g.B2, lam=0.5, max_outer=6, max_inner=200)
    np.testing.assert_array_equal(r2["inner"], r["inner"])
    np.testing.assert_allclose(r2["X"], r["X"], rtol=1e-9, atol=1e-12)
    np.testing.assert_array_equal(r2["perm"], r["perm"])


def test_nothing_to_match_gives_the_uniform_matrix():
    n = 6
    A = np.zeros((n, n))
    r = ga.solve(A, A, beta=100.0, max_outer=5, max_inner=50)
    np.testing.assert_allclose(r["X"], 1.0 / n, rtol=0, atol=1e-15)
    # uniform 1/(n n) start, then 1/n twice: converged at the second iteration
    assert r["outer_iters"] == 2 and r["converged"]
    assert r["delta"][1] == 0.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_recovers_a_noiseless_permuted_copy(seed):
    g = synth.graph_pair(30, p=0.3, sigma=0.0, k=0, seed=seed)
    r = ga.solve(g.A, g.A2, beta=100.0)
    np.testing.assert_array_equal(r["perm"], g.gt)
    assert r["converged"]
    # the other orientation gives the inverse correspondence
    rt = ga.solve(g.A2, g.A, beta=100.0)
    np.testing.assert_array_equal(rt["perm"][r["perm"]], np.arange(30))


def test_partial_match_assigns_every_node_of_the_smaller_graph_once():
    g = synth.graph_pair(24, p=0.3, sigma=0.0, k=4, n_out=6, lam=0.5, seed=4)
    r = ga.solve(g.A, g.A2, g.B, g.B2, lam=0.5, beta=100.0, tol_inner=1e-12, max_inner=5000)
    X = r["X"]                                   # 24 x 30: graph 1's nodes are the rows here
    assert X.shape == (24, 30)
    np.testing.assert_allclose(X.sum(1), 1.0, atol=1e-9)      # each node of the smaller graph (the
    # column normalisation is the last step); at most one unit per node of the larger, up to how far
    # the 5000 normalisation steps got (Sinkhorn converges slowly on a near-permutation)
    assert (X.sum(0) <= 1.0 + 1e-4).all()
    np.testing.assert_array_equal(r["perm"], g.gt)


def test_replaying_the_inner_counts_reproduces_the_run():
    g = synth.graph_pair(20, p=0.3, sigma=0.05, k=0, seed=7)
    r = ga.solve(g.A, g.A2, beta=100.0, max_outer=6, max_inner=300)
    rr = ga.solve(g.A, g.A2, beta=100.0, max_outer=6, max_inner=300, replay_inner=r["inner"])
    np.testing.assert_array_equal(rr["X"], r["X"])
    np.testing.assert_array_equal(rr["inner"], r["inner"])
    with pytest.raises(ValueError):
        ga.solve(g.A, g.A2, beta=100.0, max_outer=2, replay_inner=[3, 0])
