"""Host side of the synthetic experiments: the Section 5.1 graph generator
and the matching-error measure, checked against what their definitions fix."""
import numpy as np
import pytest

from paper_1207_1114_gb300 import synth
from paper_1207_1114_gb300.experiments import lipschitz_step, matching_error


@pytest.mark.parametrize("case", ["a", "b", "c", "d"])
def test_e1_pairs_follow_section_5_1(case):
    n = 80
    g = synth.e1_pair(n, case, seed=3)
    m = n - n // 10 if case in "cd" else n
    assert g.A.shape == (n, n) and g.A2.shape == (m, m) and g.B.shape == (n, 0)
    for M in (g.A, g.A2):
        assert (M == M.T).all() and (np.diag(M) == 0).all() and set(np.unique(M)) <= {0.0, 1.0}
    assert abs(g.A.sum() / (n * (n - 1)) - 0.5) < 0.05          # 50 % connectivity
    kept = np.where(g.gt >= 0)[0]
    assert len(kept) == m and sorted(g.gt[kept].tolist()) == list(range(m))
    back = g.A2[np.ix_(g.gt[kept], g.gt[kept])]
    flips = int((back != g.A[np.ix_(kept, kept)]).sum())
    if case == "a" or case == "c":
        assert flips == 0
    if case == "b":
        assert flips == 2 * n                                     # n edited pairs, both triangles
    if case == "d":
        assert 0 < flips <= 2 * n


def test_matching_error_is_the_frobenius_residual():
    """||A - X A' X^T||_F^2: zero for the hidden isomorphism, 2n after n edge
    editions, and the brute-force matrix product for any partial map."""
    g = synth.e1_pair(40, "a", seed=5)
    assert matching_error(g.A, g.A2, g.gt) == 0.0
    gb = synth.e1_pair(40, "b", seed=5)
    assert matching_error(gb.A, gb.A2, gb.gt) == 2 * 40
    rng = np.random.default_rng(0)
    perm = rng.permutation(40).astype(np.int32)
    perm[rng.choice(40, 5, replace=False)] = -1
    X = np.zeros((40, 40))
    X[np.where(perm >= 0)[0], perm[perm >= 0]] = 1.0
    ref = ((g.A - X @ g.A2 @ X.T) ** 2).sum()
    assert matching_error(g.A, g.A2, perm) == pytest.approx(ref, abs=1e-9)


def test_lipschitz_step_of_a_complete_graph():
    """The complete graph's adjacency J - I has spectral norm n - 1."""
    n = 30
    A = np.ones((n, n)) - np.eye(n)
    assert lipschitz_step(A, A) == pytest.approx(1.0 / (n - 1) ** 2, rel=1e-9)


def test_torch_training_pairs_follow_the_recipe():
    """The learned warm start's training pairs drawn with torch (on the CPU
    here): symmetric zero-diagonal graphs, graph 2 a relabelled noisy copy of
    graph 1 plus outliers, attributes copied with small noise; seeded, so the
    same seed gives the same pairs."""
    torch = pytest.importorskip("torch")
    a = list(synth.warm_start_train_torch(3, seed=4, device="cpu", n_lo=20, n_hi=40))
    b = list(synth.warm_start_train_torch(3, seed=4, device="cpu", n_lo=20, n_hi=40))
    for (A, A2, B, B2, gt), (A_, _, _, _, gt_) in zip(a, b):
        assert torch.equal(A, A_) and torch.equal(gt, gt_)
        n, n2 = A.shape[0], A2.shape[0]
        assert 20 <= n <= 40 and n <= n2 <= n + n // 5 and B.shape == (n, 15) and B2.shape == (n2, 15)
        for M in (A, A2):
            assert torch.equal(M, M.T) and (M.diagonal() == 0).all()
        g = gt.long()
        assert len(set(g.tolist())) == n and int(g.max()) < n2
        back = A2[g][:, g]
        assert ((back != 0) == (A != 0)).all()                 # noise only on existing edges
        assert float((back - A).abs().max()) < 0.3               # sigma = 0.03
        assert float((B2[g] - B).abs().max()) < 0.5              # attr sigma = 0.05
