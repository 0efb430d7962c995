"""Pins for the FP64 warm-start oracle (oracle/warmstart.py): the analytic
gradient against central finite differences of the loss, the loss against a
second evaluation with scipy's logsumexp, the feature definitions on a
hand-built graph, Sinkhorn's limit, and Adam's first step.  CPU only."""
import numpy as np
import pytest
from scipy.special import logsumexp

from oracle import warmstart as ws
from paper_1207_1114_gb300 import synth


def _pair(n=7, n_out=3, k=4, seed=0):
    return synth.graph_pair(n, p=0.5, sigma=0.05, k=k, n_out=n_out, lam=0.5, seed=seed)


@pytest.mark.parametrize("swap", [False, True])
def test_gradient_matches_finite_differences(swap):
    g = _pair()
    A, A2, B, B2 = g.A, g.A2, g.B, g.B2
    perm = g.gt.copy()                    # node of graph 2 matched to node i of graph 1
    if swap:                              # graph 1 is the larger one
        A, A2, B, B2 = A2, A, B2, B
        inv = -np.ones(g.n2, dtype=np.int32)
        inv[g.gt] = np.arange(g.n, dtype=np.int32)
        perm = inv
    rng = np.random.default_rng(1)
    params = ws.init_params(3).astype(np.float64) + rng.normal(0, 0.05, ws.NPARAMS)
    loss, grad = ws.loss_and_grad(A, A2, B, B2, perm, params)
    idx = rng.choice(ws.NPARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(ws.NPARAMS)
        e[i] = h
        lp, _ = ws.loss_and_grad(A, A2, B, B2, perm, params + e)
        lm, _ = ws.loss_and_grad(A, A2, B, B2, perm, params - e)
        assert abs((lp - lm) / (2 * h) - grad[i]) <= 1e-6 + 1e-5 * abs(grad[i])


def test_loss_matches_logsumexp_definition():
    g = _pair(seed=2)
    params = ws.init_params(5)
    loss, _ = ws.loss_and_grad(g.A, g.A2, g.B, g.B2, g.gt, params)
    # columns = graph 1 (smaller); t(j) = gt[j]
    _, Eb = ws.mlp_forward(ws.features(g.A2, g.B2), params)
    _, Es = ws.mlp_forward(ws.features(g.A, g.B), params)
    S = Eb @ Es.T / 8
    m = S.shape[1]
    ref = 0.0
    for j in range(m):
        t = g.gt[j]
        ref -= (S[t, j] - logsumexp(S[:, j])) / m
        ref -= (S[t, j] - logsumexp(S[t, :])) / m
    assert loss == pytest.approx(ref, rel=1e-12)


def test_features_on_hand_built_graph():
    W = np.array([[0.0, 0.5, 0.0625, 0.0],
                  [0.5, 0.0, 1.0, 0.0],
                  [0.0625, 1.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0]])
    F = ws.features(W, None)
    # node 0: weights 0.5 -> bin 8, 0.0625 -> bin 1; node 1: 0.5 -> 8, 1.0 -> 15
    assert F[0, 1 + 8] == 0.5 and F[0, 1 + 1] == 0.5
    assert F[1, 1 + 8] == 0.5 and F[1, 1 + 15] == 0.5
    assert F[3, 1:17].sum() == 0.0                      # isolated node: empty histogram
    deg = W.sum(1)
    np.testing.assert_allclose(F[:, 0], (deg - deg.mean()) / (deg.std() + 1e-6))
    assert np.all(F[:, 17:] == 0)


def test_sinkhorn_converges_to_doubly_stochastic():
    rng = np.random.default_rng(4)
    S = rng.normal(size=(9, 9))
    K = ws.sinkhorn(S, iters=500)
    assert np.abs(K.sum(0) - 1).max() < 1e-12
    assert np.abs(K.sum(1) - 1).max() < 1e-9
    # Sinkhorn scaling keeps the cross ratios of exp(S)
    E = np.exp(S)
    r1 = K[0, 0] * K[1, 1] / (K[0, 1] * K[1, 0])
    r2 = E[0, 0] * E[1, 1] / (E[0, 1] * E[1, 0])
    assert r1 == pytest.approx(r2, rel=1e-10)


def test_sinkhorn_of_peaked_or_far_apart_rows_stays_finite():
    """Rows far below the global maximum (a trained S can span thousands):
    shifting by each row's own maximum keeps them; the result is the same
    doubly stochastic matrix a plain global shift gives where that does not
    underflow."""
    K = ws.sinkhorn(np.array([[0.0, 0.0], [-2000.0, -2000.0]]), iters=3)
    np.testing.assert_array_equal(K, np.full((2, 2), 0.5))
    # a very peaked similarity: the permutation it encodes, off entries at the floor
    perm = np.array([2, 0, 3, 1])
    S = np.full((4, 4), -1.0)
    S[np.arange(4), perm] = 1e4
    K = ws.sinkhorn(S, iters=20)
    assert np.isfinite(K).all()
    np.testing.assert_allclose(K[np.arange(4), perm], 1.0, rtol=1e-12)
    off = np.ones((4, 4), bool)
    off[np.arange(4), perm] = False
    assert (K[off] <= 2.0 ** -99).all() and (K[off] > 0).all()
    # where nothing underflows the row shift changes nothing
    S = np.random.default_rng(5).normal(size=(6, 5))
    E = np.exp(S - S.max())
    for _ in range(4):
        E = E / E.sum(1, keepdims=True)
        E = E / E.sum(0, keepdims=True)
    np.testing.assert_allclose(ws.sinkhorn(S, iters=4), E, rtol=1e-13)


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -7.0, 1e-3])
    p1, m, v = ws.adam_step(p, np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=0, atol=1e-7)
