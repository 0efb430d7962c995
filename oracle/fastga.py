"""FP64 oracle of FastGA -- test infrastructure.

FastGA is graduated assignment with the compatibility C_aibj = A_ij A'_ab,
for which the soft-assignment's O(n^4) sum Q_ia = sum_{j,b} C X (Eq. GAO4)
becomes the product Q = A X A' (Eq. GAO3), an O(n^3) step (Appendix).  With
the attribute term of Eq. (3) the soft-assignment's argument is the same
gradient FastPFP uses, Q = A X A' + lambda K.  The experiments of Section 5
run it with two loops and the stopping rules of FastPFP: the soft-assignment
(outer) loop stops when max|X(t+1) - X(t)| < eps_1 or after I_0 iterations,
the normalisation (inner) loop when max|Y(k+1) - Y(k)| < eps_2 or after I_1
iterations; the result is discretised by the same greedy rule.

The paper gives neither beta nor an annealing schedule.  Reading used here
(and by the CUDA path): beta is fixed for a solve (a parameter) and applies
to Q divided by its largest magnitude, so that one beta serves graphs whose
products differ in scale (Q grows with n and the edge density; an absolute
beta that suits weighted sparse pairs leaves dense unweighted ones with no
soft-assignment at all); the start is FastPFP's uniform X, and graphs of
different sizes are handled as in FastPFP's slacked projection -- the larger
graph's N nodes are the rows, the smaller graph's m nodes the first m of N
columns, and the N - m slack columns (dummy nodes) take Q = 0.  One outer
iteration, with s = max |Q| (1 if Q = 0):

  Y(0)   = max(exp(beta (Q/s - rowmax Q/s)), 2^-100)    over the N x N Q
           (a per-row factor does not change the normalised result; the
           floor keeps every row and column positive where exp underflows)
  Y(k+1) = C(R(Y(k))),  R: rows divided by their sums, C: columns divided
           by their sums, each result floored at 2^-100
  X(t+1) = Y[:, :m] at the inner loop's end.

Only tests/ (and bench.py's oracle legs) may import this module.  Plain
numpy in float64; the products and the greedy rule are the oracle's own
pinned routines (oracle.gradient, oracle.greedy_literal).
"""
from __future__ import annotations

import numpy as np

from . import affinity, error_objective, gradient, greedy_literal, qap_objective

FLOOR = 2.0 ** -100


def soft_assign(Q, beta):
    """Y(0) of the inner loop from the N x N argument Q (slack columns
    included), scaled by its largest magnitude."""
    Q = np.asarray(Q, dtype=np.float64)
    s = float(np.abs(Q).max())
    Q = Q / (s if s > 0 else 1.0)
    return np.maximum(np.exp(beta * (Q - Q.max(axis=1, keepdims=True))), FLOOR)


def normalise_step(Y):
    """One inner iteration: rows to unit sums, then columns, floored."""
    Z = np.maximum(Y / Y.sum(axis=1, keepdims=True), FLOOR)
    return np.maximum(Z / Z.sum(axis=0, keepdims=True), FLOOR)


def normalise(Y, tol=1e-6, max_iter=1000, fixed_iters=0):
    """The inner loop: normalise_step until max|Y(k+1) - Y(k)| < tol or
    max_iter steps (exactly fixed_iters steps when it is > 0).  Returns
    (Y, steps, last change)."""
    k, d = 0, np.inf
    cap = fixed_iters if fixed_iters > 0 else max_iter
    while k < cap:
        Yn = normalise_step(Y)
        d = float(np.abs(Yn - Y).max())
        Y = Yn
        k += 1
        if fixed_iters <= 0 and d < tol:
            break
    return Y, k, d


def solve(A, A2, B=None, B2=None, lam=0.0, beta=100.0, tol_outer=1e-6, tol_inner=1e-6,
          max_outer=100, max_inner=1000, X0=None, replay_inner=None):
    """FastGA end to end in the caller's orientation; the same dict as
    oracle.solve (perm, X, inner / delta traces, stats).  replay_inner:
    run exactly replay_inner[t] inner iterations in outer iteration t (to
    follow a run whose inner counts are known)."""
    A_in = np.asarray(A, dtype=np.float64)
    A2_in = np.asarray(A2, dtype=np.float64)
    n_a, n_b = A_in.shape[0], A2_in.shape[0]
    transposed = n_a < n_b
    A, A2 = (A2_in, A_in) if transposed else (A_in, A2_in)
    has_k = B is not None and B2 is not None and np.asarray(B).ndim == 2 and np.asarray(B).shape[1] > 0
    if has_k:
        Bc, B2c = (B2, B) if transposed else (B, B2)
        K = affinity(np.asarray(Bc, np.float64), np.asarray(B2c, np.float64))
    else:
        K = None
    N, m = A.shape[0], A2.shape[0]
    if X0 is not None:
        X = np.array(X0, dtype=np.float64)
        if transposed:
            X = X.T.copy()
    else:
        X = np.full((N, m), 1.0 / (N * m))
    if replay_inner is not None:
        replay_inner = np.asarray(replay_inner, dtype=np.int64)
        if (replay_inner < 1).any():
            raise ValueError("replay_inner needs a positive inner count per outer iteration")
    inner, delta = [], []
    converged = False
    for t in range(max_outer):
        Q = np.zeros((N, N))
        Q[:, :m] = gradient(A, X, A2, K, lam)
        fixed = int(replay_inner[t]) if replay_inner is not None and t < len(replay_inner) else 0
        Y, k, _ = normalise(soft_assign(Q, beta), tol_inner, max_inner, fixed)
        Xn = Y[:, :m].copy()
        d = float(np.abs(Xn - X).max())
        X = Xn
        inner.append(k)
        delta.append(d)
        if d < tol_outer:
            converged = True
            break
    row_of_col = greedy_literal(X)
    if transposed:
        perm = np.asarray(row_of_col, dtype=np.int32).copy()
        X_out = X.T.copy()
    else:
        perm = np.full(n_a, -1, dtype=np.int32)
        perm[row_of_col] = np.arange(m, dtype=np.int32)
        X_out = X
    Bk = (np.asarray(Bc, np.float64), np.asarray(B2c, np.float64)) if has_k else (None, None)
    return dict(perm=perm, X=X_out, inner=np.array(inner, dtype=np.int32), delta=np.array(delta),
                outer_iters=len(inner), inner_total=int(sum(inner)), inner_max=int(max(inner) if inner else 0),
                converged=converged, transposed=transposed, final_delta=delta[-1] if delta else 0.0,
                objective=qap_objective(A, A2, row_of_col, K, lam),
                error=error_objective(A, A2, row_of_col, Bk[0], Bk[1], lam))
