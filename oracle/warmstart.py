"""FP64 oracle of the learned warm start -- test infrastructure.

The paper notes that FastPFP's accuracy depends on the initial X (discussion
after Algorithm 1) and recommends the uniform start.  The warm start replaces
it by a learned similarity: per-node features -> shared MLP -> S = E E'^T / 8
-> Sinkhorn normalisation -> X(0).  It is trained on pairs that plain FastPFP
solved.  None of this is in the paper; the definitions below are this
project's and the CUDA kernels follow them.

Everything is plain numpy in float64, in canonical orientation (graph with
more nodes on the rows).  Only tests/ may import this module.

  features  F_i = [zscore(deg)_i, hist_i[0..15], zscore(B)_i[0..14]]    (32)
            deg_i = sum_j W_ij; hist_i[b] = #{j: W_ij != 0, bin(W_ij) = b} /
            max(#{j: W_ij != 0}, 1), bin(w) = min(15, max(0, floor(16 w)));
            zscore over the graph's nodes with the population std + 1e-6
  MLP       H = relu(F W1 + b1) (128), E = H W2 + b2 (64), shared weights
  S         E_big E_small^T / 8
  X(0)      K = max(exp(S - rowmax S), 2^-100), then `iters` times: rows /
            row sums, columns / column sums, each result floored at 2^-100
            (shifting each row by its own maximum is the same start as one
            global shift once rows are normalised; the floor keeps every row
            and column positive when a trained S is so peaked that whole
            columns would underflow -- it moves no entry above 2^-100)
  loss      t(j) = row matched to column j;
            L = -(1/m) sum_j [S[t(j),j] - logsumexp_i S[i,j]]
                -(1/m) sum_j [S[t(j),j] - logsumexp_j' S[t(j),j']]
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 32, 128, 64
NPARAMS = IN * HID + HID + HID * OUT + OUT


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + IN * HID].reshape(IN, HID); o += IN * HID
    b1 = p[o:o + HID]; o += HID
    W2 = p[o:o + HID * OUT].reshape(HID, OUT); o += HID * OUT
    b2 = p[o:o + OUT]
    return W1, b1, W2, b2


def init_params(seed=0):
    """He-style initialisation (the same numbers feed the GPU, as an input)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / IN), (IN, HID))
    W2 = rng.normal(0, np.sqrt(1.0 / HID), (HID, OUT))
    return np.concatenate([W1.ravel(), np.zeros(HID), W2.ravel(), np.zeros(OUT)]).astype(np.float32)


def _zscore(v):
    return (v - v.mean(axis=0)) / (v.std(axis=0) + 1e-6)


def features(W, B):
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    deg = W.sum(axis=1)
    nz = W != 0
    cnt = nz.sum(axis=1)
    bins = np.clip(np.floor(16.0 * W), 0, 15).astype(int)
    hist = np.zeros((n, 16))
    for b in range(16):
        hist[:, b] = (nz & (bins == b)).sum(axis=1)
    hist /= np.maximum(cnt, 1)[:, None]
    F = np.zeros((n, IN))
    F[:, 0] = _zscore(deg)
    F[:, 1:17] = hist
    if B is not None and np.asarray(B).shape[1] > 0:
        Bz = _zscore(np.asarray(B, dtype=np.float64))
        k = min(Bz.shape[1], 15)
        F[:, 17:17 + k] = Bz[:, :k]
    return F


def mlp_forward(F, params):
    W1, b1, W2, b2 = unpack(params)
    Z = F @ W1 + b1
    H = np.maximum(Z, 0.0)
    E = H @ W2 + b2
    return H, E


def similarity(E, E2):
    return E @ E2.T / 8.0


FLOOR = 2.0 ** -100


def sinkhorn(S, iters=20):
    K = np.maximum(np.exp(S - S.max(axis=1, keepdims=True)), FLOOR)
    for _ in range(iters):
        K = np.maximum(K / K.sum(axis=1, keepdims=True), FLOOR)
        K = np.maximum(K / K.sum(axis=0, keepdims=True), FLOOR)
    return K


def warm_start(A, A2, B, B2, params, iters=20):
    """X(0) in the caller's orientation (n_a x n_b)."""
    tr = A.shape[0] < A2.shape[0]
    Ab, As, Bb, Bs = (A2, A, B2, B) if tr else (A, A2, B, B2)
    _, E = mlp_forward(features(Ab, Bb), params)
    _, E2 = mlp_forward(features(As, Bs), params)
    X = sinkhorn(similarity(E, E2), iters)
    return X.T if tr else X


def _logsumexp(S, axis):
    m = S.max(axis=axis, keepdims=True)
    return (m + np.log(np.exp(S - m).sum(axis=axis, keepdims=True))).squeeze(axis)


def loss_and_grad(A, A2, B, B2, perm, params):
    """Loss and its gradient w.r.t. the parameter vector.  perm: n_a entries,
    node of graph 2 matched to node i of graph 1 (or -1)."""
    A = np.asarray(A, dtype=np.float64)
    A2 = np.asarray(A2, dtype=np.float64)
    perm = np.asarray(perm)
    tr = A.shape[0] < A2.shape[0]
    if tr:   # columns are graph 1: t(j) = perm[j]
        Ab, As, Bb, Bs = A2, A, B2, B
        t = perm.astype(int)
    else:    # columns are graph 2: t(perm[i]) = i
        Ab, As, Bb, Bs = A, A2, B, B2
        t = np.full(A2.shape[0], -1)
        for i, j in enumerate(perm):
            if j >= 0:
                t[j] = i
    W1, b1, W2, b2 = unpack(params)
    Fb, Fs = features(Ab, Bb), features(As, Bs)
    Hb, Eb = mlp_forward(Fb, params)
    Hs, Es = mlp_forward(Fs, params)
    S = similarity(Eb, Es)
    N, m = S.shape
    cols = np.arange(m)
    lse_c = _logsumexp(S, 0)                 # per column
    lse_r = _logsumexp(S[t], 1)              # per matched row
    st = S[t, cols]
    loss = -(np.sum(st - lse_c) + np.sum(st - lse_r)) / m
    # dL/dS
    Pc = np.exp(S - lse_c[None, :])          # column softmax
    dS = Pc / m
    dS[t, cols] -= 1.0 / m
    Pr = np.exp(S[t] - lse_r[:, None])       # row softmax of matched rows
    dS[t] += Pr / m
    dS[t, cols] -= 1.0 / m
    # through S = Eb Es^T / 8
    dEb = dS @ Es / 8.0
    dEs = dS.T @ Eb / 8.0
    gW1 = np.zeros_like(W1); gb1 = np.zeros_like(b1)
    gW2 = np.zeros_like(W2); gb2 = np.zeros_like(b2)
    for F, H, dE in ((Fb, Hb, dEb), (Fs, Hs, dEs)):
        gW2 += H.T @ dE
        gb2 += dE.sum(axis=0)
        dH = (dE @ W2.T) * (H > 0)
        gW1 += F.T @ dH
        gb1 += dH.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])
    return loss, grad


def adam_step(params, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
