"""Seeded synthetic graph pairs shaped like the paper's experiments.

This module only draws inputs.  It holds none of FastPFP's arithmetic, so both
the CUDA path and the FP64 oracle consume exactly the same arrays from it.

Recipe (Section 5.1 builds random graphs and hides a ground-truth
correspondence; the weighted / attributed / outlier variants follow the
weighted real-image and 3D experiments of Sections 5.2-5.4):

* graph 1: ``n`` nodes, each unordered pair {i, j} (i != j) is an edge with
  probability ``p``; edge weight ~ U(0, 1); symmetric; zero diagonal.
* inlier copy: the same matrix plus symmetric N(0, sigma^2) noise on the
  existing edges only (the sparsity pattern is kept, weights are not clipped).
* outliers: ``n_out`` extra nodes in graph 2; every pair that touches an
  outlier is an edge with probability ``p_out`` (default ``p``), weight U(0,1).
* a uniformly random permutation of all ``n + n_out`` nodes of graph 2 hides
  the correspondence; ``gt[i]`` is the node of graph 2 matched to node i.
* attributes: ``B`` ~ N(0, 1) of shape n x k; inlier rows of ``B2`` are the
  matched rows of ``B`` plus N(0, attr_sigma^2); outlier rows ~ N(0, 1).

All arrays are float32 (the GPU path's input type); the oracle widens the
same values to float64.  numpy's PCG64 generator, seeded per pair.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GraphPair:
    A: np.ndarray      # n x n float32, symmetric
    A2: np.ndarray     # n2 x n2 float32, symmetric
    B: np.ndarray      # n x k float32
    B2: np.ndarray     # n2 x k float32
    gt: np.ndarray     # n int32, node of graph 2 matched to node i of graph 1
    lam: float         # lambda the workload uses

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def n2(self) -> int:
        return self.A2.shape[0]

    @property
    def k(self) -> int:
        return self.B.shape[1]


def random_graph(rng: np.random.Generator, n: int, p: float) -> np.ndarray:
    """Symmetric weighted Bernoulli(p) graph with U(0,1) weights, zero diagonal."""
    mask = np.triu(rng.random((n, n)) < p, 1)
    w = np.triu(rng.random((n, n)), 1) * mask
    return w + w.T


def graph_pair(n: int, *, p: float, sigma: float, k: int = 0, attr_sigma: float = 0.05,
               n_out: int = 0, p_out: float | None = None, lam: float = 0.0,
               seed: int = 0) -> GraphPair:
    rng = np.random.default_rng(seed)
    A = random_graph(rng, n, p)
    noise = np.triu(rng.normal(0.0, sigma, (n, n)), 1) if sigma > 0 else np.zeros((n, n))
    noise = (noise + noise.T) * (A != 0)
    n2 = n + n_out
    M = np.zeros((n2, n2))
    M[:n, :n] = A + noise
    if n_out > 0:
        po = p if p_out is None else p_out
        O = random_graph(rng, n2, po)
        M[n:, :] = O[n:, :]
        M[:, n:] = O[:, n:]
    perm2 = rng.permutation(n2)
    A2 = np.zeros((n2, n2))
    A2[np.ix_(perm2, perm2)] = M
    if k > 0:
        B = rng.normal(0.0, 1.0, (n, k))
        MB = np.empty((n2, k))
        MB[:n] = B + rng.normal(0.0, attr_sigma, (n, k))
        if n_out > 0:
            MB[n:] = rng.normal(0.0, 1.0, (n_out, k))
        B2 = np.empty((n2, k))
        B2[perm2] = MB
    else:
        B = np.zeros((n, 0))
        B2 = np.zeros((n2, 0))
    return GraphPair(A.astype(np.float32), A2.astype(np.float32), B.astype(np.float32),
                     B2.astype(np.float32), perm2[:n].astype(np.int32), float(lam))


# Workload presets.  Sizes, densities and noise levels are those of the
# plain / attributed / partial / batched / large workloads; the seed picks
# the instance.

def plain_100(seed: int = 0, sigma: float = 0.02) -> GraphPair:
    """n = n' = 100, p = 0.3, U(0,1) weights, edge noise sigma, no attributes."""
    return graph_pair(100, p=0.3, sigma=sigma, k=0, lam=0.0, seed=seed)


def attributed_1000(seed: int = 0, n: int = 1000) -> GraphPair:
    """n = n' = 1000, p = 0.1, edge noise 0.05, 16-dim N(0,1) attributes with
    N(0, 0.05^2) noise, lambda = 1."""
    return graph_pair(n, p=0.1, sigma=0.05, k=16, attr_sigma=0.05, lam=1.0, seed=seed)


def partial_1000_1200(seed: int = 0, n: int = 1000, n_out: int = 200) -> GraphPair:
    """1000 inliers into 1200 nodes: edge noise 0.03, 200 outliers with p=0.1
    edges, 16-dim attributes, lambda = 0.5."""
    return graph_pair(n, p=0.1, sigma=0.03, k=16, attr_sigma=0.05, n_out=n_out, lam=0.5, seed=seed)


def batch_mixed_sizes(count: int = 512, seed: int = 0, n_lo: int = 50, n_hi: int = 600,
                      out_hi: int = 100) -> list[tuple[int, int]]:
    """(n, outliers) of every pair of batch_mixed(count, seed, ...), drawn
    without generating the graphs."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    outs = rng.integers(0, out_hi + 1, size=count)
    return [(int(ns[b]), int(outs[b])) for b in range(count)]


def batch_mixed_pair(b: int, n: int, n_out: int, seed: int = 0) -> GraphPair:
    """Pair b of batch_mixed(..., seed) given its drawn (n, outliers)."""
    return graph_pair(n, p=0.15, sigma=0.03, k=8, attr_sigma=0.05, n_out=n_out, lam=0.5,
                      seed=seed * 100003 + b + 1)


def batch_mixed(count: int = 512, seed: int = 0, n_lo: int = 50, n_hi: int = 600,
                out_hi: int = 100) -> list[GraphPair]:
    """Batch of pairs with n ~ U{n_lo..n_hi}, n' = n + U{0..out_hi} outliers,
    p = 0.15, noise 0.03, 8-dim attributes, lambda = 0.5."""
    sizes = batch_mixed_sizes(count, seed, n_lo, n_hi, out_hi)
    return [batch_mixed_pair(b, n, o, seed) for b, (n, o) in enumerate(sizes)]


def large_4000(seed: int = 0, n: int = 4000) -> GraphPair:
    """n = n' = 4000, p = 0.05, edge noise 0.05, 15-dim attributes, lambda = 0.5."""
    return graph_pair(n, p=0.05, sigma=0.05, k=15, attr_sigma=0.05, lam=0.5, seed=seed)


def warm_start_train(count: int, seed: int = 0, n_lo: int = 200, n_hi: int = 800) -> list[GraphPair]:
    """Training pairs for the learned warm start, shaped like the partial
    workload: n ~ U{n_lo..n_hi} inliers plus up to n/5 outliers, p = 0.1,
    sigma = 0.03, 15-dim attributes, lambda = 0.5."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    return [graph_pair(int(n), p=0.1, sigma=0.03, k=15, attr_sigma=0.05,
                       n_out=int(rng.integers(0, int(n) // 5 + 1)), lam=0.5,
                       seed=seed * 1000003 + b + 1) for b, n in enumerate(ns)]


def e1_pair(n: int, case: str, seed: int = 0) -> GraphPair:
    """Section 5.1's synthetic random graphs: unweighted, each pair {i, j} an
    edge with probability 1/2, and graph 2 a hidden relabelling of graph 1
    with (case 'a') no change, ('b') n edge editions — n distinct pairs
    {i, j} whose edge is flipped (present <-> absent) —, ('c') 10 % of the
    nodes deleted (floor(n / 10) nodes; subgraph isomorphism), or ('d')
    both.  gt[i] is node i's label in graph 2, -1 for a deleted node.  No
    attributes (lambda = 0)."""
    if case not in ("a", "b", "c", "d"):
        raise ValueError("case is one of 'a', 'b', 'c', 'd'")
    rng = np.random.default_rng(seed)
    up = np.triu(rng.random((n, n)) < 0.5, 1)
    A = (up | up.T).astype(np.float32)
    A2 = A.copy()
    if case in ("b", "d"):
        iu, ju = np.triu_indices(n, 1)
        pick = rng.choice(len(iu), size=min(n, len(iu)), replace=False)
        i, j = iu[pick], ju[pick]
        A2[i, j] = 1.0 - A2[i, j]
        A2[j, i] = A2[i, j]
    keep = np.arange(n)
    if case in ("c", "d"):
        keep = np.sort(rng.choice(n, size=n - n // 10, replace=False))
    A2 = A2[np.ix_(keep, keep)]
    m = len(keep)
    label = rng.permutation(m)           # node keep[t] of graph 1 is node label[t] of graph 2
    A2p = np.zeros_like(A2)
    A2p[np.ix_(label, label)] = A2
    gt = np.full(n, -1, dtype=np.int32)
    gt[keep] = label
    return GraphPair(A, A2p, np.zeros((n, 0), np.float32), np.zeros((m, 0), np.float32), gt, 0.0)


def graph_pair_torch(n: int, *, p: float, sigma: float, k: int, attr_sigma: float, n_out: int,
                     generator, device):
    """graph_pair's recipe drawn with torch on `device` (for the learned warm
    start's training pairs, which are generated, solved and consumed on the
    GPU in chunks; never compared with the oracle).  Returns float32 tensors
    (A, A2, B, B2) and the int32 ground truth gt."""
    import torch
    kw = dict(generator=generator, device=device)

    def rgraph(m, pp):
        up = torch.triu((torch.rand((m, m), **kw) < pp).float() * torch.rand((m, m), **kw), 1)
        return up + up.T

    A = rgraph(n, p)
    noise = torch.triu(torch.randn((n, n), **kw) * sigma, 1)
    noise = (noise + noise.T) * (A != 0)
    n2 = n + n_out
    M = torch.zeros((n2, n2), device=device)
    M[:n, :n] = A + noise
    if n_out > 0:
        O = rgraph(n2, p)
        M[n:, :] = O[n:, :]
        M[:, n:] = O[:, n:]
    perm2 = torch.randperm(n2, **kw)
    A2 = torch.zeros((n2, n2), device=device)
    A2[perm2[:, None], perm2[None, :]] = M
    B = torch.randn((n, k), **kw)
    MB = torch.empty((n2, k), device=device)
    MB[:n] = B + torch.randn((n, k), **kw) * attr_sigma
    if n_out > 0:
        MB[n:] = torch.randn((n_out, k), **kw)
    B2 = torch.empty((n2, k), device=device)
    B2[perm2] = MB
    return A.contiguous(), A2.contiguous(), B.contiguous(), B2.contiguous(), perm2[:n].to(torch.int32)


def warm_start_train_torch(count: int, seed: int, device, n_lo: int = 200, n_hi: int = 800):
    """Yields the `count` training pairs of the learned warm start (shaped like
    warm_start_train: n ~ U{n_lo..n_hi} inliers plus up to n/5 outliers,
    p = 0.1, sigma = 0.03, 15-dim attributes), drawn on `device` one at a
    time from a seeded torch generator."""
    import torch
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        n_out = int(rng.integers(0, n // 5 + 1))
        yield graph_pair_torch(n, p=0.1, sigma=0.03, k=15, attr_sigma=0.05, n_out=n_out,
                               generator=gen, device=device)
