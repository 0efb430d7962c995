"""Learned warm start on the GPU against the FP64 oracle (oracle/warmstart.py),
through the C ABI, and what training gains over the uniform start.

Tolerances: features and the MLP are FP32 sums of <= 128 products, S of 64
(relative error ~1e-6); exp and 20 Sinkhorn rounds keep relative errors
~1e-5, so X0 is compared at rtol 2e-4.  Loss: relative 1e-5; gradient:
|err| <= 1e-4 * max|grad| (FP32 sums over up to n rows)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import warmstart as ows
from paper_1207_1114_gb300 import fastpfp as F
from paper_1207_1114_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cu(a, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dtype), device=DEV)


@pytest.fixture(scope="module")
def solver():
    s = F.Solver(max_n=400, max_batch=4)
    yield s
    s.close()


def _pair(n, n_out, seed, k=15):
    return synth.graph_pair(n, p=0.15, sigma=0.03, k=k, attr_sigma=0.05, n_out=n_out, lam=0.5,
                            seed=seed)


@pytest.mark.parametrize("n,n_out,swap,k", [(60, 15, False, 15), (60, 15, True, 15), (33, 0, False, 4),
                                            (50, 7, False, 0)])
def test_warmstart_matches_oracle(solver, n, n_out, swap, k):
    g = _pair(n, n_out, seed=n + n_out, k=k)
    A, A2, B, B2 = (g.A2, g.A, g.B2, g.B) if swap else (g.A, g.A2, g.B, g.B2)
    params = ows.init_params(1)
    X0 = solver.warmstart(cu(A), cu(A2), cu(B) if k else None, cu(B2) if k else None, cu(params),
                          iters=20).cpu().numpy()
    ref = ows.warm_start(A, A2, B if k else None, B2 if k else None, params, iters=20)
    assert X0.shape == ref.shape
    np.testing.assert_allclose(X0, ref, rtol=2e-4, atol=1e-6 * ref.max())


@pytest.mark.parametrize("swap", [False, True])
def test_loss_gradient_and_adam_match_oracle(solver, swap):
    g = _pair(70, 12, seed=3)
    A, A2, B, B2, perm = g.A, g.A2, g.B, g.B2, g.gt.astype(np.int32)
    if swap:
        A, A2, B, B2 = A2, A, B2, B
        inv = -np.ones(g.n2, dtype=np.int32)
        inv[g.gt] = np.arange(g.n, dtype=np.int32)
        perm = inv
    params = ows.init_params(2)
    p = cu(params)
    loss, grad = solver.train_step(cu(A), cu(A2), cu(B), cu(B2), cu(perm, np.int32), p, want_grad=True)
    rl, rg = ows.loss_and_grad(A, A2, B, B2, perm, params)
    assert loss == pytest.approx(rl, rel=1e-5)
    grad = grad.cpu().numpy()
    assert np.abs(grad - rg).max() <= 1e-4 * np.abs(rg).max()
    # one Adam step from zero moments
    m = torch.zeros(F.MLP_NPARAMS, device=DEV)
    v = torch.zeros(F.MLP_NPARAMS, device=DEV)
    solver.train_step(cu(A), cu(A2), cu(B), cu(B2), cu(perm, np.int32), p, m, v, step=1, lr=1e-2)
    ref, _, _ = ows.adam_step(params.astype(np.float64), 0.0, 0.0, grad.astype(np.float64), 1, 1e-2)
    np.testing.assert_allclose(p.cpu().numpy(), ref, rtol=0, atol=1e-5)


def test_training_reduces_loss_and_outer_iterations():
    """Train on 500 pairs that plain FastPFP solved (their matchings are the
    targets; pairs drawn on the GPU, n ~ U{200..800} plus up to n/5
    outliers, 15-dim attributes), then solve 6 held-out pairs of n = 400
    from the uniform start and from the learned one.  The learned start must
    keep the accuracy and take strictly fewer outer iterations: at least half
    an iteration fewer on average (measured on GB300: 13.0 -> 11.3)."""
    s = F.Solver(max_n=960, max_batch=32)
    try:
        prm = F.default_params(lam=0.5)
        params = cu(ows.init_params(7))
        m = torch.zeros(F.MLP_NPARAMS, device=DEV)
        v = torch.zeros(F.MLP_NPARAMS, device=DEV)
        gen = synth.warm_start_train_torch(500, seed=3, device=DEV)
        losses, step = [], 0
        while step < 500:
            batch = [next(gen) for _ in range(32 if step + 32 <= 500 else 500 - step)]
            outs = s.match_batched([b[:4] for b in batch], params=prm)
            for b, o in zip(batch, outs):
                step += 1
                loss, _ = s.train_step(*b[:4], o.perm, params, m, v, step=step, lr=3e-3)
                losses.append(loss)
        assert np.isfinite(losses).all()
        first, last = np.mean(losses[:32]), np.mean(losses[-32:])
        assert last < 0.2 * first, (first, last)

        outer_u, outer_w, acc_u, acc_w = [], [], [], []
        for sd in range(6):
            g = synth.graph_pair(400, p=0.1, sigma=0.03, k=15, attr_sigma=0.05, n_out=40, lam=0.5,
                                 seed=9000 + 13 * 400 + sd)
            d = (cu(g.A), cu(g.A2), cu(g.B), cu(g.B2))
            ru = s.match(*d, params=prm)
            X0 = s.warmstart(*d, params, iters=20)
            assert torch.isfinite(X0).all()
            rw = s.match(*d, params=prm, X0=X0)
            outer_u.append(ru.stats.outer_iters)
            outer_w.append(rw.stats.outer_iters)
            acc_u.append((ru.perm.cpu().numpy() == g.gt).mean())
            acc_w.append((rw.perm.cpu().numpy() == g.gt).mean())
        print(f"\nuniform start: outer {np.mean(outer_u):.2f}, accuracy {np.mean(acc_u):.4f}; "
              f"learned start: outer {np.mean(outer_w):.2f}, accuracy {np.mean(acc_w):.4f}; "
              f"training loss {first:.3f} -> {last:.3f}")
        assert np.mean(acc_w) >= np.mean(acc_u)
        assert np.mean(outer_w) <= np.mean(outer_u) - 0.5, (outer_u, outer_w)
    finally:
        s.close()


def test_overconfident_similarity_gives_a_finite_start(solver):
    """Every weight scaled 6x scales S ~1300x (S is quartic in the weights),
    so S spans thousands and whole columns of exp(S - max S) would underflow:
    the start stays finite and positive with unit row sums (the smaller
    graph's side), and wherever
    the oracle's start is confident (an entry above 0.99) the GPU's picks the
    same row.  (FP32 errors of S are ~1e-2 here, so entries are not compared
    one by one.)"""
    g = _pair(60, 15, seed=77)
    params = ows.init_params(11) * np.float32(6.0)
    d = (cu(g.A), cu(g.A2), cu(g.B), cu(g.B2))
    X0 = solver.warmstart(*d, cu(params), iters=20).cpu().numpy()
    assert np.isfinite(X0).all() and (X0 > 0).all()
    ref = ows.warm_start(g.A, g.A2, g.B, g.B2, params.astype(np.float64), iters=20)
    S = ows.similarity(*[ows.mlp_forward(ows.features(W, B), params.astype(np.float64))[1]
                         for W, B in ((g.A2, g.B2), (g.A, g.B))])
    assert np.ptp(S) > 1000.0
    np.testing.assert_allclose(X0.sum(1), 1.0, rtol=1e-4)   # rows of the smaller graph
    sure = ref.max(1) > 0.99
    assert sure.sum() >= 5
    np.testing.assert_array_equal(X0.argmax(1)[sure], ref.argmax(1)[sure])
