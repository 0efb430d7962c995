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


def test_training_reduces_loss_and_outer_iterations(solver):
    """Train on pairs solved by plain FastPFP (their matchings are the
    targets), then compare warm-started and uniform-start solves on held-out
    pairs: the trained start must not lose accuracy, and the gain in outer
    iterations is reported."""
    rng = np.random.default_rng(0)
    prm = F.default_params(lam=0.5, max_outer=60, max_inner=300)
    train = []
    for s in range(16):
        g = _pair(int(rng.integers(80, 160)), int(rng.integers(0, 20)), seed=1000 + s)
        d = (cu(g.A), cu(g.A2), cu(g.B), cu(g.B2))
        r = solver.match(*d, params=prm)
        train.append((d, r.perm))
    params = cu(ows.init_params(7))
    m = torch.zeros(F.MLP_NPARAMS, device=DEV)
    v = torch.zeros(F.MLP_NPARAMS, device=DEV)
    losses = []
    for step in range(1, 241):
        d, perm = train[step % len(train)]
        loss, _ = solver.train_step(*d, perm, params, m, v, step=step, lr=3e-3)
        losses.append(loss)
    first, last = np.mean(losses[:16]), np.mean(losses[-16:])
    assert last < 0.5 * first, (first, last)

    outer_u, outer_w, acc_u, acc_w = [], [], [], []
    for s in range(6):
        g = _pair(int(rng.integers(80, 160)), int(rng.integers(0, 20)), seed=5000 + s)
        d = (cu(g.A), cu(g.A2), cu(g.B), cu(g.B2))
        ru = solver.match(*d, params=prm)
        X0 = solver.warmstart(*d, params, iters=20)
        rw = solver.match(*d, params=prm, X0=X0)
        outer_u.append(ru.stats.outer_iters)
        outer_w.append(rw.stats.outer_iters)
        acc_u.append((ru.perm.cpu().numpy() == g.gt).mean())
        acc_w.append((rw.perm.cpu().numpy() == g.gt).mean())
    print(f"\nuniform start: outer {np.mean(outer_u):.1f}, accuracy {np.mean(acc_u):.4f}; "
          f"learned start: outer {np.mean(outer_w):.1f}, accuracy {np.mean(acc_w):.4f}; "
          f"training loss {first:.3f} -> {last:.3f}")
    assert np.mean(acc_w) >= np.mean(acc_u) - 0.02
    assert np.mean(outer_w) <= np.mean(outer_u) + 1.0
