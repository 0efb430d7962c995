"""FastGA on the GPU (csrc/fastga.cu through the C ABI) against its FP64
oracle (oracle/fastga.py).

Tolerances.  The products are FP32 (|err| <~ 3e-5 of |A||X||A'|, the
split-TF32 bound), so beta Q / max|Q| carries up to ~3e-3 absolute error at
beta = 100; exp turns it into that relative error of Y(0) at worst, which
the normalisation keeps relative (typical errors are ~100 times smaller).  X entries are at most 1, so X is compared at
the FP32 X bound of FastPFP's tests, max-abs 1e-4, after a few replayed
outer iterations (errors do not grow: each outer iteration starts from the
normalised soft assignment; measured on GB300 ~2e-6), with the GPU's inner
counts replayed by the oracle.  The column sums are exact
integer sums, so a solve gives the same bits every run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import fastga as oga
from paper_1207_1114_gb300 import fastpfp as F
from paper_1207_1114_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


def dev_pair(g):
    return (cu(g.A), cu(g.A2), cu(g.B) if g.k else None, cu(g.B2) if g.k else None)


@pytest.fixture(scope="module")
def solver():
    s = F.Solver(max_n=300, max_batch=4)
    yield s
    s.close()


def ga_params(**kw):
    base = dict(algorithm=F.ALG_FASTGA, beta=100.0, max_outer=100, max_inner=1000)
    base.update(kw)
    return F.default_params(**base)


@pytest.mark.parametrize("case", ["plain", "partial", "transposed"])
@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_fastga_matches_oracle_replay(solver, case, precision):
    if case == "plain":
        g = synth.graph_pair(60, p=0.3, sigma=0.02, k=0, seed=3)
    else:
        g = synth.graph_pair(48, p=0.3, sigma=0.02, k=6, n_out=12, lam=0.5, seed=5)
    A, A2, B, B2 = g.A, g.A2, g.B, g.B2
    if case == "transposed":   # graph 1 the larger one
        A, A2, B, B2 = g.A2, g.A, g.B2, g.B
    prec = F.FP32 if precision == "fp32" else F.FP32_SIMT
    prm = ga_params(lam=g.lam, max_outer=5, max_inner=400, precision=prec)
    d = (cu(A), cu(A2), cu(B) if g.k else None, cu(B2) if g.k else None)
    r = solver.match(*d, params=prm, want_X=True)
    inner, _ = solver.last_trace()
    t = r.stats.outer_iters
    assert 1 <= t <= 5 and (inner[:t] >= 1).all()
    ref = oga.solve(A, A2, B if g.k else None, B2 if g.k else None, lam=g.lam, beta=100.0,
                    max_outer=t, max_inner=400, replay_inner=inner[:t])
    X = r.X.cpu().numpy()
    err = np.abs(X - ref["X"]).max()
    print(f"\nFastGA {case} {precision}: {t} outer iterations, max|X - X_oracle| = {err:.2e}")
    assert err <= 1e-4
    np.testing.assert_array_equal(r.perm.cpu().numpy(), ref["perm"])


def test_fastga_free_run_recovers_the_ground_truth_like_the_oracle(solver):
    """Free runs (the GPU's own stopping decisions): same permutation as the
    oracle's free run, and both recover the hidden correspondence."""
    for seed in range(3):
        g = synth.graph_pair(80, p=0.3, sigma=0.0, k=0, seed=seed)
        r = solver.match(*dev_pair(g), params=ga_params())
        ref = oga.solve(g.A, g.A2, beta=100.0)
        perm = r.perm.cpu().numpy()
        np.testing.assert_array_equal(ref["perm"], g.gt)
        np.testing.assert_array_equal(perm, g.gt)
        assert r.stats.converged
        assert abs(r.stats.outer_iters - ref["outer_iters"]) <= 2


def test_fastga_is_bit_reproducible_and_batches_equal_single_solves(solver):
    pairs = [synth.graph_pair(n, p=0.3, sigma=0.03, k=4, n_out=o, lam=0.5, seed=10 + n)
             for n, o in ((50, 0), (40, 9), (64, 3))]
    prm = ga_params(lam=0.5, max_outer=8, max_inner=300)
    singles = [solver.match(*dev_pair(g), params=prm, want_X=True) for g in pairs]
    again = solver.match(*dev_pair(pairs[0]), params=prm, want_X=True)
    assert torch.equal(again.X, singles[0].X) and torch.equal(again.perm, singles[0].perm)
    batch = solver.match_batched([dev_pair(g) for g in pairs], params=prm, want_X=True)
    for a, b in zip(batch, singles):
        assert torch.equal(a.X, b.X) and torch.equal(a.perm, b.perm)
        assert a.stats.outer_iters == b.stats.outer_iters


def test_fastga_rejects_what_it_does_not_run(solver):
    g = synth.graph_pair(20, p=0.3, sigma=0.0, k=0, seed=1)
    for bad in (ga_params(beta=0.0), ga_params(beta=float("nan")), ga_params(precision=F.BF16)):
        with pytest.raises(F.FastPFPError) as e:
            solver.match(*dev_pair(g), params=bad)
        assert e.value.code == F.FASTPFP_ERR_ARG
