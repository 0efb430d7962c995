"""fastpfp_project_noalloc -- the projection entry point for callers that
may not allocate device memory (a plugin handed a fixed device-memory arena
by its host application, a real-time loop that forbids allocation after
start-up).  It must give what the handle-based fastpfp_project gives on the
same input, call after call, although every call reuses the same static
scratch array, and both must match the FP64 oracle's successive projection
(Section 4.3) run for the same number of rounds.

This file is collected last so that a failure here comes after every other
test has run; it also passes when run alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1207_1114_gb300 import fastpfp as F

pytestmark = pytest.mark.gpu


def _noalloc_raw(Y, tol, max_iter):
    """Straight through the C ABI, no Python helper in between."""
    lib = F.lib()
    it = C.c_int(-1)
    d = C.c_double(-1.0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fastpfp_project_noalloc(stream, C.c_void_p(Y.data_ptr()), Y.shape[0], float(tol),
                                     int(max_iter), C.byref(it), C.byref(d))
    return rc, it.value, d.value


# N = 3200: the band no longer fits in shared memory and the kernel streams
# it through L2 (the N range (2900, 4096] of this entry point)
@pytest.mark.parametrize("N,tol,rounds", [(1000, 0.0, 60), (256, 1e-5, 3000), (4, 0.0, 10),
                                          (3200, 0.0, 6)])
def test_noalloc_matches_handle_projection_and_oracle_twice(N, tol, rounds):
    rng = np.random.default_rng(N)
    with F.Solver(max_n=N) as s:
        for call in range(2):   # the second call starts from the first call's leftovers
            Y0 = (rng.random((N, N)) * (3.0 + call)).astype(np.float32)
            ref = torch.as_tensor(Y0, device="cuda:0")
            it_ref, d_ref = s.project(ref, tol=tol, max_iter=rounds)
            got = torch.as_tensor(Y0, device="cuda:0")
            rc, it, d = _noalloc_raw(got, tol, rounds)
            assert rc == F.FASTPFP_OK, F.error_string(rc)
            assert it == it_ref
            assert abs(d - d_ref) <= 2e-5
            assert (got - ref).abs().max().item() <= 2e-5
            want, _, _ = oracle.pd(Y0, fixed_iters=it)
            assert np.abs(got.cpu().numpy() - want).max() <= 2e-5


def test_noalloc_rejects_sizes_beyond_its_limit():
    big = torch.zeros((4100, 4100), device="cuda:0")
    rc, _, _ = _noalloc_raw(big, 0.0, 1)
    assert rc == F.FASTPFP_ERR_SIZE
    odd = torch.zeros((10, 10), device="cuda:0")
    rc, _, _ = _noalloc_raw(odd, 0.0, 1)
    assert rc == F.FASTPFP_ERR_ARG
