"""FP64 CPU oracle for FastPFP -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It is a
ctypes front end to ``fastpfp_oracle.c`` (plain C, FP64, OpenMP), built here
with gcc.  It shares no code with the CUDA library and never calls it.

Every wrapper takes numpy arrays in the orientation documented in
``fastpfp_oracle.h`` and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fastpfp_oracle.c")
_HDR = os.path.join(_HERE, "fastpfp_oracle.h")
_LIB = os.path.join(_HERE, "liborc_fastpfp.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP contraction off so x86
    and Arm builds round identically).  Returns the library path."""
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class orc_params(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("alpha", C.c_double), ("tol_outer", C.c_double),
                ("tol_inner", C.c_double), ("max_outer", C.c_int), ("max_inner", C.c_int),
                ("normalize_max", C.c_int), ("slack_policy", C.c_int), ("algorithm", C.c_int)]


class orc_stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_total", C.c_int), ("inner_max", C.c_int),
                ("converged", C.c_int), ("transposed", C.c_int), ("final_delta", C.c_double),
                ("objective", C.c_double), ("error", C.c_double)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            l.orc_num_threads.restype = C.c_int
            l.orc_set_num_threads.argtypes = [C.c_int]
            l.orc_affinity.argtypes = [_D, _D, C.c_int, C.c_int, C.c_int, _D]
            l.orc_gradient.argtypes = [_D, _D, _D, _D, C.c_double, C.c_int, C.c_int, _D]
            l.orc_p1.argtypes = [_D, C.c_int]
            l.orc_p2.argtypes = [_D, C.c_int]
            l.orc_pd.argtypes = [_D, C.c_int, C.c_double, C.c_int, C.c_int, _D]
            l.orc_pd.restype = C.c_int
            l.orc_blend.argtypes = [_D, _D, C.c_int, C.c_int, C.c_double, C.c_int]
            l.orc_blend.restype = C.c_double
            l.orc_greedy_literal.argtypes = [_D, C.c_int, C.c_int, _I]
            l.orc_greedy_sorted.argtypes = [_D, C.c_int, C.c_int, _I]
            l.orc_qap_objective.argtypes = [_D, _D, _D, C.c_double, _I, C.c_int, C.c_int]
            l.orc_qap_objective.restype = C.c_double
            l.orc_error_objective.argtypes = [_D, _D, _D, _D, C.c_int, C.c_double, _I, C.c_int,
                                              C.c_int]
            l.orc_error_objective.restype = C.c_double
            l.orc_relaxed_objective.argtypes = [_D, _D, _D, C.c_double, _D, C.c_int, C.c_int]
            l.orc_relaxed_objective.restype = C.c_double
            l.orc_solve.argtypes = [_D, C.c_int, _D, C.c_int, _D, _D, C.c_int,
                                    C.POINTER(orc_params), _D, _I, C.c_int, _I, _D, _I, _D,
                                    C.POINTER(orc_stats)]
            l.orc_solve.restype = C.c_int
            _lib = l
    return _lib


def _d(a):
    """Contiguous float64 copy (or view) of ``a`` and its ctypes pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def affinity(B, B2):
    B, pb = _d(B)
    B2, pb2 = _d(B2)
    N, k = B.shape
    m = B2.shape[0]
    K = np.empty((N, m))
    lib().orc_affinity(pb, pb2, N, m, k, _dp(K))
    return K


def gradient(A, X, A2, K=None, lam=0.0):
    A, pa = _d(A)
    X, px = _d(X)
    A2, pa2 = _d(A2)
    N, m = X.shape
    Kp = None
    if K is not None:
        K, Kp = _d(K)
    G = np.empty((N, m))
    lib().orc_gradient(pa, px, pa2, Kp, float(lam), N, m, _dp(G))
    return G


def p1(Y):
    Y = np.array(Y, dtype=np.float64, order="C", copy=True)
    lib().orc_p1(_dp(Y), Y.shape[0])
    return Y


def p2(Y):
    Y = np.array(Y, dtype=np.float64, order="C", copy=True)
    lib().orc_p2(_dp(Y), Y.shape[0])
    return Y


def pd(Y, tol=1e-6, max_iter=1000, fixed_iters=0):
    """Successive projection; returns (Y_out, iterations, last_delta)."""
    Y = np.array(Y, dtype=np.float64, order="C", copy=True)
    last = C.c_double(0.0)
    it = lib().orc_pd(_dp(Y), Y.shape[0], float(tol), int(max_iter), int(fixed_iters),
                      C.byref(last))
    return Y, it, last.value


def blend(X, Y, alpha=0.5, normalize=True):
    """Returns (X_new, max|dX|)."""
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    Y, py = _d(Y)
    N, m = X.shape
    d = lib().orc_blend(_dp(X), py, N, m, float(alpha), int(bool(normalize)))
    return X, d


def greedy_literal(X):
    X, px = _d(X)
    N, m = X.shape
    out = np.empty(m, dtype=np.int32)
    lib().orc_greedy_literal(px, N, m, out.ctypes.data_as(_I))
    return out


def greedy_sorted(X):
    X, px = _d(X)
    N, m = X.shape
    out = np.empty(m, dtype=np.int32)
    lib().orc_greedy_sorted(px, N, m, out.ctypes.data_as(_I))
    return out


def qap_objective(A, A2, row_of_col, K=None, lam=0.0):
    A, pa = _d(A)
    A2, pa2 = _d(A2)
    r = np.ascontiguousarray(row_of_col, dtype=np.int32)
    Kp = None
    if K is not None:
        K, Kp = _d(K)
    return lib().orc_qap_objective(pa, pa2, Kp, float(lam), r.ctypes.data_as(_I), A.shape[0],
                                   A2.shape[0])


def error_objective(A, A2, row_of_col, B=None, B2=None, lam=0.0):
    A, pa = _d(A)
    A2, pa2 = _d(A2)
    r = np.ascontiguousarray(row_of_col, dtype=np.int32)
    k = 0
    pb = pb2 = None
    if B is not None and B2 is not None and B.shape[1] > 0:
        B, pb = _d(B)
        B2, pb2 = _d(B2)
        k = B.shape[1]
    return lib().orc_error_objective(pa, pa2, pb, pb2, k, float(lam), r.ctypes.data_as(_I),
                                     A.shape[0], A2.shape[0])


def relaxed_objective(A, A2, X, K=None, lam=0.0):
    A, pa = _d(A)
    A2, pa2 = _d(A2)
    X, px = _d(X)
    Kp = None
    if K is not None:
        K, Kp = _d(K)
    return lib().orc_relaxed_objective(pa, pa2, Kp, float(lam), px, X.shape[0], X.shape[1])


def solve(A, A2, B=None, B2=None, lam=0.0, alpha=0.5, tol_outer=1e-6, tol_inner=1e-6,
          max_outer=100, max_inner=1000, normalize_max=True, slack_policy=0, X0=None,
          replay_inner=None, replay_outer=0, algorithm="fastpfp"):
    """Algorithm 1 end to end in the caller's orientation (algorithm="pg":
    the projected gradient method of Eq. (pg) in the same loop).

    Returns a dict with ``perm`` (n_a entries, -1 for unmatched), ``X``
    (n_a x n_b), ``inner`` and ``delta`` traces and the stats fields."""
    A, pa = _d(A)
    A2, pa2 = _d(A2)
    n_a, n_b = A.shape[0], A2.shape[0]
    k = 0
    pb = pb2 = None
    if B is not None and B2 is not None and np.asarray(B).ndim == 2 and np.asarray(B).shape[1] > 0:
        B, pb = _d(B)
        B2, pb2 = _d(B2)
        k = B.shape[1]
    if algorithm not in ("fastpfp", "pg"):
        raise ValueError("algorithm is 'fastpfp' or 'pg'")
    prm = orc_params(float(lam), float(alpha), float(tol_outer), float(tol_inner), int(max_outer),
                     int(max_inner), int(bool(normalize_max)), int(slack_policy),
                     1 if algorithm == "pg" else 0)
    cap = max(int(max_outer), int(replay_outer))
    X0p = None
    if X0 is not None:
        X0, X0p = _d(X0)
    rip = None
    if replay_inner is not None:
        replay_inner = np.ascontiguousarray(replay_inner, dtype=np.int32)
        need = int(replay_outer) if int(replay_outer) > 0 else int(max_outer)
        if len(replay_inner) < need or (replay_inner[:need] < 1).any():
            raise ValueError("replay_inner needs a positive inner count for every outer iteration "
                             "the replay runs")
        rip = replay_inner.ctypes.data_as(_I)
    perm = np.empty(n_a, dtype=np.int32)
    X = np.empty((n_a, n_b))
    inner = np.zeros(cap, dtype=np.int32)
    delta = np.zeros(cap)
    st = orc_stats()
    rc = lib().orc_solve(pa, n_a, pa2, n_b, pb, pb2, k, C.byref(prm), X0p, rip, int(replay_outer),
                         perm.ctypes.data_as(_I), _dp(X), inner.ctypes.data_as(_I), _dp(delta),
                         C.byref(st))
    if rc != 0:
        raise ValueError("oracle solve rejected its arguments")
    t = st.outer_iters
    return dict(perm=perm, X=X, inner=inner[:t].copy(), delta=delta[:t].copy(),
                outer_iters=t, inner_total=st.inner_total, inner_max=st.inner_max,
                converged=bool(st.converged), transposed=bool(st.transposed),
                final_delta=st.final_delta, objective=st.objective, error=st.error)
