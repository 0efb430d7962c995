"""Thin ctypes binding of libfastpfp.so (include/fastpfp.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (float32, contiguous),
passed by ``data_ptr()`` together with the current CUDA stream.  There is no
CPU fallback: if the library cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfastpfp.so")

FASTPFP_OK = 0
FASTPFP_ERR_ARG = -1
FASTPFP_ERR_SIZE = -2
FASTPFP_ERR_CUDA = -3
FASTPFP_ERR_TIMEOUT = -4
FASTPFP_ERR_NONFINITE = -5
FASTPFP_ERR_UNSUPPORTED = -6
FP32, BF16, FP8, FP32_SIMT = 0, 1, 2, 3
ALG_FASTPFP, ALG_PG, ALG_FASTGA = 0, 1, 2

# Every symbol include/fastpfp.h declares.
EXPORTS = ("fastpfp_default_params", "fastpfp_create", "fastpfp_destroy", "fastpfp_match",
           "fastpfp_match_host", "fastpfp_match_batched", "fastpfp_match_batched_host",
           "fastpfp_last_trace",
           "fastpfp_gradient", "fastpfp_affinity", "fastpfp_project", "fastpfp_discretize",
           "fastpfp_project_noalloc", "fastpfp_warmstart", "fastpfp_warmstart_train_step",
           "fastpfp_bandwidth_probe", "fastpfp_gemm_probe", "fastpfp_autotune", "fastpfp_get_tiles", "fastpfp_set_tiles",
           "fastpfp_error_string")
TUNE_SIZES, TUNE_COUNTS = 8, 4
MLP_NPARAMS = 32 * 128 + 128 + 128 * 64 + 64


class fastpfp_params(C.Structure):
    _fields_ = [("lambda_", C.c_float), ("alpha", C.c_float), ("tol_outer", C.c_double),
                ("tol_inner", C.c_double), ("max_outer", C.c_int), ("max_inner", C.c_int),
                ("precision", C.c_int), ("refine_iters", C.c_int), ("switch_tol", C.c_double),
                ("normalize_max", C.c_int), ("slack_policy", C.c_int), ("timeout_ms", C.c_int),
                ("profile", C.c_int), ("loop_mode", C.c_int), ("debug_flags", C.c_int),
                ("algorithm", C.c_int), ("beta", C.c_float)]


class fastpfp_stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters_total", C.c_int),
                ("inner_iters_max", C.c_int), ("converged", C.c_int), ("lowp_iters", C.c_int),
                ("transposed", C.c_int), ("status", C.c_int), ("launches", C.c_int),
                ("wave_pairs", C.c_int),
                ("final_delta", C.c_double), ("objective", C.c_double), ("ms_gemm", C.c_float),
                ("ms_proj", C.c_float), ("ms_disc", C.c_float), ("host_syncs", C.c_int)]


class fastpfp_pair(C.Structure):
    _fields_ = [("A", C.c_void_p), ("A2", C.c_void_p), ("B", C.c_void_p), ("B2", C.c_void_p),
                ("n_a", C.c_int), ("n_b", C.c_int), ("k", C.c_int), ("X0", C.c_void_p),
                ("perm_out", C.c_void_p), ("X_out", C.c_void_p)]


class FastPFPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


_lib = None


def lib():
    """Loads libfastpfp.so; raises if it is missing (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libfastpfp.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    l = C.CDLL(LIB_PATH)
    P, V, I = C.c_void_p, C.c_void_p, C.c_int
    l.fastpfp_default_params.argtypes = [C.POINTER(fastpfp_params)]
    l.fastpfp_default_params.restype = None
    l.fastpfp_create.argtypes = [C.POINTER(C.c_void_p), I, I, I]
    l.fastpfp_destroy.argtypes = [P]
    l.fastpfp_destroy.restype = None
    sig = [P, V, P, I, P, I, P, P, I, C.POINTER(fastpfp_params), P, P, P, C.POINTER(fastpfp_stats)]
    l.fastpfp_match.argtypes = sig
    l.fastpfp_match_host.argtypes = sig
    l.fastpfp_match_batched_host.argtypes = [P, V, I, C.POINTER(fastpfp_pair),
                                             C.POINTER(fastpfp_params), C.POINTER(fastpfp_stats)]
    l.fastpfp_match_batched.argtypes = [P, V, I, C.POINTER(fastpfp_pair), C.POINTER(fastpfp_params),
                                        C.POINTER(fastpfp_stats)]
    l.fastpfp_last_trace.argtypes = [P, I, P, P, I]
    l.fastpfp_gradient.argtypes = [P, V, P, P, P, P, C.c_float, I, I, P, I, I]
    l.fastpfp_affinity.argtypes = [P, V, P, P, I, I, I, P]
    l.fastpfp_project.argtypes = [P, V, P, I, C.c_double, I, C.POINTER(C.c_int),
                                  C.POINTER(C.c_double)]
    l.fastpfp_discretize.argtypes = [P, V, P, I, I, P]
    l.fastpfp_project_noalloc.argtypes = [V, P, I, C.c_double, I, C.POINTER(C.c_int),
                                          C.POINTER(C.c_double)]
    l.fastpfp_warmstart.argtypes = [P, V, P, I, P, I, P, P, I, P, I, P]
    l.fastpfp_warmstart_train_step.argtypes = [P, V, P, I, P, I, P, P, I, P, P, P, P, I, C.c_float,
                                               C.POINTER(C.c_double), P]
    l.fastpfp_bandwidth_probe.argtypes = [I, I, I, C.POINTER(C.c_double)]
    l.fastpfp_gemm_probe.argtypes = [I, I, I, I, C.POINTER(C.c_double)]
    l.fastpfp_autotune.argtypes = [P, V, I, P]
    l.fastpfp_get_tiles.argtypes = [P, I, I, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    l.fastpfp_set_tiles.argtypes = [P, I, I, I, I]
    l.fastpfp_error_string.argtypes = [I]
    l.fastpfp_error_string.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("fastpfp_default_params", "fastpfp_destroy", "fastpfp_error_string"):
            getattr(l, name).restype = C.c_int
    _lib = l
    return l


def bandwidth_probe(level: int, sweeps: int = 200, device: int = 0) -> float:
    """GB/s of shared memory (0), L2 (1), HBM (2) or tensor memory (3) under
    the projection rounds' read + write pattern (fastpfp_bandwidth_probe)."""
    out = C.c_double(0.0)
    _check(lib().fastpfp_bandwidth_probe(int(device), int(level), int(sweeps), C.byref(out)),
           "fastpfp_bandwidth_probe")
    return float(out.value)


def gemm_probe(precision: int, n: int = 4096, reps: int = 10, device: int = 0) -> float:
    """TFLOP/s of one n^3 product on the solver's FP32 (split TF32 on the
    tensor cores), BF16, FP8 or FP32_SIMT kernel (fastpfp_gemm_probe)."""
    out = C.c_double(0.0)
    _check(lib().fastpfp_gemm_probe(int(device), int(precision), int(n), int(reps), C.byref(out)),
           "fastpfp_gemm_probe")
    return float(out.value)


def init_mlp_params(seed: int = 0):
    """Initial weights of the warm-start MLP (32 -> 128 -> 64) as one flat
    float32 array in the library's packing [W1 (32x128), b1, W2 (128x64),
    b2]: Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((32, 128), (128, 64)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def error_string(code: int) -> str:
    return lib().fastpfp_error_string(int(code)).decode()


def default_params(**kw) -> fastpfp_params:
    p = fastpfp_params()
    lib().fastpfp_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k in ("lam", "lambda") else k, v)
    return p


def _check(rc: int, where: str) -> None:
    if rc != FASTPFP_OK:
        raise FastPFPError(rc, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_f32(t, shape, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape {shape}")
    return t


@dataclass
class MatchResult:
    perm: object            # int32 tensor/array of n_a entries (-1 = unmatched)
    X: object | None        # n_a x n_b soft assignment, if requested
    stats: fastpfp_stats


class Solver:
    """One fastpfp handle (device scratch sized for graphs of up to max_n)."""

    def __init__(self, max_n: int, max_batch: int = 1, device: int = 0):
        self._h = C.c_void_p()
        _check(lib().fastpfp_create(C.byref(self._h), int(device), int(max_n), int(max_batch)),
               "fastpfp_create")
        self.max_n, self.max_batch, self.device = max_n, max_batch, device

    def close(self):
        if self._h:
            lib().fastpfp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------- whole solve
    def match(self, A, A2, B=None, B2=None, params=None, X0=None, want_X=False, stream=None):
        """fastpfp_match on torch CUDA tensors; returns MatchResult."""
        import torch
        n_a, n_b = A.shape[0], A2.shape[0]
        k = 0 if B is None else B.shape[1]
        _dev_f32(A, (n_a, n_a), "A")
        _dev_f32(A2, (n_b, n_b), "A2")
        if k:
            _dev_f32(B, (n_a, k), "B")
            _dev_f32(B2, (n_b, k), "B2")
        _dev_f32(X0, (n_a, n_b), "X0")
        p = params if params is not None else default_params()
        perm = torch.empty(n_a, dtype=torch.int32, device=A.device)
        X = torch.empty((n_a, n_b), dtype=torch.float32, device=A.device) if want_X else None
        st = fastpfp_stats()
        rc = lib().fastpfp_match(self._h, _stream(stream), _ptr(A), n_a, _ptr(A2), n_b,
                                 _ptr(B) if k else None, _ptr(B2) if k else None, k, C.byref(p),
                                 _ptr(X0), _ptr(perm), _ptr(X), C.byref(st))
        _check(rc, "fastpfp_match")
        return MatchResult(perm, X, st)

    def match_host(self, A, A2, B=None, B2=None, params=None, X0=None, want_X=False, stream=None):
        """fastpfp_match_host on host float32 arrays: numpy arrays, or torch CPU
        tensors (pinned tensors are passed without a copy)."""
        def host(a):
            if a is None or (hasattr(a, "data_ptr") and not a.is_cuda and a.is_contiguous()
                             and str(a.dtype) == "torch.float32"):
                return a
            return np.ascontiguousarray(a, dtype=np.float32)
        A, A2, B, B2, X0 = host(A), host(A2), host(B), host(B2), host(X0)
        n_a, n_b = A.shape[0], A2.shape[0]
        k = 0 if B is None else B.shape[1]
        p = params if params is not None else default_params()
        perm = np.empty(n_a, dtype=np.int32)
        X = np.empty((n_a, n_b), dtype=np.float32) if want_X else None
        st = fastpfp_stats()

        def hp(a):
            if a is None:
                return None
            return C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        rc = lib().fastpfp_match_host(self._h, _stream(stream), hp(A), n_a, hp(A2), n_b,
                                      hp(B) if k else None, hp(B2) if k else None, k, C.byref(p),
                                      hp(X0), hp(perm), hp(X), C.byref(st))
        _check(rc, "fastpfp_match_host")
        return MatchResult(perm, X, st)

    def match_batched(self, pairs, params=None, want_X=False, stream=None):
        """pairs: list of (A, A2, B, B2) or (A, A2, B, B2, X0) CUDA tensors
        (B/B2 may be None; X0, an n_a x n_b start, may be None)."""
        import torch
        p = params if params is not None else default_params()
        n = len(pairs)
        arr = (fastpfp_pair * max(1, n))()
        outs = []
        keep = []
        for b, pr in enumerate(pairs):
            A, A2, B, B2 = pr[:4]
            X0 = pr[4] if len(pr) > 4 else None
            n_a, n_b = A.shape[0], A2.shape[0]
            k = 0 if B is None else B.shape[1]
            perm = torch.empty(n_a, dtype=torch.int32, device=A.device)
            X = torch.empty((n_a, n_b), dtype=torch.float32, device=A.device) if want_X else None
            arr[b] = fastpfp_pair(A.data_ptr(), A2.data_ptr(), B.data_ptr() if k else None,
                                  B2.data_ptr() if k else None, n_a, n_b, k,
                                  X0.data_ptr() if X0 is not None else None, perm.data_ptr(),
                                  X.data_ptr() if X is not None else None)
            outs.append((perm, X))
            keep.append(pr)
        sts = (fastpfp_stats * max(1, n))()
        rc = lib().fastpfp_match_batched(self._h, _stream(stream), n, arr, C.byref(p), sts)
        _check(rc, "fastpfp_match_batched")
        return [MatchResult(perm, X, sts[b]) for b, (perm, X) in enumerate(outs)]

    def match_batched_host(self, pairs, params=None, want_X=False, stream=None):
        """fastpfp_match_batched_host: pairs of host float32 arrays (numpy, or
        pinned torch CPU tensors passed without a copy); returns host results."""
        p = params if params is not None else default_params()
        n = len(pairs)
        arr = (fastpfp_pair * max(1, n))()
        keep, outs = [], []

        def host(a):
            if a is None or (hasattr(a, "data_ptr") and not a.is_cuda and a.is_contiguous()
                             and str(a.dtype) == "torch.float32"):
                return a
            return np.ascontiguousarray(a, dtype=np.float32)

        def addr(a):
            if a is None:
                return None
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        for b, (A, A2, B, B2) in enumerate(pairs):
            A, A2, B, B2 = host(A), host(A2), host(B), host(B2)
            n_a, n_b = A.shape[0], A2.shape[0]
            k = 0 if B is None else B.shape[1]
            perm = np.empty(n_a, dtype=np.int32)
            X = np.empty((n_a, n_b), dtype=np.float32) if want_X else None
            arr[b] = fastpfp_pair(addr(A), addr(A2), addr(B) if k else None, addr(B2) if k else None,
                                  n_a, n_b, k, None, perm.ctypes.data,
                                  X.ctypes.data if X is not None else None)
            keep.append((A, A2, B, B2))
            outs.append((perm, X))
        sts = (fastpfp_stats * max(1, n))()
        rc = lib().fastpfp_match_batched_host(self._h, _stream(stream), n, arr, C.byref(p), sts)
        _check(rc, "fastpfp_match_batched_host")
        return [MatchResult(perm, X, sts[b]) for b, (perm, X) in enumerate(outs)]

    def last_trace(self, pair: int = 0, cap: int = 4096):
        """(inner counts, max|dX|) per outer iteration of pair `pair` of the
        last call (0 after match; any pair's index after a batch)."""
        inner = np.zeros(cap, dtype=np.int32)
        delta = np.zeros(cap, dtype=np.float64)
        n = lib().fastpfp_last_trace(self._h, int(pair), C.c_void_p(inner.ctypes.data),
                                     C.c_void_p(delta.ctypes.data), cap)
        if n < 0:
            raise FastPFPError(n, "fastpfp_last_trace")
        n = min(n, cap)
        return inner[:n].copy(), delta[:n].copy()

    # ------------------------------------------------------- tile shapes
    def autotune(self, reps: int = 3, stream=None):
        """fastpfp_autotune: times both tiles of both gradient products per
        size and count class and keeps the faster.  Returns the best times
        (ms) as a (TUNE_SIZES, TUNE_COUNTS, 4) array: FP32 tile 128, FP32
        tile 64, BF16 tile 256, BF16 tile 128 (0 = class not measured)."""
        t = np.zeros((TUNE_SIZES, TUNE_COUNTS, 4), dtype=np.float64)
        _check(lib().fastpfp_autotune(self._h, _stream(stream), int(reps), C.c_void_p(t.ctypes.data)),
               "fastpfp_autotune")
        return t

    def get_tiles(self, n: int, count: int = 1):
        """(FP32 tile rows, BF16 tile columns) used for a group of `count`
        pairs whose largest canonical size is n."""
        a, b = C.c_int(0), C.c_int(0)
        _check(lib().fastpfp_get_tiles(self._h, int(n), int(count), C.byref(a), C.byref(b)),
               "fastpfp_get_tiles")
        return a.value, b.value

    def set_tiles(self, f32_tile_m: int, tc_tile_n: int, n: int = 0, count: int = 0):
        """Sets the tiles of the classes of n and count (0 = every class)."""
        _check(lib().fastpfp_set_tiles(self._h, int(n), int(count), int(f32_tile_m), int(tc_tile_n)),
               "fastpfp_set_tiles")

    # ------------------------------------------------------- single steps
    def gradient(self, A, X, A2, K=None, lam=0.0, precision=FP32, stream=None):
        import torch
        N, m = X.shape
        Y = torch.zeros((N, m), dtype=torch.float32, device=X.device)
        _check(lib().fastpfp_gradient(self._h, _stream(stream), _ptr(A), _ptr(X), _ptr(A2),
                                      _ptr(K), float(lam), N, m, _ptr(Y), m, int(precision)),
               "fastpfp_gradient")
        return Y

    def affinity(self, B, B2, stream=None):
        import torch
        N, k = B.shape
        m = B2.shape[0]
        K = torch.empty((N, m), dtype=torch.float32, device=B.device)
        _check(lib().fastpfp_affinity(self._h, _stream(stream), _ptr(B), _ptr(B2), N, m, k,
                                      _ptr(K)), "fastpfp_affinity")
        return K

    def project(self, Y, tol=1e-6, max_iter=1000, stream=None):
        """In-place P_D on the N x N tensor Y; returns (iterations, last delta)."""
        it = C.c_int(0)
        d = C.c_double(0.0)
        _check(lib().fastpfp_project(self._h, _stream(stream), _ptr(Y), Y.shape[0], float(tol),
                                     int(max_iter), C.byref(it), C.byref(d)), "fastpfp_project")
        return it.value, d.value

    # ---------------------------------------------------- learned start
    def warmstart(self, A, A2, B, B2, params, iters=20, stream=None):
        """fastpfp_warmstart: the learned X0 (n_a x n_b CUDA tensor)."""
        import torch
        n_a, n_b = A.shape[0], A2.shape[0]
        k = 0 if B is None else B.shape[1]
        X0 = torch.empty((n_a, n_b), dtype=torch.float32, device=A.device)
        _check(lib().fastpfp_warmstart(self._h, _stream(stream), _ptr(A), n_a, _ptr(A2), n_b,
                                       _ptr(B) if k else None, _ptr(B2) if k else None, k,
                                       _ptr(params), int(iters), _ptr(X0)), "fastpfp_warmstart")
        return X0

    def train_step(self, A, A2, B, B2, perm, params, adam_m=None, adam_v=None, step=0, lr=0.0,
                   want_grad=False, stream=None):
        """fastpfp_warmstart_train_step; returns (loss, grad or None)."""
        import torch
        n_a, n_b = A.shape[0], A2.shape[0]
        k = 0 if B is None else B.shape[1]
        grad = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=A.device) if want_grad else None
        loss = C.c_double(0.0)
        _check(lib().fastpfp_warmstart_train_step(
            self._h, _stream(stream), _ptr(A), n_a, _ptr(A2), n_b, _ptr(B) if k else None,
            _ptr(B2) if k else None, k, _ptr(perm), _ptr(params), _ptr(adam_m), _ptr(adam_v),
            int(step), float(lr), C.byref(loss), _ptr(grad)), "fastpfp_warmstart_train_step")
        return loss.value, grad

    def discretize(self, X, stream=None):
        import torch
        N, m = X.shape
        out = torch.empty(m, dtype=torch.int32, device=X.device)
        _check(lib().fastpfp_discretize(self._h, _stream(stream), _ptr(X), N, m, _ptr(out)),
               "fastpfp_discretize")
        return out


def project_noalloc(Y, tol=1e-6, max_iter=1000, stream=None):
    """fastpfp_project_noalloc: in-place P_D on the N x N CUDA tensor Y
    without a handle and without any device allocation (N a multiple of 4,
    N <= 4096).  Returns (iterations, last delta)."""
    it = C.c_int(0)
    d = C.c_double(0.0)
    _check(lib().fastpfp_project_noalloc(_stream(stream), _ptr(Y), Y.shape[0], float(tol),
                                         int(max_iter), C.byref(it), C.byref(d)),
           "fastpfp_project_noalloc")
    return it.value, d.value
