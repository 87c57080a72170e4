"""Python side of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It loads ``ft_oracle.c`` compiled with gcc
(``build()``), and shares nothing with the CUDA library.

All arrays are numpy: factor matrices float64 row-major (I_n x J_n), core
matrices float64 (J_n x R), coordinates int32 per mode, values float64.
Every function cites the passage of the paper it follows in ``ft_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ft_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Plain IEEE FP64: no fused multiply-add contraction, no fast-math, so the
# oracle gives the same numbers on x86-64 and aarch64.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math"]


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle with gcc (skipped when the library is newer than
    the source)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    with _lock:
        if path is not None:
            return _declare(ctypes.CDLL(path))
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


class use_library:
    """Context manager: route every call of this module to another build of
    the oracle (the tests use it to run the pins against planted mistakes)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        load()
        with _lock:
            self.saved = _lib
            _lib = _declare(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_DBL = ctypes.c_double


def _declare(lib):
    sig = {
        "orc_predict": [_INT, _P, _INT, _P, _P, _I64, _P, _P, _INT],
        "orc_nonzero_terms": [_INT, _P, _INT, _P, _P, _P, _I64, _P, _P, _P, _P],
        "orc_factor_grads": [_INT, _P, _INT, _P, _P, _P, _I64, _DBL, _DBL, _P],
        "orc_factor_epoch": [_INT, _P, _P, _INT, _P, _P, _I64, _P, _P, _I64, _DBL, _DBL, _P],
        "orc_factor_epoch_hogwild": [_INT, _P, _INT, _P, _P, _I64, _P, _P, _DBL, _DBL, _INT],
        "orc_core_grad": [_INT, _P, _INT, _P, _P, _I64, _P, _P, _P, _INT],
        "orc_core_epoch": [_INT, _P, _INT, _P, _P, _I64, _P, _P, _DBL, _DBL, _INT],
        "orc_core_epoch_sgd": [_INT, _P, _INT, _P, _P, _I64, _P, _P, _I64, _DBL, _DBL, _INT],
        "orc_errors": [_INT, _P, _INT, _P, _P, _I64, _P, _P, _P, _INT],
        "orc_objective": [_INT, _P, _P, _INT, _P, _P, _I64, _P, _P, _DBL, _DBL, _P, _INT],
        "orc_row_stats": [_INT, _P, _P, _INT, _P, _P, _I64, _P, _P, _DBL, _DBL, _DBL, _P, _P, _P],
        "orc_mlp_nparams": [],
        "orc_mlp_forward": [_P, _I64, _P, _P],
        "orc_mlp_grad": [_P, _I64, _P, _P, _P, _P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return lib


# ---------------------------------------------------------------- marshalling
class _Model:
    """Keeps contiguous float64 copies alive and builds pointer arrays."""

    def __init__(self, A, B):
        self.A = [np.ascontiguousarray(a, dtype=np.float64) for a in A]
        self.B = [np.ascontiguousarray(b, dtype=np.float64) for b in B]
        N = len(self.A)
        if len(self.B) != N:
            raise ValueError("A and B must have one matrix per mode")
        self.N = N
        self.R = int(self.B[0].shape[1])
        self.J = np.array([a.shape[1] for a in self.A], dtype=np.int32)
        self.I = np.array([a.shape[0] for a in self.A], dtype=np.int64)
        for b, Jn in zip(self.B, self.J):
            if b.shape != (Jn, self.R):
                raise ValueError("B^(n) must be J_n x R")
        self.pA = (ctypes.c_void_p * N)(*[a.ctypes.data for a in self.A])
        self.pB = (ctypes.c_void_p * N)(*[b.ctypes.data for b in self.B])


def _coords(idx, N):
    cols = [np.ascontiguousarray(np.asarray(idx[n]), dtype=np.int32) for n in range(N)]
    nnz = int(cols[0].shape[0]) if N else 0
    for c in cols:
        if c.shape[0] != nnz:
            raise ValueError("every mode needs the same number of coordinates")
    ptrs = (ctypes.c_void_p * N)(*[c.ctypes.data for c in cols])
    return cols, ptrs, nnz


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed with status {rc}")


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def predict(A, B, idx, nthreads: int = 1) -> np.ndarray:
    """xhat for every coordinate (Eq. "fasttucker")."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    out = np.empty(nnz, dtype=np.float64)
    _check(load().orc_predict(m.N, _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(out), nthreads),
           "orc_predict")
    return out


def nonzero_terms(A, B, idx, m_index: int):
    """(c [N,R], d [N,R], p list of J_n-vectors, xhat) of one nonzero."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    c = np.empty(m.N * m.R)
    d = np.empty(m.N * m.R)
    p = np.empty(int(m.J.sum()))
    xh = np.empty(1)
    _check(load().orc_nonzero_terms(m.N, _ptr(m.J), m.R, m.pA, m.pB, pidx, int(m_index),
                                    _ptr(c), _ptr(d), _ptr(p), _ptr(xh)), "orc_nonzero_terms")
    offs = np.concatenate([[0], np.cumsum(m.J)])
    return (c.reshape(m.N, m.R), d.reshape(m.N, m.R),
            [p[offs[n]:offs[n + 1]] for n in range(m.N)], float(xh[0]))


def factor_grads(A, B, idx, m_index: int, x: float, lam: float):
    """Per-mode factor gradients of one nonzero (Eq. "Gradient_low_rank_cp")."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    g = np.empty(int(m.J.sum()))
    _check(load().orc_factor_grads(m.N, _ptr(m.J), m.R, m.pA, m.pB, pidx, int(m_index),
                                   float(x), float(lam), _ptr(g)), "orc_factor_grads")
    offs = np.concatenate([[0], np.cumsum(m.J)])
    return [g[offs[n]:offs[n + 1]] for n in range(m.N)]


def factor_epoch(A, B, idx, x, S: int, gamma: float, lam: float, row_scale=None):
    """One batch-synchronous factor epoch; returns the new factor matrices
    (the inputs are not modified)."""
    m = _Model([np.array(a, dtype=np.float64, copy=True) for a in A], B)
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    keep = None
    prs = None
    if row_scale is not None:
        keep = [None if s is None else np.ascontiguousarray(s, dtype=np.float64) for s in row_scale]
        prs = (ctypes.c_void_p * m.N)(*[0 if s is None else s.ctypes.data for s in keep])
    _check(load().orc_factor_epoch(m.N, _ptr(m.I), _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx,
                                   _ptr(xv), int(S), float(gamma), float(lam), prs),
           "orc_factor_epoch")
    del keep
    return m.A


def factor_epoch_hogwild(A, B, idx, x, gamma: float, lam: float, nthreads: int = 1):
    """The factor epoch as Hogwild on `nthreads` host threads (S = 1 within a
    thread, concurrent row updates may be lost): for timing the CPU baseline,
    never as a parity reference.  Returns the new factor matrices."""
    m = _Model([np.array(a, dtype=np.float64, copy=True) for a in A], B)
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    _check(load().orc_factor_epoch_hogwild(m.N, _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(xv),
                                           float(gamma), float(lam), int(nthreads)),
           "orc_factor_epoch_hogwild")
    return m.A


def core_grad(A, B, idx, x, nthreads: int = 1):
    """sum over nonzeros of (xhat - x) a^(n)T d^(n), per mode (J_n x R)."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    G = [np.empty((int(Jn), m.R)) for Jn in m.J]
    pG = (ctypes.c_void_p * m.N)(*[g.ctypes.data for g in G])
    _check(load().orc_core_grad(m.N, _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(xv), pG,
                                nthreads), "orc_core_grad")
    return G


def core_epoch(A, B, idx, x, gamma: float, lam: float, nthreads: int = 1):
    """One core phase (Algorithm 5); returns the new core matrices."""
    m = _Model(A, [np.array(b, dtype=np.float64, copy=True) for b in B])
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    _check(load().orc_core_epoch(m.N, _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(xv),
                                 float(gamma), float(lam), nthreads), "orc_core_epoch")
    return m.B


def core_epoch_sgd(A, B, idx, x, S: int, gamma: float, lam: float, nthreads: int = 1):
    """Core phase in the per-sample-set reading of Algorithm 3: consecutive
    sets of S nonzeros, one averaged core step per set; returns the new core
    matrices."""
    m = _Model(A, [np.array(b, dtype=np.float64, copy=True) for b in B])
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    _check(load().orc_core_epoch_sgd(m.N, _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(xv), int(S),
                                     float(gamma), float(lam), nthreads), "orc_core_epoch_sgd")
    return m.B


def errors(A, B, idx, x, nthreads: int = 1):
    """(rmse, mae, sum of squared errors) over the given nonzeros."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(3)
    _check(load().orc_errors(m.N, _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(xv), _ptr(out),
                             nthreads), "orc_errors")
    return float(out[0]), float(out[1]), float(out[2])


def objective(A, B, idx, x, lam_a: float, lam_b: float, nthreads: int = 1) -> float:
    """Eq. "low_rank_optimization_all" with the regulariser summed over modes."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(1)
    _check(load().orc_objective(m.N, _ptr(m.I), _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx,
                                _ptr(xv), float(lam_a), float(lam_b), _ptr(out), nthreads),
           "orc_objective")
    return float(out[0])


# ------------------------------------------------------ learned step sizes
def row_stats(A, B, idx, x, lam: float, gamma: float, beta: float = 0.0, ema_in=None, labels=True):
    """(features [rows, 3], labels [rows] or None), rows of all modes
    concatenated; see orc_row_stats in ft_oracle.c for the definitions."""
    m = _Model(A, B)
    cols, pidx, nnz = _coords(idx, m.N)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    rows = int(m.I.sum())
    feat = np.empty((rows, 3))
    lab = np.empty(rows) if labels else None
    ema = None if ema_in is None else np.ascontiguousarray(ema_in, dtype=np.float64)
    _check(load().orc_row_stats(m.N, _ptr(m.I), _ptr(m.J), m.R, m.pA, m.pB, nnz, pidx, _ptr(xv),
                                float(lam), float(gamma), float(beta),
                                None if ema is None else _ptr(ema), _ptr(feat),
                                None if lab is None else _ptr(lab)), "orc_row_stats")
    return feat, lab


def mlp_nparams() -> int:
    return int(load().orc_mlp_nparams())


def mlp_forward(params, X) -> np.ndarray:
    """Multipliers exp(clamp(u, log 1/16, log 16)) of every row of features."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    Xv = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    out = np.empty(Xv.shape[0])
    _check(load().orc_mlp_forward(_ptr(P), Xv.shape[0], _ptr(Xv), _ptr(out)), "orc_mlp_forward")
    return out


def mlp_grad(params, X, y):
    """(gradient of mean 1/2 (u - y)^2 w.r.t. the parameters, loss): u the
    network's linear output (log-multiplier), y log-multiplier labels."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    Xv = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    yv = np.ascontiguousarray(y, dtype=np.float64)
    G = np.empty_like(P)
    loss = np.empty(1)
    _check(load().orc_mlp_grad(_ptr(P), Xv.shape[0], _ptr(Xv), _ptr(yv), _ptr(G), _ptr(loss)), "orc_mlp_grad")
    return G, float(loss[0])
