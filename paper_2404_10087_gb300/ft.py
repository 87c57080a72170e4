"""Thin ctypes binding of the C ABI in ``include/ft.h``.

The functions below carry the C names and only marshal arguments (device
pointers from torch tensors, host arrays of pointers, the current stream);
every step of the epoch runs in the CUDA library.  There is no fallback: if
``_build/libft.so`` is missing or cannot be loaded, ``load()`` raises.

``FastTuckerPlus`` is a small convenience wrapper that owns the workspace
(a torch byte tensor) and keeps the borrowed tensors alive.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

FT_FP32, FT_TF32, FT_BF16 = 0, 1, 2
FT_HOGWILD, FT_DETERMINISTIC = 0, 1
PRECISIONS = {"fp32": FT_FP32, "tf32": FT_TF32, "bf16": FT_BF16}
SCATTERS = {"hogwild": FT_HOGWILD, "deterministic": FT_DETERMINISTIC}
FT_ENGINE_WARP, FT_ENGINE_TCGEN05 = 0, 1
ENGINES = {"warp": FT_ENGINE_WARP, "tcgen05": FT_ENGINE_TCGEN05}
FT_CORE_CALC, FT_CORE_STORE = 0, 1
CORE_SCHEMES = {"calc": FT_CORE_CALC, "store": FT_CORE_STORE}

FT_OK = 0
FT_ERR_NONFINITE = -5
STATUS = {0: "FT_OK", -1: "FT_ERR_ARG", -2: "FT_ERR_INDEX", -3: "FT_ERR_SHAPE", -4: "FT_ERR_CUDA",
          -5: "FT_ERR_NONFINITE", -6: "FT_ERR_TIMEOUT", -7: "FT_ERR_WORKSPACE"}

# Every symbol the header declares (checked by the tests against the library).
EXPORTS = ["ft_config_default", "ft_workspace_size", "ft_init", "ft_epoch_factors",
           "ft_epoch_core", "ft_epoch_core_sgd", "ft_permute", "ft_rebind", "ft_core_grad",
           "ft_core_apply", "ft_predict", "ft_rmse", "ft_check",
           "ft_launch_count", "ft_destroy", "ft_status_str", "ft_core_grad_noalloc",
           "ft_batch_workspace_size", "ft_batch_init", "ft_batch_tune", "ft_batch_epoch",
           "ft_batch_rmse", "ft_batch_num_classes", "ft_batch_class_info", "ft_batch_launch_count",
           "ft_batch_destroy", "ft_row_stats", "ft_stepnet_bytes", "ft_stepnet_init",
           "ft_stepnet_forward", "ft_stepnet_train", "ft_stepnet_get"]


class FtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class ft_tensor_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("I", ctypes.c_void_p), ("J", ctypes.c_void_p), ("R", ctypes.c_int),
                ("nnz", ctypes.c_int64), ("idx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p)]


class ft_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("scatter", ctypes.c_int),
                ("det_batch", ctypes.c_int64), ("blocks_per_sm", ctypes.c_int),
                ("hot_rows", ctypes.c_int), ("hot_window", ctypes.c_int),
                ("hot_min_count", ctypes.c_int), ("engine", ctypes.c_int), ("core_scheme", ctypes.c_int),
                ("l2_persist", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p


def library_path() -> str:
    """The in-tree library, or the file named by FT_LIBRARY (a variant build)."""
    return os.environ.get("FT_LIBRARY") or _build.LIB_PATH


def load(path: str | None = None):
    """Load the CUDA library (no build, no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or library_path()
        if not os.path.exists(p):
            raise ImportError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        _declare(lib)
        if path is None:
            _lib = lib
        return lib


def _declare(lib):
    I64, INT, FLT = ctypes.c_int64, ctypes.c_int, ctypes.c_float
    sigs = {
        "ft_config_default": (None, [_P]),
        "ft_workspace_size": (INT, [INT, _P, _P, INT, I64, _P, _P]),
        "ft_init": (INT, [_P, INT, _P, _P, INT, I64, _P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P]),
        "ft_epoch_factors": (INT, [_P, FLT, FLT, _P, _P]),
        "ft_epoch_core": (INT, [_P, FLT, FLT, _P]),
        "ft_epoch_core_sgd": (INT, [_P, FLT, FLT, I64, _P]),
        "ft_permute": (INT, [_P, _P, _P, _P, _P]),
        "ft_rebind": (INT, [_P, _P, _P, _P]),
        "ft_core_grad": (INT, [_P, _P, _P]),
        "ft_core_apply": (INT, [_P, _P, I64, FLT, FLT, _P]),
        "ft_predict": (INT, [_P, I64, _P, _P, _P]),
        "ft_rmse": (INT, [_P, I64, _P, _P, _P, _P]),
        "ft_check": (INT, [_P, _P]),
        "ft_launch_count": (I64, [_P]),
        "ft_destroy": (None, [_P]),
        "ft_status_str": (ctypes.c_char_p, [INT]),
        "ft_core_grad_noalloc": (INT, [INT, _P, _P, INT, I64, _P, _P, _P, _P, INT, _P, _P]),
        "ft_batch_workspace_size": (INT, [INT, _P, _P, _P]),
        "ft_batch_init": (INT, [_P, INT, _P, _P, _P, ctypes.c_size_t, _P]),
        "ft_batch_tune": (INT, [_P, _P]),
        "ft_batch_epoch": (INT, [_P, FLT, FLT, FLT, FLT, _P]),
        "ft_batch_rmse": (INT, [_P, INT, I64, _P, _P, _P, _P]),
        "ft_batch_num_classes": (INT, [_P]),
        "ft_batch_class_info": (INT, [_P, INT, _P]),
        "ft_batch_launch_count": (I64, [_P]),
        "ft_batch_destroy": (None, [_P]),
        "ft_row_stats": (INT, [_P, FLT, FLT, FLT, _P, _P, _P, _P]),
        "ft_stepnet_bytes": (ctypes.c_size_t, []),
        "ft_stepnet_init": (INT, [_P, ctypes.c_uint64, _P]),
        "ft_stepnet_forward": (INT, [_P, I64, _P, _P, _P]),
        "ft_stepnet_train": (INT, [_P, I64, _P, _P, FLT, INT, _P, _P]),
        "ft_stepnet_get": (INT, [_P, INT, _P, _P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _check(status: int, where: str):
    if status != FT_OK:
        raise FtError(status, where)


def _ptrs(tensors, ctype=ctypes.c_void_p):
    return (ctype * len(tensors))(*[0 if t is None else t.data_ptr() for t in tensors])


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def make_config(precision="fp32", scatter="hogwild", det_batch=4096, blocks_per_sm=0,
                hot_rows=None, hot_window=None, hot_min_count=None, engine="warp",
                core_scheme="calc", l2_persist=False) -> ft_config:
    c = ft_config()
    load().ft_config_default(ctypes.byref(c))
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.scatter = SCATTERS[scatter] if isinstance(scatter, str) else int(scatter)
    c.det_batch = int(det_batch)
    c.blocks_per_sm = int(blocks_per_sm)
    if hot_rows is not None:
        c.hot_rows = int(hot_rows)
    if hot_window is not None:
        c.hot_window = int(hot_window)
    if hot_min_count is not None:
        c.hot_min_count = int(hot_min_count)
    c.engine = ENGINES[engine] if isinstance(engine, str) else int(engine)
    c.core_scheme = CORE_SCHEMES[core_scheme] if isinstance(core_scheme, str) else int(core_scheme)
    c.l2_persist = int(l2_persist)
    return c


# ------------------------------------------------------ C-named functions
def ft_workspace_size(I, J, R, nnz, cfg: ft_config) -> int:
    N = len(I)
    Ia = (ctypes.c_int64 * N)(*[int(v) for v in I])
    Ja = (ctypes.c_int * N)(*[int(v) for v in J])
    out = ctypes.c_size_t(0)
    _check(load().ft_workspace_size(N, Ia, Ja, int(R), int(nnz), ctypes.byref(cfg), ctypes.byref(out)),
           "ft_workspace_size")
    return int(out.value)


def ft_init(I, J, R, idx, vals, A, B, workspace, cfg: ft_config, stream=None):
    """idx, A, B: lists of device tensors (int32 / float32); returns the
    context handle (an int)."""
    N = len(I)
    Ia = (ctypes.c_int64 * N)(*[int(v) for v in I])
    Ja = (ctypes.c_int * N)(*[int(v) for v in J])
    nnz = int(vals.numel())
    ctx = ctypes.c_void_p(0)
    _check(load().ft_init(ctypes.byref(ctx), N, Ia, Ja, int(R), nnz, _ptrs(idx), vals.data_ptr(),
                          _ptrs(A), _ptrs(B), workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                          ctypes.byref(cfg), _stream(stream)), "ft_init")
    return ctx.value


def ft_epoch_factors(ctx, lr_a, lambda_a, row_step_scale=None, stream=None):
    scale = None if row_step_scale is None else _ptrs(row_step_scale)
    _check(load().ft_epoch_factors(ctx, float(lr_a), float(lambda_a), scale, _stream(stream)),
           "ft_epoch_factors")


def ft_epoch_core(ctx, lr_b, lambda_b, stream=None):
    _check(load().ft_epoch_core(ctx, float(lr_b), float(lambda_b), _stream(stream)), "ft_epoch_core")


def ft_permute(ctx, perm, idx_out, vals_out, stream=None):
    """perm: int32 device tensor (nnz,); idx_out: list of N int32 device
    tensors (nnz,); vals_out: float32 device tensor (nnz,)."""
    n = int(perm.numel())
    _check(load().ft_permute(ctx, perm.data_ptr() if n else None, _ptrs(idx_out) if n else None,
                             vals_out.data_ptr() if n else None, _stream(stream)), "ft_permute")


def ft_rebind(ctx, idx, vals, stream=None):
    """idx: list of N int32 device tensors (nnz,); vals: float32 (nnz,)."""
    n = int(vals.numel())
    _check(load().ft_rebind(ctx, _ptrs(idx) if n else None, vals.data_ptr() if n else None, _stream(stream)),
           "ft_rebind")


def ft_epoch_core_sgd(ctx, lr_b, lambda_b, set_size, stream=None):
    _check(load().ft_epoch_core_sgd(ctx, float(lr_b), float(lambda_b), int(set_size), _stream(stream)),
           "ft_epoch_core_sgd")


def ft_core_grad(ctx, G_out, stream=None):
    _check(load().ft_core_grad(ctx, G_out.data_ptr(), _stream(stream)), "ft_core_grad")


def ft_core_apply(ctx, G, nnz_total, lr_b, lambda_b, stream=None):
    _check(load().ft_core_apply(ctx, G.data_ptr(), int(nnz_total), float(lr_b), float(lambda_b),
                                _stream(stream)), "ft_core_apply")


def ft_core_grad_noalloc(idx, vals, A, B, G_out, precision="fp32", stream=None):
    """Core gradient without a context or workspace (the library's static
    scratch is used; see include/ft.h).  idx, A, B: lists of device tensors;
    G_out: device float32 tensor of sum_n J_n * R entries."""
    N = len(A)
    I = (ctypes.c_int64 * N)(*[int(a.shape[0]) for a in A])
    J = (ctypes.c_int * N)(*[int(a.shape[1]) for a in A])
    R = int(B[0].shape[1])
    nnz = int(vals.numel())
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(load().ft_core_grad_noalloc(N, I, J, R, nnz, _ptrs(idx) if nnz else None,
                                       vals.data_ptr() if nnz else None, _ptrs(A), _ptrs(B), prec,
                                       G_out.data_ptr(), _stream(stream)), "ft_core_grad_noalloc")


def ft_predict(ctx, idx, out, stream=None):
    n = int(out.numel())
    _check(load().ft_predict(ctx, n, _ptrs(idx) if n else None, out.data_ptr() if n else None,
                             _stream(stream)), "ft_predict")


def ft_rmse(ctx, idx, vals, stream=None):
    """Returns (rmse, mae, sum of squared errors); synchronises the stream."""
    n = int(vals.numel())
    out = (ctypes.c_double * 3)()
    _check(load().ft_rmse(ctx, n, _ptrs(idx) if n else None, vals.data_ptr() if n else None, out,
                          _stream(stream)), "ft_rmse")
    return float(out[0]), float(out[1]), float(out[2])


def ft_check(ctx, stream=None):
    _check(load().ft_check(ctx, _stream(stream)), "ft_check")


def ft_launch_count(ctx) -> int:
    return int(load().ft_launch_count(ctx))


def ft_destroy(ctx):
    if ctx:
        load().ft_destroy(ctx)


def ft_status_str(status: int) -> str:
    return load().ft_status_str(int(status)).decode()


# ----------------------------------------------------------- convenience
class FastTuckerPlus:
    """One sparse tensor's training context.

    idx: list of N int32 device tensors (nnz,), vals: float32 (nnz,),
    A: list of N float32 (I_n, J_n), B: list of N float32 (J_n, R), all on
    the same CUDA device and contiguous.  A and B are updated in place.
    """

    def __init__(self, idx, vals, A, B, precision="fp32", scatter="hogwild", det_batch=4096,
                 blocks_per_sm=0, stream=None, hot_rows=None, hot_window=None, hot_min_count=None,
                 engine="warp", core_scheme="calc", l2_persist=False):
        N = len(A)
        if not (len(idx) == len(B) == N):
            raise ValueError("idx, A and B need one entry per mode")
        for t in list(idx) + [vals] + list(A) + list(B):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("every tensor must be a contiguous CUDA tensor")
        self.idx = [t for t in idx]
        self.vals = vals
        self.A = list(A)
        self.B = list(B)
        self.I = [int(a.shape[0]) for a in A]
        self.J = [int(a.shape[1]) for a in A]
        self.R = int(B[0].shape[1])
        self.nnz = int(vals.numel())
        self.cfg = make_config(precision, scatter, det_batch, blocks_per_sm, hot_rows, hot_window,
                               hot_min_count, engine, core_scheme, l2_persist)
        ws = ft_workspace_size(self.I, self.J, self.R, self.nnz, self.cfg)
        self.workspace = torch.empty(max(ws, 256), dtype=torch.uint8, device=vals.device)
        self.ctx = ft_init(self.I, self.J, self.R, self.idx, vals, self.A, self.B, self.workspace,
                           self.cfg, stream)

    def epoch_factors(self, lr, lam, row_step_scale=None, stream=None):
        ft_epoch_factors(self.ctx, lr, lam, row_step_scale, stream)

    def epoch_core(self, lr, lam, stream=None):
        ft_epoch_core(self.ctx, lr, lam, stream)

    def epoch_core_sgd(self, lr, lam, set_size, stream=None):
        ft_epoch_core_sgd(self.ctx, lr, lam, set_size, stream)

    def rebind(self, idx, vals, stream=None):
        """Train on another copy of the nonzeros from now on (same nnz)."""
        if len(idx) != len(self.idx) or int(vals.numel()) != self.nnz:
            raise ValueError("rebind needs N coordinate arrays and nnz values")
        for t in list(idx) + [vals]:
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("every tensor must be a contiguous CUDA tensor")
        ft_rebind(self.ctx, idx, vals, stream)
        self.idx, self.vals = list(idx), vals

    def permute(self, perm, stream=None):
        """Reorder the training nonzeros by perm (int32 device tensor).  The
        reordered copies live in two buffers this object owns and alternates
        between, so the caller's arrays are never overwritten."""
        if not hasattr(self, "_spare"):
            self._spare = [([torch.empty_like(t) for t in self.idx], torch.empty_like(self.vals))
                           for _ in range(2)]
            self._next = 0
        idx_out, vals_out = self._spare[self._next]
        ft_permute(self.ctx, perm, idx_out, vals_out, stream)
        self.idx, self.vals = idx_out, vals_out
        self._next ^= 1

    def core_grad(self, stream=None):
        G = torch.empty(sum(j * self.R for j in self.J), dtype=torch.float32, device=self.vals.device)
        ft_core_grad(self.ctx, G, stream)
        out, off = [], 0
        for j in self.J:
            out.append(G[off:off + j * self.R].view(j, self.R))
            off += j * self.R
        return out

    def core_apply(self, G, nnz_total, lr, lam, stream=None):
        """B <- B - lr (G / nnz_total + lam B), G flat in the layout of
        ft_core_grad (or a list of J_n x R tensors, concatenated here)."""
        if isinstance(G, (list, tuple)):
            G = torch.cat([g.reshape(-1) for g in G])
        if not G.is_cuda or G.dtype != torch.float32 or not G.is_contiguous() \
                or G.numel() != sum(j * self.R for j in self.J):
            raise ValueError("G must be a contiguous float32 CUDA tensor of sum_n J_n R entries")
        ft_core_apply(self.ctx, G, nnz_total, lr, lam, stream)

    def predict(self, idx, stream=None):
        out = torch.empty(int(idx[0].numel()), dtype=torch.float32, device=self.vals.device)
        ft_predict(self.ctx, idx, out, stream)
        return out

    def rmse(self, idx, vals, stream=None):
        return ft_rmse(self.ctx, idx, vals, stream)

    def check(self, stream=None):
        ft_check(self.ctx, stream)

    @property
    def launches(self) -> int:
        return ft_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ft_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- batches
class _Descs:
    """ft_tensor_desc array plus the host arrays it points to."""

    def __init__(self, tensors):
        self.keep = []
        self.arr = (ft_tensor_desc * len(tensors))()
        for d, (idx, vals, A, B) in zip(self.arr, tensors):
            N = len(A)
            I = (ctypes.c_int64 * N)(*[int(a.shape[0]) for a in A])
            J = (ctypes.c_int * N)(*[int(a.shape[1]) for a in A])
            pi, pa, pb = _ptrs(idx), _ptrs(A), _ptrs(B)
            self.keep += [I, J, pi, pa, pb]
            d.N, d.R, d.nnz = N, int(B[0].shape[1]), int(vals.numel())
            d.I, d.J = ctypes.addressof(I), ctypes.addressof(J)
            d.idx, d.A, d.B = ctypes.addressof(pi), ctypes.addressof(pa), ctypes.addressof(pb)
            d.vals = vals.data_ptr() if vals.numel() else 0


def ft_batch_workspace_size(tensors, cfg: ft_config) -> int:
    ds = _Descs(tensors)
    out = ctypes.c_size_t(0)
    _check(load().ft_batch_workspace_size(len(tensors), ds.arr, ctypes.byref(cfg), ctypes.byref(out)),
           "ft_batch_workspace_size")
    return int(out.value)


def ft_batch_init(tensors, workspace, cfg: ft_config, stream=None):
    ds = _Descs(tensors)
    h = ctypes.c_void_p(0)
    _check(load().ft_batch_init(ctypes.byref(h), len(tensors), ds.arr, ctypes.byref(cfg),
                                workspace.data_ptr(), workspace.numel(), _stream(stream)), "ft_batch_init")
    return h.value


def ft_batch_tune(b, stream=None):
    _check(load().ft_batch_tune(b, _stream(stream)), "ft_batch_tune")


def ft_batch_epoch(b, lr_a, lambda_a, lr_b, lambda_b, stream=None):
    _check(load().ft_batch_epoch(b, float(lr_a), float(lambda_a), float(lr_b), float(lambda_b),
                                 _stream(stream)), "ft_batch_epoch")


def ft_batch_rmse(b, tensor, idx, vals, stream=None):
    n = int(vals.numel())
    out = (ctypes.c_double * 3)()
    _check(load().ft_batch_rmse(b, int(tensor), n, _ptrs(idx) if n else None,
                                vals.data_ptr() if n else None, out, _stream(stream)), "ft_batch_rmse")
    return float(out[0]), float(out[1]), float(out[2])


def ft_batch_num_classes(b) -> int:
    return int(load().ft_batch_num_classes(b))


def ft_batch_class_info(b, cls):
    out = (ctypes.c_int64 * 6)()
    _check(load().ft_batch_class_info(b, int(cls), out), "ft_batch_class_info")
    keys = ("N", "K", "tensors", "unit_tiles", "ctas_per_sm", "units")
    return dict(zip(keys, [int(v) for v in out]))


def ft_batch_launch_count(b) -> int:
    return int(load().ft_batch_launch_count(b))


def ft_batch_destroy(b):
    if b:
        load().ft_batch_destroy(b)


class FastTuckerBatch:
    """Independent tensors trained together.  tensors: list of
    (idx list, vals, A list, B list) device tensors, as for FastTuckerPlus."""

    def __init__(self, tensors, precision="fp32", stream=None, tune=False):
        self.tensors = [(list(i), v, list(a), list(b)) for i, v, a, b in tensors]
        self.cfg = make_config(precision, "hogwild")
        ws = ft_batch_workspace_size(self.tensors, self.cfg)
        dev = self.tensors[0][1].device
        self.workspace = torch.empty(max(ws, 256), dtype=torch.uint8, device=dev)
        self.handle = ft_batch_init(self.tensors, self.workspace, self.cfg, stream)
        if tune:
            self.tune(stream)

    def tune(self, stream=None):
        ft_batch_tune(self.handle, stream)

    def epoch(self, lr_a, lam_a, lr_b=None, lam_b=None, stream=None):
        ft_batch_epoch(self.handle, lr_a, lam_a, lr_a if lr_b is None else lr_b,
                       lam_a if lam_b is None else lam_b, stream)

    def rmse(self, tensor, idx, vals, stream=None):
        return ft_batch_rmse(self.handle, tensor, idx, vals, stream)

    def classes(self):
        return [ft_batch_class_info(self.handle, c) for c in range(ft_batch_num_classes(self.handle))]

    @property
    def launches(self) -> int:
        return ft_batch_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            ft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- learned step sizes
STEPNET_PARAMS = 4481


def ft_row_stats(ctx, lambda_a, lr_a, ema_beta, ema, features, labels=None, stream=None):
    _check(load().ft_row_stats(ctx, float(lambda_a), float(lr_a), float(ema_beta),
                               None if ema is None else ema.data_ptr(), features.data_ptr(),
                               None if labels is None else labels.data_ptr(), _stream(stream)),
           "ft_row_stats")


def ft_stepnet_bytes() -> int:
    return int(load().ft_stepnet_bytes())


def ft_stepnet_init(net, seed=0, stream=None):
    _check(load().ft_stepnet_init(net.data_ptr(), int(seed), _stream(stream)), "ft_stepnet_init")


def ft_stepnet_forward(net, features, scale, stream=None):
    rows = int(scale.numel())
    _check(load().ft_stepnet_forward(net.data_ptr(), rows, features.data_ptr() if rows else None,
                                     scale.data_ptr() if rows else None, _stream(stream)), "ft_stepnet_forward")


def ft_stepnet_train(net, features, labels, lr, steps, stream=None):
    loss = ctypes.c_double(0.0)
    _check(load().ft_stepnet_train(net.data_ptr(), int(labels.numel()), features.data_ptr(), labels.data_ptr(),
                                   float(lr), int(steps), ctypes.byref(loss), _stream(stream)),
           "ft_stepnet_train")
    return float(loss.value)


def ft_stepnet_get(net, which, stream=None):
    import numpy as np
    out = np.empty(STEPNET_PARAMS, dtype=np.float32)
    _check(load().ft_stepnet_get(net.data_ptr(), int(which), out.ctypes.data, _stream(stream)), "ft_stepnet_get")
    return out


def new_stepnet(device, seed=0):
    """A device buffer holding an initialised step-size network."""
    net = torch.empty(ft_stepnet_bytes(), dtype=torch.uint8, device=device)
    ft_stepnet_init(net, seed)
    return net
