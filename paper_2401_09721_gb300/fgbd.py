"""Thin ctypes binding of the FGBD C ABI (include/fgbd.h).

Argument marshalling only: every step of the method runs in the CUDA library
``libfgbd.so``.  Tensors are passed as device pointers; the current PyTorch
CUDA stream is used unless one is given.  If the library is missing or fails
to load, every call raises ``RuntimeError``: there is no CPU fallback.

The functions below carry the names of the C entry points.  ``Context`` is a
small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfgbd.so")

FGBD_U8 = 0
FGBD_F32 = 1
PATCH_DIM = 21        # FGBD_PATCH_DIM (window 1)
MAX_WINDOW = 3        # FGBD_MAX_WINDOW
PATCH_DIM_MAX = 57    # FGBD_PATCH_DIM_MAX
Q_CAP = 256
ABI_VERSION = 3

STATUS = {
    0: "FGBD_OK",
    1: "FGBD_EINVAL",
    2: "FGBD_ERANGE",
    3: "FGBD_ENOMEM",
    4: "FGBD_ECUDA",
    5: "FGBD_ETIMEOUT",
    6: "FGBD_ESTATE",
    7: "FGBD_ENOTIMPL",
}


class FgbdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class Params(ctypes.Structure):
    _fields_ = [
        ("bits", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("fslr_factor", ctypes.c_double),
        ("q_max", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 5),
    ]


VARIANT_NO_FSLR = 1          # FGBD_VARIANT_NO_FSLR
VARIANT_UNSORTED_PATCH = 2   # FGBD_VARIANT_UNSORTED_PATCH
VARIANT_SAME_LINE = 4        # FGBD_VARIANT_SAME_LINE
VARIANT_SIGMA_NODE = 8       # FGBD_VARIANT_SIGMA_NODE
VARIANT_SIGMA_PAIR = 16      # FGBD_VARIANT_SIGMA_PAIR
VARIANT_POOLED_PATCH = 32    # FGBD_VARIANT_POOLED_PATCH
VARIANT_GLOBAL_Q = 64        # FGBD_VARIANT_GLOBAL_Q
FLAG_FUSED_SELECT = 1        # FGBD_FLAG_FUSED_SELECT


class BatchShape(ctypes.Structure):
    _fields_ = [
        ("seg_frames", ctypes.c_int32),
        ("scatter_threads", ctypes.c_int32),
        ("filter_threads", ctypes.c_int32),
        ("filter_blocks_per_sm", ctypes.c_int32),
        ("ms", ctypes.c_float),
        ("reserved", ctypes.c_int32 * 3),
    ]

    def as_dict(self) -> dict:
        return dict(seg_frames=self.seg_frames, scatter_threads=self.scatter_threads,
                    filter_threads=self.filter_threads, filter_blocks_per_sm=self.filter_blocks_per_sm, ms=self.ms)


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("n_edges", ctypes.c_int64),
        ("sigma_g", ctypes.c_double),
        ("n_patches", ctypes.c_int64),
        ("patch_dim", ctypes.c_int32),
        ("eigenvalues", ctypes.c_double * PATCH_DIM_MAX),
        ("m", ctypes.c_int32),
        ("q", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("sigma_est", ctypes.c_double),
        ("n_keep", ctypes.c_int64),
        ("n_objective", ctypes.c_int32),
        ("valid", ctypes.c_int32),
        ("objective", ctypes.c_double * (Q_CAP + 1)),
        ("launches", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return dict(
            n=self.n, n_edges=self.n_edges, sigma_g=self.sigma_g, n_patches=self.n_patches,
            patch_dim=self.patch_dim,
            eigenvalues=list(self.eigenvalues[: self.patch_dim]), m=self.m, q=self.q, tau=self.tau,
            sigma_est=self.sigma_est, n_keep=self.n_keep, valid=self.valid,
            objective=list(self.objective[: self.n_objective]), launches=self.launches,
        )


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "fgbd_abi_version": (ctypes.c_int32, []),
    "fgbd_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "fgbd_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "fgbd_ctx_create": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    "fgbd_ctx_destroy": (None, [_P]),
    "fgbd_last_error": (ctypes.c_char_p, [_P]),
    "fgbd_build_graph": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "fgbd_estimate_noise": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "fgbd_select_filter": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_int32), _P]),
    "fgbd_denoise": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P]),
    "fgbd_run": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
    "fgbd_run_reuse": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
    "fgbd_run_host": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
    "fgbd_debug_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int64]),
    "fgbd_debug_div": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    "fgbd_debug_moments": (ctypes.c_int, [_P, _P, _P, _P]),
    "fgbd_run_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_P),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _P]),
    "fgbd_tune_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_P),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _P, _P]),
    "fgbd_get_batch_shape": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P]),
    "fgbd_set_batch_shape": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P]),
    "fgbd_filter_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                           _P, _P]),
    "fgbd_filter_backward": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "fgbd_sync": (ctypes.c_int, [_P, _P]),
    "fgbd_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats), _P]),
    "fgbd_graph_csr_copy": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _P]),
    "fgbd_graph_export": (ctypes.c_int, [_P, ctypes.POINTER(_P), _P]),
    "fgbd_graph_csr": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_double)]),
    "fgbd_graph_free": (None, [_P]),
    "fgbd_get_orders": (ctypes.c_int, [_P, _P, _P]),
    "fgbd_get_fslr": (ctypes.c_int, [_P, _P, _P, _P]),
    "fgbd_set_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
    "fgbd_get_timings": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P, _P]),
    "fgbd_scan_orders_static": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P]),
}
NAME_LEN = 32
TIMING_CAP = 256


def lib() -> ctypes.CDLL:
    """Load libfgbd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2401_09721_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        if handle.fgbd_abi_version() != ABI_VERSION:
            raise RuntimeError(f"{LIB_PATH} has ABI {handle.fgbd_abi_version()}, this binding expects "
                               f"{ABI_VERSION}: rebuild it")
        _lib = handle
    return _lib


def _check(status: int, where: str, ctx=None):
    if status != 0:
        detail = ""
        if ctx is not None and status == 4:
            detail = (lib().fgbd_last_error(ctx) or b"").decode(errors="replace")
        raise FgbdError(status, where, detail)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return FGBD_U8
    if t.dtype == torch.float32:
        return FGBD_F32
    raise TypeError(f"colours must be uint8 or float32, not {t.dtype}")


def _need_cuda(t: torch.Tensor, name: str, shape_n=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_n is not None and tuple(t.shape) != (shape_n, 3):
        raise ValueError(f"{name} must have shape [{shape_n}, 3], got {tuple(t.shape)}")


# ---------------------------------------------------------------- C-named functions

def fgbd_params_default() -> Params:
    p = Params()
    _check(lib().fgbd_params_default(ctypes.byref(p)), "fgbd_params_default")
    return p


def fgbd_ctx_create(capacity: int, params: Params | None = None) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(lib().fgbd_ctx_create(int(capacity), ctypes.byref(params) if params else None, ctypes.byref(out)),
           "fgbd_ctx_create")
    return out


def fgbd_ctx_destroy(ctx) -> None:
    lib().fgbd_ctx_destroy(ctx)


def fgbd_build_graph(ctx, xyz: torch.Tensor, stream=None) -> None:
    if xyz.dtype != torch.int32:
        raise TypeError("xyz must be int32")
    _need_cuda(xyz, "xyz", xyz.shape[0])
    _check(lib().fgbd_build_graph(ctx, _ptr(xyz), xyz.shape[0], _stream(stream)), "fgbd_build_graph", ctx)


def fgbd_estimate_noise(ctx, rgb: torch.Tensor, sigma_out: torch.Tensor | None = None, stream=None,
                        host: bool = False):
    """Enqueue the noise estimate; with host=True also synchronise and return sigma_est (float)."""
    _need_cuda(rgb, "rgb")
    if sigma_out is not None and (sigma_out.dtype != torch.float64 or not sigma_out.is_cuda):
        raise TypeError("sigma_out must be a CUDA float64 tensor")
    h = ctypes.c_double() if host else None
    _check(lib().fgbd_estimate_noise(ctx, _ptr(rgb), _dtype_code(rgb), _ptr(sigma_out),
                                     ctypes.byref(h) if host else None, _stream(stream)),
           "fgbd_estimate_noise", ctx)
    return h.value if host else None


def fgbd_select_filter(ctx, rgb: torch.Tensor, sigma_est: torch.Tensor | None = None,
                       q_out: torch.Tensor | None = None, stream=None, host: bool = False):
    """Enqueue the q search; with host=True also synchronise and return q* (int)."""
    _need_cuda(rgb, "rgb")
    if sigma_est is not None and (sigma_est.dtype != torch.float64 or not sigma_est.is_cuda):
        raise TypeError("sigma_est must be a CUDA float64 tensor")
    if q_out is not None and (q_out.dtype != torch.int32 or not q_out.is_cuda):
        raise TypeError("q_out must be a CUDA int32 tensor")
    h = ctypes.c_int32() if host else None
    _check(lib().fgbd_select_filter(ctx, _ptr(rgb), _dtype_code(rgb), _ptr(sigma_est), _ptr(q_out),
                                    ctypes.byref(h) if host else None, _stream(stream)), "fgbd_select_filter", ctx)
    return h.value if host else None


def fgbd_denoise(ctx, rgb_in: torch.Tensor | None, q: int, rgb_out: torch.Tensor, stream=None) -> None:
    _need_cuda(rgb_out, "rgb_out")
    in_code = FGBD_U8
    if rgb_in is not None:
        _need_cuda(rgb_in, "rgb_in")
        in_code = _dtype_code(rgb_in)
    _check(lib().fgbd_denoise(ctx, _ptr(rgb_in), in_code, int(q), _ptr(rgb_out), _dtype_code(rgb_out),
                              _stream(stream)), "fgbd_denoise", ctx)


def fgbd_run(ctx, xyz: torch.Tensor, rgb_in: torch.Tensor, rgb_out: torch.Tensor, stream=None) -> None:
    if xyz.dtype != torch.int32:
        raise TypeError("xyz must be int32")
    n = xyz.shape[0]
    _need_cuda(xyz, "xyz", n)
    _need_cuda(rgb_in, "rgb_in", n)
    _need_cuda(rgb_out, "rgb_out", n)
    _check(lib().fgbd_run(ctx, _ptr(xyz), n, _ptr(rgb_in), _dtype_code(rgb_in), _ptr(rgb_out),
                          _dtype_code(rgb_out), _stream(stream)), "fgbd_run", ctx)


def fgbd_run_reuse(ctx, xyz: torch.Tensor, rgb_in: torch.Tensor, rgb_out: torch.Tensor, stream=None) -> None:
    if xyz.dtype != torch.int32:
        raise TypeError("xyz must be int32")
    n = xyz.shape[0]
    _need_cuda(xyz, "xyz", n)
    _need_cuda(rgb_in, "rgb_in", n)
    _need_cuda(rgb_out, "rgb_out", n)
    _check(lib().fgbd_run_reuse(ctx, _ptr(xyz), n, _ptr(rgb_in), _dtype_code(rgb_in), _ptr(rgb_out),
                                _dtype_code(rgb_out), _stream(stream)), "fgbd_run_reuse", ctx)


def _need_host(t: torch.Tensor, name: str, n: int) -> None:
    if t.device.type != "cpu" or not t.is_contiguous() or tuple(t.shape) != (n, 3):
        raise ValueError(f"{name} must be a contiguous [n, 3] CPU tensor")


def fgbd_run_host(ctx, xyz: torch.Tensor, rgb_in: torch.Tensor, rgb_out: torch.Tensor, stream=None) -> None:
    """fgbd_run on host tensors (pin them for asynchronous copies); see fgbd_run_host in fgbd.h
    for when the buffers are free again."""
    if xyz.dtype != torch.int32:
        raise TypeError("xyz must be int32")
    n = xyz.shape[0]
    _need_host(xyz, "xyz", n)
    _need_host(rgb_in, "rgb_in", n)
    _need_host(rgb_out, "rgb_out", n)
    _check(lib().fgbd_run_host(ctx, _ptr(xyz), n, _ptr(rgb_in), _dtype_code(rgb_in), _ptr(rgb_out),
                               _dtype_code(rgb_out), _stream(stream)), "fgbd_run_host", ctx)


BATCH_MAX = 64  # FGBD_BATCH_MAX


def _batch_args(ctxs, xyzs, rgbs_in, rgbs_out):
    count = len(ctxs)
    if not (len(xyzs) == len(rgbs_in) == len(rgbs_out) == count):
        raise ValueError("one xyz, rgb_in and rgb_out per context")
    for xyz, ci, co in zip(xyzs, rgbs_in, rgbs_out):
        if xyz.dtype != torch.int32:
            raise TypeError("xyz must be int32")
        n = xyz.shape[0]
        _need_cuda(xyz, "xyz", n)
        _need_cuda(ci, "rgb_in", n)
        _need_cuda(co, "rgb_out", n)

    def arr(t, vals):
        return (t * count)(*[v.value if isinstance(v, ctypes.c_void_p) else v for v in vals])

    return (arr(_P, ctxs), arr(_P, [_ptr(x) for x in xyzs]), arr(ctypes.c_int64, [x.shape[0] for x in xyzs]),
            arr(_P, [_ptr(c) for c in rgbs_in]), arr(ctypes.c_int32, [_dtype_code(c) for c in rgbs_in]),
            arr(_P, [_ptr(c) for c in rgbs_out]), arr(ctypes.c_int32, [_dtype_code(c) for c in rgbs_out]), count)


def fgbd_run_batch(ctxs, xyzs, rgbs_in, rgbs_out, stream=None) -> None:
    """fgbd_run on several frames at once, frame f in context ctxs[f] (handles)."""
    _check(lib().fgbd_run_batch(*_batch_args(ctxs, xyzs, rgbs_in, rgbs_out), _stream(stream)), "fgbd_run_batch")


def fgbd_tune_batch(ctxs, xyzs, rgbs_in, rgbs_out, stream=None) -> dict:
    """Time candidate block shapes on this batch and keep the fastest (see fgbd.h)."""
    out = BatchShape()
    _check(lib().fgbd_tune_batch(*_batch_args(ctxs, xyzs, rgbs_in, rgbs_out), _stream(stream), ctypes.byref(out)),
           "fgbd_tune_batch")
    return out.as_dict()


def fgbd_get_batch_shape(device: int, mean_points: int) -> dict:
    out = BatchShape()
    _check(lib().fgbd_get_batch_shape(int(device), int(mean_points), ctypes.byref(out)), "fgbd_get_batch_shape")
    return out.as_dict()


def fgbd_set_batch_shape(device: int, mean_points: int, shape: dict | None) -> None:
    if shape is None:
        _check(lib().fgbd_set_batch_shape(int(device), int(mean_points), None), "fgbd_set_batch_shape")
        return
    b = BatchShape()
    b.seg_frames = int(shape.get("seg_frames", 16))
    b.scatter_threads = int(shape["scatter_threads"])
    b.filter_threads = int(shape["filter_threads"])
    b.filter_blocks_per_sm = int(shape["filter_blocks_per_sm"])
    _check(lib().fgbd_set_batch_shape(int(device), int(mean_points), ctypes.byref(b)), "fgbd_set_batch_shape")


def fgbd_filter_forward(ctx, rgb_in: torch.Tensor, q: int, alpha: float, sigma: float, checkpoint: int,
                        rgb_out: torch.Tensor, n: int, stream=None) -> None:
    if rgb_in.dtype != torch.float32 or rgb_out.dtype != torch.float32:
        raise TypeError("the differentiable filter takes float32 colours")
    _need_cuda(rgb_in, "rgb_in", n)
    _need_cuda(rgb_out, "rgb_out", n)
    _check(lib().fgbd_filter_forward(ctx, _ptr(rgb_in), int(q), float(alpha), float(sigma), int(checkpoint),
                                     _ptr(rgb_out), _stream(stream)), "fgbd_filter_forward", ctx)


def fgbd_filter_backward(ctx, grad_out: torch.Tensor, grad_in: torch.Tensor, grad_params: torch.Tensor, n: int,
                         stream=None) -> None:
    if grad_out.dtype != torch.float32 or grad_in.dtype != torch.float32 or grad_params.dtype != torch.float64:
        raise TypeError("float32 colour gradients and a float64 [2] parameter gradient")
    _need_cuda(grad_out, "grad_out", n)
    _need_cuda(grad_in, "grad_in", n)
    if not grad_params.is_cuda or grad_params.numel() < 2:
        raise ValueError("grad_params must be a CUDA float64 tensor of 2 entries")
    _check(lib().fgbd_filter_backward(ctx, _ptr(grad_out), _ptr(grad_in), _ptr(grad_params), _stream(stream)),
           "fgbd_filter_backward", ctx)


class GraphFilter(torch.autograd.Function):
    """x_q = ((1 - alpha) I + alpha D^-1 W(sigma))^q rgb on a context's graph.

    Differentiable in rgb (float32 [n, 3], input order), alpha and sigma (Python
    floats or CPU tensors; sigma = 0 means sigma_g).  The backward pass runs
    the library's adjoint kernels and is valid for the context's last forward
    call only.
    """

    @staticmethod
    def forward(fctx, rgb, alpha, sigma, context, q, checkpoint):
        a = float(alpha)
        sg = float(sigma)
        out = torch.empty_like(rgb)
        fgbd_filter_forward(context.handle, rgb.contiguous(), q, a, sg, checkpoint, out, context.n)
        context._diff_token = getattr(context, "_diff_token", 0) + 1
        fctx.context = context
        fctx.token = context._diff_token
        meta = lambda t: (t.device, t.dtype, t.shape) if isinstance(t, torch.Tensor) else None
        fctx.alpha_meta, fctx.sigma_meta = meta(alpha), meta(sigma)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        context = fctx.context
        if getattr(context, "_diff_token", None) != fctx.token:
            raise RuntimeError("the context ran another filter forward since this one; backward needs its state")
        grad_in = torch.empty_like(grad_out)
        gp = torch.zeros(2, dtype=torch.float64, device=grad_out.device)
        fgbd_filter_backward(context.handle, grad_out.contiguous(), grad_in, gp, context.n)
        like = lambda v, m: None if m is None else v.to(device=m[0], dtype=m[1]).reshape(m[2])
        ga, gs = like(gp[0], fctx.alpha_meta), like(gp[1], fctx.sigma_meta)
        return grad_in, ga, gs, None, None, None


def fgbd_sync(ctx, stream=None) -> None:
    _check(lib().fgbd_sync(ctx, _stream(stream)), "fgbd_sync", ctx)


def fgbd_get_stats(ctx, stream=None) -> dict:
    s = Stats()
    _check(lib().fgbd_get_stats(ctx, ctypes.byref(s), _stream(stream)), "fgbd_get_stats", ctx)
    return s.as_dict()


def fgbd_graph_csr_copy(ctx, n: int, device, with_weights: bool = True, stream=None):
    nnz = ctypes.c_int64()
    _check(lib().fgbd_graph_csr_copy(ctx, None, None, None, 0, ctypes.byref(nnz), _stream(stream)),
           "fgbd_graph_csr_copy", ctx)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=device)
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    w = torch.empty(max(nnz.value, 1), dtype=torch.float32, device=device) if with_weights else None
    _check(lib().fgbd_graph_csr_copy(ctx, _ptr(row_ptr), _ptr(col), _ptr(w), col.numel(), ctypes.byref(nnz),
                                     _stream(stream)), "fgbd_graph_csr_copy", ctx)
    return row_ptr, col[: nnz.value], (w[: nnz.value] if w is not None else None)


class _DeviceArray:
    """A borrowed device array, exposed through __cuda_array_interface__ so that
    torch.as_tensor views it without a copy; it keeps its owner alive."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2}


class Graph:
    """An exported graph (fgbd_graph): CSR in input order, the Eq. 4 weights and
    sigma_g.  row_ptr, col and w are tensors viewing the library's device
    memory (no copy); they stay valid while this object (or a view) is alive."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device
        rp, col, w = _P(), _P(), _P()
        n, nnz, sg = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().fgbd_graph_csr(handle, ctypes.byref(rp), ctypes.byref(col), ctypes.byref(w), ctypes.byref(n),
                                    ctypes.byref(nnz), ctypes.byref(sg)), "fgbd_graph_csr")
        self.n, self.nnz, self.sigma_g = n.value, nnz.value, sg.value

        def view(ptr, count, typestr, dtype):
            if not ptr.value or count == 0:
                return torch.empty(count, dtype=dtype, device=device)
            return torch.as_tensor(_DeviceArray(ptr.value, count, typestr, self), device=device)

        self.row_ptr = view(rp, self.n + 1 if self.n > 0 else 0, "<i8", torch.int64)
        self.col = view(col, self.nnz, "<i4", torch.int32)
        self.w = view(w, self.nnz, "<f4", torch.float32)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h is not None:
            try:
                lib().fgbd_graph_free(h)
            except Exception:
                pass


def fgbd_graph_export(ctx, device, stream=None) -> Graph:
    out = _P()
    _check(lib().fgbd_graph_export(ctx, ctypes.byref(out), _stream(stream)), "fgbd_graph_export", ctx)
    return Graph(out, device)


def fgbd_get_orders(ctx, n: int, device, stream=None) -> torch.Tensor:
    out = torch.empty((3, max(n, 1)), dtype=torch.int32, device=device)
    _check(lib().fgbd_get_orders(ctx, _ptr(out), _stream(stream)), "fgbd_get_orders", ctx)
    return out[:, :n]


def fgbd_get_fslr(ctx, n: int, device, stream=None):
    spread = torch.empty(max(n, 1), dtype=torch.float32, device=device)
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device=device)
    _check(lib().fgbd_get_fslr(ctx, _ptr(spread), _ptr(keep), _stream(stream)), "fgbd_get_fslr", ctx)
    return spread[:n], keep[:n]


def fgbd_set_timing(ctx, enable: bool) -> None:
    _check(lib().fgbd_set_timing(ctx, 1 if enable else 0), "fgbd_set_timing", ctx)


def fgbd_get_timings(ctx) -> list:
    """[(kernel name, milliseconds)] of the launches timed since the last call."""
    names = ctypes.create_string_buffer(TIMING_CAP * NAME_LEN)
    ms = (ctypes.c_float * TIMING_CAP)()
    count = ctypes.c_int32()
    _check(lib().fgbd_get_timings(ctx, TIMING_CAP, ctypes.byref(count), names, ms), "fgbd_get_timings", ctx)
    out = []
    for i in range(count.value):
        raw = names.raw[i * NAME_LEN:(i + 1) * NAME_LEN].split(b"\0", 1)[0]
        out.append((raw.decode(), float(ms[i])))
    return out


# ---------------------------------------------------------------- convenience wrapper

class Context:
    """One FGBD context on the current CUDA device, for frames of up to ``capacity`` points."""

    def __init__(self, capacity: int, bits: int = 10, window: int = 1, fslr_factor: float = 2.0,
                 q_max: int = 64, variant: int = 0, flags: int = 0):
        p = fgbd_params_default()
        p.bits, p.window, p.fslr_factor, p.q_max, p.variant = bits, window, fslr_factor, q_max, variant
        p.flags = flags
        self.params = p
        self.capacity = int(capacity)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle = fgbd_ctx_create(capacity, p)
        self.n = 0

    def close(self):
        if getattr(self, "handle", None):
            fgbd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_graph(self, xyz, stream=None):
        fgbd_build_graph(self.handle, xyz, stream)
        self.n = xyz.shape[0]

    def estimate_noise(self, rgb, sigma_out=None, stream=None, host=False):
        return fgbd_estimate_noise(self.handle, rgb, sigma_out, stream, host)

    def select_filter(self, rgb, sigma_est=None, q_out=None, stream=None, host=False):
        return fgbd_select_filter(self.handle, rgb, sigma_est, q_out, stream, host)

    def denoise(self, rgb_in, q, out_dtype=torch.float32, out=None, stream=None):
        if out is None:
            out = torch.empty((self.n, 3), dtype=out_dtype, device=self.device)
        fgbd_denoise(self.handle, rgb_in, q, out, stream)
        return out

    def run(self, xyz, rgb_in, out_dtype=torch.float32, out=None, stream=None):
        if out is None:
            out = torch.empty((xyz.shape[0], 3), dtype=out_dtype, device=self.device)
        fgbd_run(self.handle, xyz, rgb_in, out, stream)
        self.n = xyz.shape[0]
        return out

    def sync(self, stream=None):
        fgbd_sync(self.handle, stream)

    def set_wait_limit(self, ns: int):
        """Testing: the time after which every device-side wait gives up (FGBD_ETIMEOUT)."""
        _check(lib().fgbd_debug_set_wait_limit(self.handle, int(ns)), "fgbd_debug_set_wait_limit", self.handle)

    def run_host(self, xyz, rgb_in, out, stream=None):
        """fgbd_run on host (CPU) tensors; `out` is complete after sync() or two calls later."""
        fgbd_run_host(self.handle, xyz, rgb_in, out, stream)
        self.n = xyz.shape[0]
        return out

    def run_reuse(self, xyz, rgb_in, out_dtype=torch.float32, out=None, stream=None):
        """Build this frame's graph and filter it with the last selected q (streaming mode)."""
        if out is None:
            out = torch.empty((xyz.shape[0], 3), dtype=out_dtype, device=self.device)
        fgbd_run_reuse(self.handle, xyz, rgb_in, out, stream)
        self.n = xyz.shape[0]
        return out

    def filter(self, rgb, alpha=0.5, sigma=0.0, q=1, checkpoint=1):
        """Differentiable filter on this context's graph (GraphFilter)."""
        return GraphFilter.apply(rgb, alpha, sigma, self, q, checkpoint)

    @staticmethod
    def run_batch(contexts, xyzs, rgbs_in, out_dtype=torch.float32, outs=None, stream=None):
        """fgbd_run_batch over Context objects; returns the outputs."""
        if outs is None:
            outs = [torch.empty((x.shape[0], 3), dtype=out_dtype, device=c.device) for c, x in zip(contexts, xyzs)]
        fgbd_run_batch([c.handle for c in contexts], xyzs, rgbs_in, outs, stream)
        for c, x in zip(contexts, xyzs):
            c.n = x.shape[0]
        return outs

    @staticmethod
    def tune_batch(contexts, xyzs, rgbs_in, out_dtype=torch.float32, outs=None, stream=None):
        """fgbd_tune_batch over Context objects; returns (the chosen shapes, the outputs)."""
        if outs is None:
            outs = [torch.empty((x.shape[0], 3), dtype=out_dtype, device=c.device) for c, x in zip(contexts, xyzs)]
        shape = fgbd_tune_batch([c.handle for c in contexts], xyzs, rgbs_in, outs, stream)
        for c, x in zip(contexts, xyzs):
            c.n = x.shape[0]
        return shape, outs

    def stats(self, stream=None) -> dict:
        return fgbd_get_stats(self.handle, stream)

    def graph_csr(self, with_weights=True, stream=None):
        return fgbd_graph_csr_copy(self.handle, self.n, self.device, with_weights, stream)

    def export_graph(self, stream=None) -> Graph:
        return fgbd_graph_export(self.handle, self.device, stream)

    def orders(self, stream=None):
        return fgbd_get_orders(self.handle, self.n, self.device, stream)

    def fslr(self, stream=None):
        return fgbd_get_fslr(self.handle, self.n, self.device, stream)

    def set_timing(self, enable: bool):
        fgbd_set_timing(self.handle, enable)

    def debug_moments(self):
        """(s2 [D, D], s1 [D], patch count) of the last uint8 noise estimate, exact int64 (testing)."""
        D = self.stats()["patch_dim"]
        s2 = np.zeros((D, D), dtype=np.int64)
        s1 = np.zeros(D, dtype=np.int64)
        npat = ctypes.c_int64(0)
        _check(lib().fgbd_debug_moments(self.handle, s2.ctypes.data, s1.ctypes.data, ctypes.byref(npat)),
               "fgbd_debug_moments")
        return s2, s1, int(npat.value)

    def timings(self) -> list:
        return fgbd_get_timings(self.handle)


def fgbd_debug_div(a: torch.Tensor, b: torch.Tensor, stream=None):
    """(div_newton(a, b), CUDA's a / b) elementwise on CUDA float64 tensors (testing)."""
    if a.dtype != torch.float64 or b.dtype != torch.float64 or a.shape != b.shape or not (a.is_cuda and b.is_cuda):
        raise TypeError("two CUDA float64 tensors of one shape")
    a, b = a.contiguous(), b.contiguous()
    qn, qd = torch.empty_like(a), torch.empty_like(a)
    _check(lib().fgbd_debug_div(_ptr(a), _ptr(b), _ptr(qn), _ptr(qd), a.numel(), _stream(stream)), "fgbd_debug_div")
    return qn, qd
