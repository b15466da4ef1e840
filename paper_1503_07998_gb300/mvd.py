"""Python binding of the C ABI in ``include/mvd.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``_lib/libmvd.so``.  Functions keep the C names; device buffers are torch
CUDA tensors (their ``data_ptr()`` is passed), host buffers numpy arrays or
CPU tensors, and the stream defaults to torch's current stream on the
tensor's device.  Loading fails loudly when the library has not been built:
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmvd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mvd.h")

MVD_OK, MVD_ERR_ARG, MVD_ERR_CUDA, MVD_ERR_NOMEM, MVD_ERR_TIMEOUT, MVD_ERR_STATE, MVD_ERR_UNSUPPORTED = range(7)
BOUNDARY = {"zero": 0, "circular": 1}
DTYPE = {"u16": 0, "f32": 1}
ALGO = {"fused": 0, "plain": 1, "direct": 2, "fft": 3, "tensor": 4, "tf32": 5, "resident": 6}
ORDER = {"simultaneous": 0, "sequential": 1}
VARIANT = {"independent": 0, "efficient_bayesian": 1, "optimization_1": 2, "optimization_2": 3}


class MvdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


class _KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("total_ms", ctypes.c_double), ("launches", ctypes.c_uint64)]


class _Info(ctypes.Structure):
    _fields_ = [
        ("views", ctypes.c_int), ("psf_size", ctypes.c_int),
        ("plane_h", ctypes.c_int), ("plane_w", ctypes.c_int),
        ("iters", ctypes.c_int), ("boundary", ctypes.c_int), ("algo", ctypes.c_int), ("order", ctypes.c_int),
        ("rank", ctypes.c_int * 16), ("blur_groups", ctypes.c_int), ("blur_terms", ctypes.c_int),
        ("tile_h", ctypes.c_int), ("tile_w", ctypes.c_int),
        ("workspace_bytes", ctypes.c_size_t),
        ("variant", ctypes.c_int), ("corr_rank", ctypes.c_int * 16),
        ("flops_blur", ctypes.c_int), ("flops_corr", ctypes.c_int),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1503_07998_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
    L.mvd_create.argtypes = [ctypes.POINTER(vp), i, vp, i, i, i, i, i, f]
    L.mvd_destroy.argtypes = [vp]
    L.mvd_set_algo.argtypes = [vp, i]
    L.mvd_set_rank_tolerance.argtypes = [vp, d]
    L.mvd_set_update_order.argtypes = [vp, i]
    L.mvd_set_variant.argtypes = [vp, i]
    L.mvd_set_weights.argtypes = [vp, vp, i]
    L.mvd_set_axial_psfs.argtypes = [vp, vp, i]
    L.mvd_embed_padded.argtypes = [vp, i, i, i, i, i, i, vp, vp, i, vp]
    L.mvd_crop_planes.argtypes = [vp, i, i, i, i, vp, vp]
    L.mvd_variant_kernels.argtypes = [vp, i, i, i, vp]
    L.mvd_device_status.argtypes = [vp, vp]
    L.mvd_psf_grad.argtypes = [vp, vp, i, i, i, ctypes.POINTER(d), vp, vp, vp]
    L.mvd_set_psfs.argtypes = [vp, vp]
    L.mvd_autotune.argtypes = [vp, vp, i, i, vp]
    L.mvd_batch_create.argtypes = [ctypes.POINTER(vp), vp, i, i, i, f, i]
    L.mvd_batch_tune.argtypes = [vp, vp]
    L.mvd_batch_run.argtypes = [vp, vp]
    L.mvd_batch_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.mvd_batch_destroy.argtypes = [vp]
    L.mvd_batch_set_schedule.argtypes = [vp, i]
    L.mvd_batch_queue_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
    L.mvd_batch_set_wait_budget.argtypes = [vp, ctypes.c_longlong]
    L.mvd_batch_device_status.argtypes = [vp]
    L.mvd_deconvolve_planes_static.argtypes = [i, vp, i, i, i, i, i, f, vp, i, vp, i, i, vp]
    L.mvd_static_device_status.argtypes = [vp]
    L.mvd_static_set_wait_budget.argtypes = [ctypes.c_longlong]
    L.mvd_debug_fail_allocations.argtypes = [i]
    L.mvd_set_wait_budget.argtypes = [vp, ctypes.c_longlong]
    L.mvd_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    L.mvd_reslice.argtypes = [vp, vp, i, i, i, i, i, vp, vp]
    L.mvd_deconvolve_planes.argtypes = [vp, vp, i, vp, i, i, vp]
    L.mvd_run_host.argtypes = [vp, vp, i, i, i, i, vp, i, vp]
    L.mvd_host_chunks.argtypes = [i, ctypes.c_longlong, i, vp, vp, i]
    L.mvd_host_chunks.restype = ctypes.c_int
    L.mvd_psf_factors.argtypes = [vp, i, i, d, vp, vp, i]
    L.mvd_profile_enable.argtypes = [vp, i]
    L.mvd_profile_read.argtypes = [vp, ctypes.POINTER(_KernelStat), i, ctypes.POINTER(i)]
    L.mvd_status_string.argtypes = [i]
    L.mvd_status_string.restype = ctypes.c_char_p
    L.mvd_last_error.argtypes = []
    L.mvd_last_error.restype = ctypes.c_char_p
    L.mvd_launch_count.argtypes = []
    L.mvd_launch_count.restype = ctypes.c_uint64
    for name in ("mvd_create", "mvd_destroy", "mvd_set_algo", "mvd_set_rank_tolerance", "mvd_get_info",
                 "mvd_set_update_order", "mvd_set_variant", "mvd_variant_kernels", "mvd_device_status",
                 "mvd_set_weights", "mvd_embed_padded", "mvd_crop_planes", "mvd_set_axial_psfs", "mvd_set_wait_budget",
                 "mvd_deconvolve_planes_static", "mvd_static_device_status", "mvd_static_set_wait_budget",
                 "mvd_debug_fail_allocations", "mvd_psf_grad", "mvd_set_psfs", "mvd_autotune",
                 "mvd_batch_create", "mvd_batch_tune", "mvd_batch_run", "mvd_batch_info", "mvd_batch_destroy",
                 "mvd_batch_set_schedule", "mvd_batch_queue_info", "mvd_batch_set_wait_budget",
                 "mvd_batch_device_status",
                 "mvd_reslice", "mvd_deconvolve_planes", "mvd_run_host", "mvd_psf_factors",
                 "mvd_profile_enable", "mvd_profile_read"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def header_functions() -> list[str]:
    """Names of the functions declared in include/mvd.h."""
    with open(HEADER) as fh:
        text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(mvd_[a-z0-9_]+)\s*\(", text)))


def _check(status: int, where: str) -> None:
    if status != MVD_OK:
        L = lib()
        detail = L.mvd_last_error().decode() or L.mvd_status_string(status).decode()
        raise MvdError(status, where, detail)


def _stream_of(t, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.uint16:
        return DTYPE["u16"]
    if t.dtype == torch.float32:
        return DTYPE["f32"]
    raise TypeError(f"data must be uint16 or float32, got {t.dtype}")


def _require_cuda(*ts):
    for t in ts:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("device buffers must be contiguous CUDA tensors")


@dataclass
class Info:
    views: int
    psf_size: int
    plane_h: int
    plane_w: int
    iters: int
    boundary: int
    algo: int
    order: int
    rank: list
    blur_groups: int
    blur_terms: int
    tile_h: int
    tile_w: int
    workspace_bytes: int
    variant: int
    corr_rank: list
    flops_blur: int
    flops_corr: int


class Context:
    """Owns an ``mvd_ctx``; created by :func:`mvd_create`."""

    def __init__(self, handle: int, views: int, K: int, H: int, W: int, iters: int):
        self.handle = ctypes.c_void_p(handle)
        self.views, self.K, self.H, self.W, self.iters = views, K, H, W, iters

    def close(self):
        if self.handle and self.handle.value:
            _check(lib().mvd_destroy(self.handle), "mvd_destroy")
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def mvd_create(views: int, psfs, psf_size: int, plane_h: int, plane_w: int, iters: int,
               boundary: str = "zero", eps: float = 1e-6) -> Context:
    p = np.ascontiguousarray(np.asarray(psfs, dtype=np.float32))
    if p.size != views * psf_size * psf_size:
        raise ValueError("psfs must hold views * K * K values")
    h = ctypes.c_void_p()
    _check(lib().mvd_create(ctypes.byref(h), int(views), p.ctypes.data_as(ctypes.c_void_p), int(psf_size),
                            int(plane_h), int(plane_w), int(iters), BOUNDARY[boundary], float(eps)), "mvd_create")
    return Context(h.value, views, psf_size, plane_h, plane_w, iters)


def mvd_destroy(ctx: Context) -> None:
    ctx.close()


def mvd_set_algo(ctx: Context, algo: str) -> None:
    _check(lib().mvd_set_algo(ctx.handle, ALGO[algo]), "mvd_set_algo")


def mvd_autotune(ctx: Context, data, stream=None) -> str:
    """Time the routes that can take this context's PSFs on `data` and keep
    the fastest; returns its name."""
    _require_cuda(data)
    _check(lib().mvd_autotune(ctx.handle, ctypes.c_void_p(data.data_ptr()), _dtype_code(data), data.shape[1],
                              _stream_of(data, stream)), "mvd_autotune")
    algo = mvd_get_info(ctx).algo
    return {v: k for k, v in ALGO.items()}[algo]


def mvd_set_update_order(ctx: Context, order: str) -> None:
    _check(lib().mvd_set_update_order(ctx.handle, ORDER[order]), "mvd_set_update_order")


def mvd_set_variant(ctx: Context, variant: str) -> None:
    """Select the MV-RL variant (keys of VARIANT; default "independent")."""
    _check(lib().mvd_set_variant(ctx.handle, VARIANT[variant]), "mvd_set_variant")


def mvd_set_axial_psfs(ctx: Context, axial) -> None:
    """3D route: [V][Ka] profiles along the rotation axis (host array), or
    None for the plane-wise method."""
    if axial is None:
        _check(lib().mvd_set_axial_psfs(ctx.handle, None, 0), "mvd_set_axial_psfs")
        return
    a = np.ascontiguousarray(np.asarray(axial, dtype=np.float32))
    if a.ndim != 2 or a.shape[0] != ctx.views:
        raise ValueError("axial profiles must be [V][Ka]")
    _check(lib().mvd_set_axial_psfs(ctx.handle, a.ctypes.data_as(ctypes.c_void_p), a.shape[1]), "mvd_set_axial_psfs")


def mvd_set_weights(ctx: Context, weights) -> None:
    """Per-pixel view weights [V][P][H][W] (CUDA float32 tensor, kept by
    reference on the context; P = 1: one plane per view for every plane) or
    None to clear."""
    if weights is None:
        _check(lib().mvd_set_weights(ctx.handle, None, 0), "mvd_set_weights")
        ctx._weights = None
        return
    _require_cuda(weights)
    import torch
    if weights.dtype != torch.float32 or not weights.is_contiguous():
        raise ValueError("weights must be contiguous float32")
    V, P, H, W = weights.shape
    if V != ctx.views or (H, W) != (ctx.H, ctx.W):
        raise ValueError("weights must be [V][P][H][W] of the context's views and plane")
    _check(lib().mvd_set_weights(ctx.handle, ctypes.c_void_p(weights.data_ptr()), P), "mvd_set_weights")
    ctx._weights = weights


def mvd_embed_padded(planes, pad: int, per_plane_weights: bool = False, stream=None):
    """planes [V][P][H][W] (CUDA uint16/float32) -> (padded planes
    [V][P][H+2pad][W+2pad], float32 weights 1 on the data: [V][1][..] shared
    by every plane, or [V][P][..] with per_plane_weights)."""
    import torch
    _require_cuda(planes)
    V, P, H, W = planes.shape
    dst = torch.empty((V, P, H + 2 * pad, W + 2 * pad), dtype=planes.dtype, device=planes.device)
    wp = P if per_plane_weights else 1
    w = torch.empty((V, wp, H + 2 * pad, W + 2 * pad), dtype=torch.float32, device=planes.device)
    _check(lib().mvd_embed_padded(ctypes.c_void_p(planes.data_ptr()), _dtype_code(planes), V, P, H, W, int(pad),
                                  ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(w.data_ptr()), wp,
                                  _stream_of(planes, stream)), "mvd_embed_padded")
    return dst, w


def mvd_crop_planes(est, pad: int, stream=None):
    """est [P][Hp][Wp] (CUDA float32) -> [P][Hp-2pad][Wp-2pad]."""
    import torch
    _require_cuda(est)
    P, Hp, Wp = est.shape
    out = torch.empty((P, Hp - 2 * pad, Wp - 2 * pad), dtype=torch.float32, device=est.device)
    _check(lib().mvd_crop_planes(ctypes.c_void_p(est.data_ptr()), P, Hp, Wp, int(pad), ctypes.c_void_p(out.data_ptr()),
                                 _stream_of(est, stream)), "mvd_crop_planes")
    return out


def mvd_variant_kernels(psfs, variant: str) -> np.ndarray:
    """Host-only: the kernels X_v [V][K][K] (unit sum) the library builds for
    a variant of the given PSFs."""
    p = np.ascontiguousarray(np.asarray(psfs, dtype=np.float32))
    V, K, _ = p.shape
    out = np.zeros_like(p)
    _check(lib().mvd_variant_kernels(p.ctypes.data_as(ctypes.c_void_p), V, K, VARIANT[variant],
                                     out.ctypes.data_as(ctypes.c_void_p)), "mvd_variant_kernels")
    return out


def mvd_device_status(ctx: Context, stream=None) -> None:
    """Raise MvdError (MVD_ERR_TIMEOUT) if a kernel's bounded wait ran out."""
    import torch
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    _check(lib().mvd_device_status(ctx.handle, ctypes.c_void_p(s)), "mvd_device_status")


def mvd_set_wait_budget(ctx: Context, cycles: int) -> None:
    _check(lib().mvd_set_wait_budget(ctx.handle, int(cycles)), "mvd_set_wait_budget")


def mvd_set_rank_tolerance(ctx: Context, tol: float) -> None:
    _check(lib().mvd_set_rank_tolerance(ctx.handle, float(tol)), "mvd_set_rank_tolerance")


def mvd_get_info(ctx: Context) -> Info:
    inf = _Info()
    _check(lib().mvd_get_info(ctx.handle, ctypes.byref(inf)), "mvd_get_info")
    return Info(inf.views, inf.psf_size, inf.plane_h, inf.plane_w, inf.iters, inf.boundary, inf.algo, inf.order,
                list(inf.rank)[:min(16, inf.views)], inf.blur_groups, inf.blur_terms, inf.tile_h, inf.tile_w,
                int(inf.workspace_bytes), inf.variant, list(inf.corr_rank)[:min(16, inf.views)], inf.flops_blur,
                inf.flops_corr)


def mvd_reslice(ctx: Context, stacks, planes, stream=None) -> None:
    """stacks [V][Z][Y][X] -> planes [V][Y][Z][X] (CUDA tensors, same dtype)."""
    _require_cuda(stacks, planes)
    V, Z, Y, X = stacks.shape
    if tuple(planes.shape) != (V, Y, Z, X) or planes.dtype != stacks.dtype:
        raise ValueError("planes must be [V][Y][Z][X] of the stacks' dtype")
    _check(lib().mvd_reslice(ctx.handle, ctypes.c_void_p(stacks.data_ptr()), _dtype_code(stacks), V, Z, Y, X,
                             ctypes.c_void_p(planes.data_ptr()), _stream_of(stacks, stream)), "mvd_reslice")


def mvd_deconvolve_planes(ctx: Context, data, estimate, init_mean: bool = True, stream=None) -> None:
    """data [V][P][H][W] (uint16/float32), estimate [P][H][W] float32, in place."""
    import torch
    _require_cuda(data, estimate)
    V, P, H, W = data.shape
    if V != ctx.views or (H, W) != (ctx.H, ctx.W):
        raise ValueError("data shape does not match the context")
    if tuple(estimate.shape) != (P, H, W) or estimate.dtype != torch.float32:
        raise ValueError("estimate must be float32 [P][H][W]")
    _check(lib().mvd_deconvolve_planes(ctx.handle, ctypes.c_void_p(data.data_ptr()), _dtype_code(data),
                                       ctypes.c_void_p(estimate.data_ptr()), P, int(bool(init_mean)),
                                       _stream_of(data, stream)), "mvd_deconvolve_planes")


def mvd_deconvolve_planes_static(psfs, data, estimate, iters: int, boundary: str = "zero", eps: float = 1e-6,
                                 init_mean: bool = True, stream=None) -> None:
    """Context-free fused deconvolution that allocates no GPU memory, for
    callers that may not call cudaMalloc (see include/mvd.h): its scratch is
    a 32 MiB static device array shared by all calls, so calls must not
    overlap on the GPU.  data [V][P][H][W] uint16/float32 and estimate
    [P][H][W] float32 are CUDA tensors; psfs [V][K][K] is host data."""
    import torch
    _require_cuda(data, estimate)
    V, P, H, W = data.shape
    p = np.ascontiguousarray(np.asarray(psfs, dtype=np.float32))
    if p.ndim != 3 or p.shape[0] != V or p.shape[1] != p.shape[2]:
        raise ValueError("psfs must be [V][K][K]")
    if tuple(estimate.shape) != (P, H, W) or estimate.dtype != torch.float32:
        raise ValueError("estimate must be float32 [P][H][W]")
    _check(lib().mvd_deconvolve_planes_static(V, p.ctypes.data_as(ctypes.c_void_p), p.shape[1], H, W, int(iters),
                                              BOUNDARY[boundary], float(eps), ctypes.c_void_p(data.data_ptr()),
                                              _dtype_code(data), ctypes.c_void_p(estimate.data_ptr()), P,
                                              int(bool(init_mean)), _stream_of(data, stream)),
           "mvd_deconvolve_planes_static")


def mvd_static_device_status(stream=None) -> None:
    """Raise MvdError (MVD_ERR_TIMEOUT) if a tile wait of the last
    mvd_deconvolve_planes_static call ran out; waits for the stream."""
    import torch
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    _check(lib().mvd_static_device_status(ctypes.c_void_p(s)), "mvd_static_device_status")


def mvd_static_set_wait_budget(cycles: int) -> None:
    _check(lib().mvd_static_set_wait_budget(int(cycles)), "mvd_static_set_wait_budget")


def mvd_debug_fail_allocations(n: int) -> None:
    """Test hook: the next n device allocations of the library fail."""
    _check(lib().mvd_debug_fail_allocations(int(n)), "mvd_debug_fail_allocations")


def mvd_run_host(ctx: Context, stacks_host, out_host, chunk_planes: int = 0, stream=None) -> None:
    """Host stacks [V][Z][Y][X] -> host result [Y][Z][X] float32 (torch CPU tensors,
    ideally pinned)."""
    import torch
    if stacks_host.is_cuda or out_host.is_cuda:
        raise ValueError("mvd_run_host takes host tensors")
    V, Z, Y, X = stacks_host.shape
    if tuple(out_host.shape) != (Y, Z, X) or out_host.dtype != torch.float32:
        raise ValueError("out must be float32 [Y][Z][X]")
    if not (stacks_host.is_contiguous() and out_host.is_contiguous()):
        raise ValueError("host buffers must be contiguous")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().mvd_run_host(ctx.handle, ctypes.c_void_p(stacks_host.data_ptr()), _dtype_code(stacks_host),
                              Z, Y, X, ctypes.c_void_p(out_host.data_ptr()), int(chunk_planes),
                              ctypes.c_void_p(int(stream))), "mvd_run_host")


def mvd_host_chunks(ny: int, plane_bytes: int, chunk_planes: int = 0):
    """The chunks of planes mvd_run_host uses: a list of (first plane, count)."""
    y0 = np.zeros(max(1, ny), dtype=np.int32)
    n = np.zeros(max(1, ny), dtype=np.int32)
    k = lib().mvd_host_chunks(int(ny), int(plane_bytes), int(chunk_planes), y0.ctypes.data_as(ctypes.c_void_p),
                              n.ctypes.data_as(ctypes.c_void_p), int(max(1, ny)))
    if k < 0:
        raise MvdError(MVD_ERR_ARG, "mvd_host_chunks", "invalid arguments or too many chunks")
    return [(int(a), int(b)) for a, b in zip(y0[:k], n[:k])]


def mvd_psf_factors(psfs, rank_tol: float = 3e-7):
    """Host-only factorisation: returns (ranks [V], taps [terms][4][K])."""
    p = np.ascontiguousarray(np.asarray(psfs, dtype=np.float32))
    V, K, _ = p.shape
    cap = V * K * 4 * K
    taps = np.zeros(cap, dtype=np.float32)
    ranks = np.zeros(V, dtype=np.int32)
    _check(lib().mvd_psf_factors(p.ctypes.data_as(ctypes.c_void_p), V, K, float(rank_tol),
                                 ranks.ctypes.data_as(ctypes.c_void_p), taps.ctypes.data_as(ctypes.c_void_p), cap),
           "mvd_psf_factors")
    return ranks, taps.reshape(-1, 4, K)


def mvd_profile_enable(ctx: Context, on: bool = True) -> None:
    _check(lib().mvd_profile_enable(ctx.handle, int(bool(on))), "mvd_profile_enable")


def mvd_profile_read(ctx: Context) -> dict:
    """{kernel name: (total_ms, launches)} since profiling was enabled."""
    cap = 32
    arr = (_KernelStat * cap)()
    n = ctypes.c_int(0)
    _check(lib().mvd_profile_read(ctx.handle, arr, cap, ctypes.byref(n)), "mvd_profile_read")
    return {arr[k].name.decode(): (arr[k].total_ms, int(arr[k].launches)) for k in range(min(n.value, cap))}


def mvd_set_psfs(ctx: Context, psfs) -> None:
    p = np.ascontiguousarray(np.asarray(psfs, dtype=np.float32))
    if p.size != ctx.views * ctx.K * ctx.K:
        raise ValueError("psfs must hold views * K * K values")
    _check(lib().mvd_set_psfs(ctx.handle, p.ctypes.data_as(ctypes.c_void_p)), "mvd_set_psfs")


def mvd_psf_grad(ctx: Context, data, checkpoint_every: int = 2, estimate=None, stream=None):
    """Poisson data fit of the deconvolved estimate and its PSF gradient.

    data [V][P][H][W] CUDA tensor.  Returns (loss: float, grad: float32 CUDA
    tensor [V][K][K]); `estimate` ([P][H][W] float32 CUDA) receives psi_T."""
    import torch
    _require_cuda(data)
    V, P, H, W = data.shape
    if V != ctx.views or (H, W) != (ctx.H, ctx.W):
        raise ValueError("data shape does not match the context")
    grad = torch.empty((V, ctx.K, ctx.K), dtype=torch.float32, device=data.device)
    loss = ctypes.c_double(0.0)
    est_ptr = None
    if estimate is not None:
        _require_cuda(estimate)
        if tuple(estimate.shape) != (P, H, W) or estimate.dtype != torch.float32:
            raise ValueError("estimate must be float32 [P][H][W]")
        est_ptr = ctypes.c_void_p(estimate.data_ptr())
    _check(lib().mvd_psf_grad(ctx.handle, ctypes.c_void_p(data.data_ptr()), _dtype_code(data), P,
                              int(checkpoint_every), ctypes.byref(loss), ctypes.c_void_p(grad.data_ptr()),
                              est_ptr, _stream_of(data, stream)), "mvd_psf_grad")
    return loss.value, grad


def mvd_poisson_loss(ctx: Context, data, estimate=None, stream=None) -> float:
    """The Poisson data fit of mvd_psf_grad without its gradient (grad_dev
    NULL: forward iterations and data fit only)."""
    import torch
    _require_cuda(data)
    V, P, H, W = data.shape
    if V != ctx.views or (H, W) != (ctx.H, ctx.W):
        raise ValueError("data shape does not match the context")
    est_ptr = None
    if estimate is not None:
        _require_cuda(estimate)
        if tuple(estimate.shape) != (P, H, W) or estimate.dtype != torch.float32:
            raise ValueError("estimate must be float32 [P][H][W]")
        est_ptr = ctypes.c_void_p(estimate.data_ptr())
    loss = ctypes.c_double(0.0)
    _check(lib().mvd_psf_grad(ctx.handle, ctypes.c_void_p(data.data_ptr()), _dtype_code(data), P, 1,
                              ctypes.byref(loss), None, est_ptr, _stream_of(data, stream)), "mvd_psf_grad")
    return loss.value


def _psf_loss_function():
    import torch

    class PoissonFitOfDeconvolution(torch.autograd.Function):
        """loss(psfs) = Poisson NLL of P_v * (MV-RL estimate after the
        context's iterations) against the data; backward is the library's
        hand-written adjoint (mvd_psf_grad)."""

        @staticmethod
        def forward(fctx, psfs, ctx, data, checkpoint_every):
            mvd_set_psfs(ctx, psfs.detach().to("cpu", torch.float32).numpy())
            if not fctx.needs_input_grad[0]:
                # loss only: the forward iterations and the data fit, no
                # reverse sweep
                loss = mvd_poisson_loss(ctx, data)
                return torch.tensor(loss, dtype=torch.float64, device=psfs.device)
            loss, grad = mvd_psf_grad(ctx, data, checkpoint_every)
            fctx.save_for_backward(grad)
            return torch.tensor(loss, dtype=torch.float64, device=psfs.device)

        @staticmethod
        def backward(fctx, gout):
            (grad,) = fctx.saved_tensors
            g = grad.to(device=gout.device, dtype=torch.float64) * gout
            return g, None, None, None

    return PoissonFitOfDeconvolution


def psf_fit_loss(psfs, ctx: Context, data, checkpoint_every: int = 2):
    """Differentiable PSF-calibration loss (torch.autograd): gradients flow to
    `psfs` ([V][K][K] tensor) through the library's adjoint."""
    return _psf_loss_function().apply(psfs, ctx, data, checkpoint_every)


class _VolumeDesc(ctypes.Structure):
    _fields_ = [("views", ctypes.c_int), ("psf_size", ctypes.c_int), ("psfs_host", ctypes.c_void_p),
                ("plane_h", ctypes.c_int), ("plane_w", ctypes.c_int), ("n_planes", ctypes.c_int),
                ("iters", ctypes.c_int), ("stacks_dev", ctypes.c_void_p), ("planes_dev", ctypes.c_void_p),
                ("estimate_dev", ctypes.c_void_p), ("variant", ctypes.c_int)]


class Batch:
    """Owns an ``mvd_batch`` (see mvd_batch_create); keeps the PSF arrays and
    tensors it was built from alive."""

    def __init__(self, handle, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep

    def close(self):
        if self.handle and self.handle.value:
            _check(lib().mvd_batch_destroy(self.handle), "mvd_batch_destroy")
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mvd_batch_create(volumes, boundary: str = "zero", eps: float = 1e-6, order: str = "simultaneous") -> Batch:
    """volumes: list of dicts with keys psfs ([V][K][K]), iters, estimate
    (CUDA float32 [P][H][W]) and either stacks (CUDA [V][H][P][W]) or planes
    (CUDA [V][P][H][W]); all data of one dtype; optional key variant (a key
    of VARIANT, default "independent")."""
    descs = (_VolumeDesc * len(volumes))()
    keep, dtype = [], None
    for i, v in enumerate(volumes):
        psfs = np.ascontiguousarray(np.asarray(v["psfs"], dtype=np.float32))
        keep.append(psfs)
        est = v["estimate"]
        _require_cuda(est)
        P, H, W = est.shape
        d = descs[i]
        d.views, d.psf_size = psfs.shape[0], psfs.shape[-1]
        d.psfs_host = psfs.ctypes.data
        d.plane_h, d.plane_w, d.n_planes, d.iters = H, W, P, int(v["iters"])
        d.estimate_dev = est.data_ptr()
        d.variant = VARIANT[v.get("variant", "independent")]
        src = v.get("stacks")
        if src is not None:
            _require_cuda(src)
            if tuple(src.shape) != (psfs.shape[0], H, P, W):
                raise ValueError(f"volume {i}: stacks must be [V][H][P][W]")
            d.stacks_dev = src.data_ptr()
        else:
            src = v["planes"]
            _require_cuda(src)
            if tuple(src.shape) != (psfs.shape[0], P, H, W):
                raise ValueError(f"volume {i}: planes must be [V][P][H][W]")
            d.planes_dev = src.data_ptr()
        keep.append(src)
        keep.append(est)
        code = _dtype_code(src)
        if dtype is None:
            dtype = code
        elif code != dtype:
            raise ValueError("all volumes of a batch share one dtype")
    h = ctypes.c_void_p()
    _check(lib().mvd_batch_create(ctypes.byref(h), descs, len(volumes), dtype, BOUNDARY[boundary], float(eps),
                                  ORDER[order]), "mvd_batch_create")
    return Batch(h.value, keep)


def mvd_batch_tune(batch: Batch, stream=None) -> None:
    import torch
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    _check(lib().mvd_batch_tune(batch.handle, ctypes.c_void_p(s)), "mvd_batch_tune")


def mvd_batch_run(batch: Batch, stream=None) -> None:
    import torch
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    _check(lib().mvd_batch_run(batch.handle, ctypes.c_void_p(s)), "mvd_batch_run")


def mvd_batch_info(batch: Batch) -> dict:
    c, m, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().mvd_batch_info(batch.handle, ctypes.byref(c), ctypes.byref(m), ctypes.byref(k)), "mvd_batch_info")
    return {"concurrent": c.value, "max_ctas": m.value, "graph_kernels": k.value}


BATCH_SCHEDULE = {"graph": 0, "queue": 1}


def mvd_batch_set_schedule(batch: Batch, schedule: str) -> None:
    _check(lib().mvd_batch_set_schedule(batch.handle, BATCH_SCHEDULE[schedule]), "mvd_batch_set_schedule")


def mvd_batch_queue_info(batch: Batch) -> dict:
    s, n, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(lib().mvd_batch_queue_info(batch.handle, ctypes.byref(s), ctypes.byref(n), ctypes.byref(q)),
           "mvd_batch_queue_info")
    names = {v: k for k, v in BATCH_SCHEDULE.items()}
    return {"schedule": names.get(s.value, s.value), "queue_volumes": n.value, "queue_items": q.value}


def mvd_batch_set_wait_budget(batch: Batch, cycles: int) -> None:
    _check(lib().mvd_batch_set_wait_budget(batch.handle, int(cycles)), "mvd_batch_set_wait_budget")


def mvd_batch_device_status(batch: Batch) -> None:
    """Raises MvdError (MVD_ERR_TIMEOUT) if a queue wait of the batch ran out."""
    _check(lib().mvd_batch_device_status(batch.handle), "mvd_batch_device_status")


def mvd_batch_destroy(batch: Batch) -> None:
    batch.close()


def mvd_launch_count() -> int:
    return int(lib().mvd_launch_count())


def mvd_status_string(status: int) -> str:
    return lib().mvd_status_string(int(status)).decode()


def mvd_last_error() -> str:
    return lib().mvd_last_error().decode()
