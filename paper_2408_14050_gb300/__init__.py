"""GB300 (sm_103a) fast edge-aware occlusion detection -- Python binding of the C ABI in include/occ.h.

Sippel, Seiler, Kaup, "Fast Edge-Aware Occlusion Detection in the Context of Multispectral Camera Arrays"
(ICIP 2024), Section 3: from a fused center-view disparity map D and the baseline angle alpha of each peripheral
camera, the occlusion sum O (Eq. 5/6) and the mask M = (O > 0) of center pixels that camera does not see.

This module only marshals arguments: every step runs in the CUDA kernels of the in-tree library
_lib/libocc.so (built by build.py for sm_103a).  There is no CPU path; if the library cannot be loaded, every call
raises.  Device memory and streams come from PyTorch (torch.Tensor.data_ptr(), torch.cuda.Stream.cuda_stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

OCC_OK = 0
OCC_ERR_INVALID_ARG = 1
OCC_ERR_NONFINITE_INPUT = 2
OCC_ERR_CAPACITY = 3
OCC_ERR_TIMEOUT = 4
OCC_ERR_CUDA = 5
OCC_MAX_VIEWS = 64
OCC_MAX_SCAN = 4094
OCC_MAX_SIDE = 65535
OCC_MAX_N = 64

OCC_NUM_STAGES = 6
STAGES = ["candidates", "scan_lines", "scan_256", "scan_1024", "scan_4096", "mask"]

OCC_NOALLOC_MAX_PIXEL_VIEWS = 16777216
OCC_STRIP_PX_MAX = 16384
STRIP_PX_DEFAULT = 4096      # default occ_tuning.strip_px

OCC_MAX_FRAMES = 1024

EXPORTED = ["occ_default_params", "occ_direction", "occ_create", "occ_destroy", "occ_detect", "occ_detect_host",
            "occ_detect_host_async", "occ_detect_batched", "occ_get_status", "occ_get_stats", "occ_set_tuning", "occ_get_tuning", "occ_set_wait_limit",
            "occ_set_profiling", "occ_get_timings", "occ_detect_noalloc", "occ_fuse_median", "occ_warp_views",
            "occ_detect_batched_tiles", "occ_net_create", "occ_net_destroy", "occ_net_set_params",
            "occ_net_get_params", "occ_net_forward", "occ_net_loss_grad", "occ_net_adam", "occ_net_propose",
            "occ_net_status", "occ_net_conv3x3", "occ_net_conv3x3_wgrad", "occ_status_string"]

NET_PARAMS = 12817   # OCC_NET_PARAMS

TILE = 32   # OCC_TILE


class occ_view(ctypes.Structure):
    """Baseline angle alpha in degrees (x toward y, y pointing down) and baseline ratio r."""
    _fields_ = [("alpha_deg", ctypes.c_double), ("ratio", ctypes.c_float)]


class occ_params(ctypes.Structure):
    """gamma (Eq. 2), zeta and beta (Eq. 5), L (Eq. 3, <= 0 automatic), N (Eq. 5)."""
    _fields_ = [("gamma", ctypes.c_float), ("zeta", ctypes.c_float), ("beta", ctypes.c_float),
                ("L", ctypes.c_int32), ("N", ctypes.c_int32)]


class occ_view_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("samples", ctypes.c_int64), ("pair_tests", ctypes.c_int64),
                ("L", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"candidates": int(self.candidates), "samples": int(self.samples),
                "pair_tests": int(self.pair_tests), "L": int(self.L)}


class occ_tuning(ctypes.Structure):
    """Mapping of the scan work: line_max_runs (0, 1, 2), line_blocks_per_sm, warp_lines_per_block (4, 8), strip_px
    (0 = no strip kernel, else 1024 .. OCC_STRIP_PX_MAX pixels per strip, a multiple of 64), fused (1 = one launch
    for calls whose views all take the strip kernel, 0 = separate launches, the default)."""
    _fields_ = [("line_max_runs", ctypes.c_int32), ("line_blocks_per_sm", ctypes.c_int32),
                ("warp_lines_per_block", ctypes.c_int32), ("strip_px", ctypes.c_int32), ("fused", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class OccError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {occ_status_string(status)} ({status})")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libocc.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_2408_14050_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.occ_default_params.argtypes = [ctypes.POINTER(occ_params)]
        L.occ_default_params.restype = None
        L.occ_direction.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
        L.occ_direction.restype = None
        L.occ_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64, i32, i64]
        L.occ_create.restype = ctypes.c_int
        L.occ_destroy.argtypes = [vp]
        L.occ_destroy.restype = None
        L.occ_detect.argtypes = [vp, vp, i32, i32, i64, ctypes.POINTER(occ_view), i32, ctypes.POINTER(occ_params),
                                 vp, vp, vp, vp, vp]
        L.occ_detect.restype = ctypes.c_int
        L.occ_detect_host.argtypes = [vp, vp, i32, i32, ctypes.POINTER(occ_view), i32, ctypes.POINTER(occ_params),
                                      vp, vp, vp]
        L.occ_detect_host.restype = ctypes.c_int
        L.occ_detect_host_async.argtypes = L.occ_detect_host.argtypes
        L.occ_detect_host_async.restype = ctypes.c_int
        L.occ_detect_batched.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(occ_view), i32, ctypes.POINTER(occ_params),
                                         ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.occ_detect_batched.restype = ctypes.c_int
        L.occ_detect_batched_tiles.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                               ctypes.POINTER(occ_view), i32, ctypes.POINTER(occ_params),
                                               ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                               ctypes.POINTER(vp), vp]
        L.occ_detect_batched_tiles.restype = ctypes.c_int
        L.occ_get_status.argtypes = [vp, vp]
        L.occ_get_status.restype = ctypes.c_int
        L.occ_get_stats.argtypes = [vp, ctypes.POINTER(occ_view_stats), i32]
        L.occ_get_stats.restype = ctypes.c_int
        L.occ_set_tuning.argtypes = [vp, ctypes.POINTER(occ_tuning)]
        L.occ_set_tuning.restype = ctypes.c_int
        L.occ_get_tuning.argtypes = [vp, ctypes.POINTER(occ_tuning), ctypes.POINTER(i32)]
        L.occ_get_tuning.restype = ctypes.c_int
        L.occ_set_wait_limit.argtypes = [vp, i64, i32]
        L.occ_set_wait_limit.restype = ctypes.c_int
        L.occ_set_profiling.argtypes = [vp, ctypes.c_int]
        L.occ_set_profiling.restype = ctypes.c_int
        L.occ_get_timings.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
        L.occ_get_timings.restype = ctypes.c_int
        L.occ_detect_noalloc.argtypes = [vp, i32, i32, i64, ctypes.POINTER(occ_view), i32,
                                         ctypes.POINTER(occ_params), vp, vp, vp, vp]
        L.occ_detect_noalloc.restype = ctypes.c_int
        L.occ_fuse_median.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i64, vp, i64, vp, vp]
        L.occ_fuse_median.restype = ctypes.c_int
        L.occ_warp_views.argtypes = [vp, i32, i32, i64, ctypes.POINTER(occ_view), i32, ctypes.POINTER(vp), i64, vp,
                                     vp, vp]
        L.occ_warp_views.restype = ctypes.c_int
        L.occ_net_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64, i32]
        L.occ_net_create.restype = ctypes.c_int
        L.occ_net_destroy.argtypes = [vp]
        L.occ_net_destroy.restype = None
        fp = ctypes.POINTER(ctypes.c_float)
        L.occ_net_set_params.argtypes = [vp, fp, i64]
        L.occ_net_set_params.restype = ctypes.c_int
        L.occ_net_get_params.argtypes = [vp, fp, i64]
        L.occ_net_get_params.restype = ctypes.c_int
        L.occ_net_forward.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(occ_view), i32, vp, vp]
        L.occ_net_forward.restype = ctypes.c_int
        L.occ_net_loss_grad.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(occ_view), i32, vp, ctypes.c_float, vp,
                                        vp, vp, vp]
        L.occ_net_loss_grad.restype = ctypes.c_int
        L.occ_net_adam.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, vp]
        L.occ_net_adam.restype = ctypes.c_int
        L.occ_net_propose.argtypes = [vp, i64, ctypes.c_float, vp, vp]
        L.occ_net_propose.restype = ctypes.c_int
        L.occ_net_status.argtypes = [vp]
        L.occ_net_status.restype = ctypes.c_int
        L.occ_net_conv3x3.argtypes = [vp, i32, i32, i32, i32, vp, vp, i32, vp, i32, vp, vp]
        L.occ_net_conv3x3.restype = ctypes.c_int
        L.occ_net_conv3x3_wgrad.argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, vp]
        L.occ_net_conv3x3_wgrad.restype = ctypes.c_int
        L.occ_status_string.argtypes = [ctypes.c_int]
        L.occ_status_string.restype = ctypes.c_char_p
        _lib = L
        return L


def library_path() -> str:
    return _build.LIB_PATH


# ---------------------------------------------------------------------------------------------------------------
# Host-only helpers

def occ_default_params(**overrides) -> occ_params:
    p = occ_params()
    load().occ_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def occ_direction(alpha_deg: float):
    c, s = ctypes.c_float(), ctypes.c_float()
    load().occ_direction(float(alpha_deg), ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def occ_status_string(status: int) -> str:
    return load().occ_status_string(int(status)).decode()


def _views(views):
    arr = (occ_view * len(views))()
    for i, (a, r) in enumerate(views):
        arr[i].alpha_deg = float(a)
        arr[i].ratio = float(r)
    return arr


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_map(D):
    """D: float32 [H][W] with unit column stride."""
    import torch
    if not isinstance(D, torch.Tensor) or D.dtype != torch.float32 or D.dim() != 2 or D.stride(1) != 1:
        raise ValueError("D must be a float32 tensor [H][W] with unit column stride")


def _check_outputs(D, specs):
    """Every given (tensor, dtype, shape): that dtype and shape, contiguous; then D on the current CUDA device and
    every tensor on D's device.  The kernels write shape-many elements, so a smaller buffer would be written past
    its end.  Shapes and dtypes are checked before devices, so that these errors show without a GPU too."""
    import torch
    for t, dt, shape in specs:
        if t is None:
            continue
        if t.dtype != dt or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"output must be a contiguous {dt} tensor of shape {tuple(shape)}, "
                             f"got {t.dtype} {tuple(t.shape)}")
    if not D.is_cuda or D.device.index != torch.cuda.current_device():
        raise ValueError("D must be a CUDA tensor on the current device")
    for t, _, _ in specs:
        if t is not None and t.device != D.device:
            raise ValueError("outputs must be CUDA tensors on D's device")


# ---------------------------------------------------------------------------------------------------------------
# Context and calls

class Context:
    """Owns one occ_ctx (device scratch of one device)."""

    def __init__(self, handle, device, max_pixels, max_views):
        self.handle = handle
        self.device = device
        self.max_pixels = max_pixels
        self.max_views = max_views
        self.last_views = 0

    def close(self):
        if self.handle:
            load().occ_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def occ_create(device: int = 0, max_pixels: int = 1920 * 1080, max_views: int = 8, max_candidates: int = 0):
    h = ctypes.c_void_p()
    rc = load().occ_create(ctypes.byref(h), int(device), int(max_pixels), int(max_views), int(max_candidates))
    if rc != OCC_OK:
        raise OccError(rc, "occ_create")
    return Context(h, device, max_pixels, max_views)


def occ_destroy(ctx: Context):
    ctx.close()


def occ_detect(ctx: Context, D, views, params: occ_params | None = None, M=None, O=None, E=None, A=None,
               stream=None, want_O: bool = True):
    """Queue the method on device tensors.  D: float32 CUDA tensor [H][W] (row stride may exceed W).  Returns
    (M uint8 [V][H][W], O int32 [V][H][W] or None).  Output tensors are allocated when not given."""
    import torch
    _check_map(D)
    H, W = D.shape
    nv = len(views)
    if M is None:
        M = torch.empty((nv, H, W), dtype=torch.uint8, device=D.device)
    if O is None and want_O:
        O = torch.empty((nv, H, W), dtype=torch.int32, device=D.device)
    _check_outputs(D, ((M, torch.uint8, (nv, H, W)), (O, torch.int32, (nv, H, W)),
                       (E, torch.float32, (H, W)), (A, torch.float32, (H, W))))
    rc = load().occ_detect(ctx.handle, _ptr(D), H, W, D.stride(0), _views(views), nv,
                           ctypes.byref(params) if params is not None else None, _ptr(M), _ptr(O), _ptr(E), _ptr(A),
                           _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_detect")
    ctx.last_views = nv
    return M, O


def tiles_of(H: int, W: int):
    """(tiles_y, tiles_x) of a frame for occ_detect_batched_tiles."""
    return (H + TILE - 1) // TILE, (W + TILE - 1) // TILE


def occ_detect_batched(ctx: Context, Ds, views, params: occ_params | None = None, Ms=None, Os=None, stream=None,
                       proposals=None, hits=None):
    """Queue the method for a list of float32 CUDA maps [H][W] (contiguous) with the same views, as one batch.
    Returns (Ms, Os): lists of uint8 / int32 [V][H][W] tensors (allocated when not given).

    proposals: optional list of uint8 CUDA tensors [V][tiles_y][tiles_x] (0 = skip the tile's candidates);
    hits: optional list of uint8 CUDA tensors of the same shape that receive the per-tile hit flags.  With either,
    the call goes through occ_detect_batched_tiles."""
    import torch
    nf = len(Ds)
    nv = len(views)
    for D in Ds:
        if D.dtype != torch.float32 or D.dim() != 2 or not D.is_cuda or not D.is_contiguous():
            raise ValueError("every map must be a contiguous float32 CUDA tensor [H][W]")
    if Ms is None:
        Ms = [torch.empty((nv, *D.shape), dtype=torch.uint8, device=D.device) for D in Ds]
    if Os is None:
        Os = [torch.empty((nv, *D.shape), dtype=torch.int32, device=D.device) for D in Ds]
    vp = ctypes.c_void_p
    d_arr = (vp * nf)(*[D.data_ptr() for D in Ds])
    m_arr = (vp * nf)(*[M.data_ptr() for M in Ms])
    o_arr = (vp * nf)(*[O.data_ptr() for O in Os])
    h_arr = (ctypes.c_int32 * nf)(*[D.shape[0] for D in Ds])
    w_arr = (ctypes.c_int32 * nf)(*[D.shape[1] for D in Ds])
    pv = ctypes.byref(params) if params is not None else None
    if proposals is None and hits is None:
        rc = load().occ_detect_batched(ctx.handle, nf, d_arr, h_arr, w_arr, _views(views), nv, pv, m_arr, o_arr,
                                       _stream_handle(stream))
    else:
        def table(ts):
            if ts is None:
                return None
            for D, t in zip(Ds, ts):
                if t is not None and (t.shape != (nv, *tiles_of(*D.shape)) or t.dtype != torch.uint8
                                      or not t.is_contiguous()):
                    raise ValueError("tile tables must be contiguous uint8 [V][tiles_y][tiles_x]")
            return (vp * nf)(*[None if t is None else t.data_ptr() for t in ts])
        rc = load().occ_detect_batched_tiles(ctx.handle, nf, d_arr, h_arr, w_arr, _views(views), nv, pv,
                                             table(proposals), m_arr, o_arr, table(hits), _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_detect_batched")
    ctx.last_views = nv
    return Ms, Os


def occ_detect_host(ctx: Context, D, views, params: occ_params | None = None, M=None, O=None, stream=None,
                    wait: bool = True):
    """The method on host buffers (numpy or CPU tensors; pinned memory is fastest): copies in, runs, copies M (and O
    if given) back, and (wait) waits.  Returns (status code, M, O); with wait=False the code only says whether the work
    was queued, M and O are complete once the stream gets there, and occ_get_status gives the device status."""
    import numpy as np
    H, W = D.shape
    nv = len(views)
    if M is None:
        M = np.empty((nv, H, W), dtype=np.uint8)

    def addr(x):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):
            return ctypes.c_void_p(x.data_ptr())
        return ctypes.c_void_p(x.ctypes.data)

    fn = load().occ_detect_host if wait else load().occ_detect_host_async
    rc = fn(ctx.handle, addr(D), H, W, _views(views), nv, ctypes.byref(params) if params is not None else None,
            addr(M), addr(O), _stream_handle(stream))
    ctx.last_views = nv
    return rc, M, O


def occ_get_status(ctx: Context, stream=None) -> int:
    return int(load().occ_get_status(ctx.handle, _stream_handle(stream)))


def occ_get_stats(ctx: Context, n_views: int | None = None):
    n = ctx.last_views if n_views is None else n_views
    out = (occ_view_stats * max(n, 1))()
    rc = load().occ_get_stats(ctx.handle, out, n)
    if rc != OCC_OK:
        raise OccError(rc, "occ_get_stats")
    return [out[i].as_dict() for i in range(n)]


def occ_set_profiling(ctx: Context, enable: bool = True):
    rc = load().occ_set_profiling(ctx.handle, 1 if enable else 0)
    if rc != OCC_OK:
        raise OccError(rc, "occ_set_profiling")


def occ_get_timings(ctx: Context) -> dict:
    """Device milliseconds of each stage of the last profiled occ_detect call."""
    ms = (ctypes.c_float * OCC_NUM_STAGES)()
    rc = load().occ_get_timings(ctx.handle, ms, OCC_NUM_STAGES)
    if rc != OCC_OK:
        raise OccError(rc, "occ_get_timings")
    return {name: float(ms[i]) for i, name in enumerate(STAGES)}


def occ_detect_noalloc(D, views, params: occ_params | None = None, M=None, O=None, status=None, stream=None) -> int:
    """occ_detect on the current CUDA device without a context and without device allocation by the library (for
    callers that cannot allocate).  D, M [V][H][W] uint8, O [V][H][W] int32 and status (int32, 1 element, or None)
    are CUDA tensors owned by the caller.  Returns the host status code; the device status lands in `status`."""
    import torch
    if M is None or O is None:
        raise ValueError("M and O must be given: this entry point allocates nothing")
    _check_map(D)
    H, W = D.shape
    nv = len(views)
    if status is not None and (status.dtype != torch.int32 or status.numel() < 1):
        raise ValueError("status must be an int32 tensor of at least one element")
    _check_outputs(D, ((M, torch.uint8, (nv, H, W)), (O, torch.int32, (nv, H, W))))
    if status is not None and status.device != D.device:
        raise ValueError("status must be on D's device")
    return int(load().occ_detect_noalloc(_ptr(D), H, W, D.stride(0), _views(views), len(views),
                                         ctypes.byref(params) if params is not None else None, _ptr(M), _ptr(O),
                                         _ptr(status), _stream_handle(stream)))


def occ_fuse_median(maps, D=None, status=None, stream=None):
    """Pixel-wise median of the disparity maps (list of CUDA float32 [H][W] tensors, same shape and row stride) into
    D (a new tensor if None), on the maps' device.  status: optional CUDA int32 tensor of one element that receives
    0 or OCC_ERR_NONFINITE_INPUT in stream order.  Returns D."""
    import torch
    if not maps:
        raise ValueError("no maps")
    H, W = maps[0].shape
    for m in maps:
        if m.shape != (H, W) or m.dtype != torch.float32 or m.stride() != maps[0].stride() or m.stride(1) != 1:
            raise ValueError("maps must be float32 [H][W] with equal shape and row stride")
    if D is None:
        D = torch.empty((H, W), dtype=torch.float32, device=maps[0].device)
    arr = (ctypes.c_void_p * len(maps))(*[m.data_ptr() for m in maps])
    rc = load().occ_fuse_median(arr, len(maps), H, W, maps[0].stride(0), _ptr(D), D.stride(0), _ptr(status),
                                _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_fuse_median")
    return D


def occ_warp_views(D, views, images, M=None, out=None, stream=None):
    """Backward warp of the peripheral images (list of CUDA float32 [H][W], one per view, equal row stride) to the
    center view along each view's baseline, bilinear, with M [V][H][W] (uint8, or None) zeroing the occluded
    pixels.  Returns out [V][H][W] float32."""
    import torch
    H, W = D.shape
    V = len(views)
    if len(images) != V:
        raise ValueError("one image per view")
    for im in images:
        if im.shape != (H, W) or im.dtype != torch.float32 or im.stride() != images[0].stride() or im.stride(1) != 1:
            raise ValueError("images must be float32 [H][W] with equal row stride")
    if M is not None and (M.shape != (V, H, W) or M.dtype != torch.uint8 or not M.is_contiguous()):
        raise ValueError("M must be a contiguous uint8 [V][H][W] tensor")
    if out is None:
        out = torch.empty((V, H, W), dtype=torch.float32, device=D.device)
    elif out.shape != (V, H, W) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 [V][H][W] tensor")
    arr = (ctypes.c_void_p * V)(*[im.data_ptr() for im in images])
    rc = load().occ_warp_views(_ptr(D), H, W, D.stride(0), _views(views), V, arr, images[0].stride(0), _ptr(M),
                               _ptr(out), _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_warp_views")
    return out


def occ_set_tuning(ctx: Context, tuning: dict | None = None):
    """Apply a tuning (dict with the occ_tuning fields; None: defaults)."""
    t = None
    if tuning is not None:
        t = occ_tuning(int(tuning["line_max_runs"]), int(tuning["line_blocks_per_sm"]),
                       int(tuning["warp_lines_per_block"]), int(tuning.get("strip_px", STRIP_PX_DEFAULT)),
                       int(tuning.get("fused", 0)))
    rc = load().occ_set_tuning(ctx.handle, ctypes.byref(t) if t is not None else None)
    if rc != OCC_OK:
        raise OccError(rc, "occ_set_tuning")


def occ_set_wait_limit(ctx: Context, wait_us: int = 0, hold: bool = False):
    """Bound of the fused launch's waits in microseconds (0: 2 s); hold=True is the test hook that withholds the
    frames' plans so that the waits reach the bound (status OCC_ERR_TIMEOUT)."""
    rc = load().occ_set_wait_limit(ctx.handle, int(wait_us), 1 if hold else 0)
    if rc != OCC_OK:
        raise OccError(rc, "occ_set_wait_limit")


def occ_get_tuning(ctx: Context):
    """(tuning dict, occupancy limit of line_blocks_per_sm)."""
    t = occ_tuning()
    m = ctypes.c_int32()
    rc = load().occ_get_tuning(ctx.handle, ctypes.byref(t), ctypes.byref(m))
    if rc != OCC_OK:
        raise OccError(rc, "occ_get_tuning")
    return t.as_dict(), int(m.value)



# ---------------------------------------------------------------------------------------------------------------
# Learned tile proposer

class Net:
    """The learned tile proposer's network (occ_net): fp32 master parameters, Adam state and activation scratch for up
    to max_pixels pixels (n x H x W) per call, on one device."""

    def __init__(self, device: int = 0, max_pixels: int = 1 << 22, max_views: int = 8):
        h = ctypes.c_void_p()
        rc = load().occ_net_create(ctypes.byref(h), device, max_pixels, max_views)
        if rc != OCC_OK:
            raise OccError(rc, "occ_net_create")
        self.handle = h
        self.device = device
        self.max_pixels = max_pixels

    def close(self):
        if self.handle:
            load().occ_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != NET_PARAMS:
            raise ValueError("parameter count")
        rc = load().occ_net_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size)
        if rc != OCC_OK:
            raise OccError(rc, "occ_net_set_params")

    def get_params(self):
        import numpy as np
        p = np.empty(NET_PARAMS, dtype=np.float32)
        rc = load().occ_net_get_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size)
        if rc != OCC_OK:
            raise OccError(rc, "occ_net_get_params")
        return p

    @staticmethod
    def _frames(D):
        import torch
        if D.dim() == 2:
            D = D.unsqueeze(0)
        if D.dtype != torch.float32 or not D.is_cuda or not D.is_contiguous():
            raise ValueError("maps must be a contiguous float32 CUDA tensor [n][H][W]")
        return D

    def forward(self, D, views, logits=None, stream=None):
        """Tile logits [n][V][tiles_y][tiles_x] of the maps D ([n][H][W] or [H][W])."""
        import torch
        D = self._frames(D)
        n, H, W = D.shape
        ty, tx = tiles_of(H, W)
        if logits is None:
            logits = torch.empty((n, len(views), ty, tx), dtype=torch.float32, device=D.device)
        rc = load().occ_net_forward(self.handle, _ptr(D), n, H, W, _views(views), len(views), _ptr(logits),
                                    _stream_handle(stream))
        if rc != OCC_OK:
            raise OccError(rc, "occ_net_forward")
        return logits

    def loss_grad(self, D, views, labels, pos_weight: float = 1.0, grads=None, loss=None, logits=None, stream=None):
        """(loss [1], grads [NET_PARAMS]) device tensors for labelled maps."""
        import torch
        D = self._frames(D)
        n, H, W = D.shape
        if labels.dtype != torch.uint8 or not labels.is_contiguous() or \
                labels.shape != (n, len(views), *tiles_of(H, W)):
            raise ValueError("labels must be contiguous uint8 [n][V][tiles_y][tiles_x]")
        if grads is None:
            grads = torch.empty(NET_PARAMS, dtype=torch.float32, device=D.device)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=D.device)
        rc = load().occ_net_loss_grad(self.handle, _ptr(D), n, H, W, _views(views), len(views), _ptr(labels),
                                      float(pos_weight), _ptr(grads), _ptr(loss), _ptr(logits), _stream_handle(stream))
        if rc != OCC_OK:
            raise OccError(rc, "occ_net_loss_grad")
        return loss, grads

    def adam(self, grads, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             stream=None):
        rc = load().occ_net_adam(self.handle, _ptr(grads), lr, beta1, beta2, eps, step, _stream_handle(stream))
        if rc != OCC_OK:
            raise OccError(rc, "occ_net_adam")


def occ_net_propose(logits, threshold: float, proposal=None, stream=None):
    """uint8 proposal table: logits > threshold."""
    import torch
    if proposal is None:
        proposal = torch.empty(logits.shape, dtype=torch.uint8, device=logits.device)
    rc = load().occ_net_propose(_ptr(logits), logits.numel(), float(threshold), _ptr(proposal), _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_net_propose")
    return proposal


def occ_net_status(stream=None) -> int:
    return int(load().occ_net_status(_stream_handle(stream)))


def occ_net_conv3x3(X, Wb, bias=None, gate=None, relu: bool = False, Y=None, stream=None):
    """One network convolution layer on bf16 NHWC tensors X [n][H][W][c_in], Wb [c_out][K] (see include/occ.h)."""
    import torch
    n, H, W, ci = X.shape
    co = Wb.shape[0]
    if Y is None:
        Y = torch.empty((n, H, W, co), dtype=torch.bfloat16, device=X.device)
    rc = load().occ_net_conv3x3(_ptr(X), n, H, W, ci, _ptr(Wb), _ptr(bias), co, _ptr(gate), 1 if relu else 0, _ptr(Y),
                                _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_net_conv3x3")
    return Y


def occ_net_conv3x3_wgrad(X, dY, dWt=None, stream=None):
    """dWt [9 c_in + 1][c_out] (fp32, accumulated) of a network convolution layer."""
    import torch
    n, H, W, ci = X.shape
    co = dY.shape[-1]
    if dWt is None:
        dWt = torch.zeros((9 * ci + 1, co), dtype=torch.float32, device=X.device)
    rc = load().occ_net_conv3x3_wgrad(_ptr(X), _ptr(dY), n, H, W, ci, co, _ptr(dWt), _stream_handle(stream))
    if rc != OCC_OK:
        raise OccError(rc, "occ_net_conv3x3_wgrad")
    return dWt
