"""GB300-native generalised geodesic distance transform by raster-scan passes.

Thin Python binding over the C ABI of ``libfgx_gb300.so`` (``include/fgx.h``):
argument marshalling only.  Every step of the transform runs in the library's
CUDA kernels; PyTorch supplies device memory and the current stream.  There is
no CPU path: if the library is missing, every call raises.

Method (FastGeodis, Implementation section; generalised GDT of the Summary):
D0 = v*M, then 4 (2D) or 6 (3D) directional passes per iteration, each
updating a line from the already-updated previous line with cost
sqrt((1-lambda)*|x-y|^2_spacing + lambda*|I(x)-I(y)|^2).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfgx_gb300.so")

OK = 0
ERR_ARG = -1
ERR_NOT_DEVICE_PTR = -2
ERR_SHAPE = -3
ERR_WORKSPACE = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_DEVICE = -7
ERR_UNSUPPORTED = -8

_lock = threading.Lock()
_lib = None


class FgxError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class Options(ctypes.Structure):
    """fgx_options: optional tuning knobs (0 = automatic)."""
    _fields_ = [("size", ctypes.c_uint32), ("tile_lines", ctypes.c_int32),
                ("tile_width", ctypes.c_int32), ("tile_height", ctypes.c_int32),
                ("max_blocks", ctypes.c_int32), ("timeout_ms", ctypes.c_int32),
                ("segments", ctypes.c_int32), ("fast_math", ctypes.c_int32),
                ("no_cost_tables", ctypes.c_int32), ("split_sms", ctypes.c_int32)]

    def __init__(self, tile_lines=0, tile_width=0, tile_height=0, max_blocks=0, timeout_ms=0,
                 segments=0, fast_math=0, no_cost_tables=0, split_sms=0):
        super().__init__(ctypes.sizeof(Options), tile_lines, tile_width, tile_height, max_blocks,
                         timeout_ms, segments, fast_math, no_cost_tables, split_sms)


class Instance(ctypes.Structure):
    """fgx_instance: one entry of a batched call."""
    _fields_ = [("ndim", ctypes.c_int32), ("channels", ctypes.c_int32), ("D", ctypes.c_int64),
                ("H", ctypes.c_int64), ("W", ctypes.c_int64), ("image", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("dist", ctypes.c_void_p),
                ("spacing", ctypes.c_float * 3), ("v", ctypes.c_float),
                ("lambda_", ctypes.c_float), ("iterations", ctypes.c_int32)]


class BatchedPlanC(ctypes.Structure):
    """fgx_batched_plan: plain data describing a prepared batched launch."""
    _fields_ = [("size", ctypes.c_uint32), ("n", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("region", ctypes.c_int32), ("kmax", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("clear_bytes", ctypes.c_uint64),
                ("desc_off", ctypes.c_uint64), ("waves_off", ctypes.c_uint64),
                ("items_off", ctypes.c_uint64), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_uint64), ("n2d", ctypes.c_int32),
                ("grid2d", ctypes.c_int32), ("rounds2d", ctypes.c_int32),
                ("channels2d", ctypes.c_int32), ("max_wp2d", ctypes.c_int32),
                ("max_hp2d", ctypes.c_int32), ("desc2d_off", ctypes.c_uint64),
                ("waves2d_off", ctypes.c_uint64), ("items2d_off", ctypes.c_uint64),
                ("n3d", ctypes.c_int32), ("grid3d", ctypes.c_int32), ("rounds3d", ctypes.c_int32),
                ("smem3d", ctypes.c_int32), ("desc3d_off", ctypes.c_uint64),
                ("waves3d_off", ctypes.c_uint64), ("items3d_off", ctypes.c_uint64),
                ("tables3d", ctypes.c_int32), ("concurrent", ctypes.c_int32)]


_i64, _i32, _f32, _vp, _sz = (ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                              ctypes.c_size_t)
_SIGS = {
    "fgx_status_string": ([_i32], ctypes.c_char_p),
    "fgx_version": ([], _i32),
    "fgx_geodesic_workspace_size": ([_i32, _i64, _i64, _i64, _i64, _i64, _vp,
                                     ctypes.POINTER(_sz)], _i32),
    "fgx_geodesic2d": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _f32, _f32, _i32, _vp, _sz, _vp,
                        _vp], _i32),
    "fgx_geodesic3d": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32, _i32, _vp,
                        _sz, _vp, _vp], _i32),
    "fgx_workspace_status": ([_vp, _vp], _i32),
    "fgx_probe_wait_timeout": ([_vp, _sz, _i32, _vp], _i32),
    "fgx_autotune": ([_i32, _vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32, _i32,
                      _vp, _sz, _vp, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_f32), _vp],
                     _i32),
    "fgx_params_workspace_size": ([_i32, _i64, _i64, _i64, _i64, _i64, _i32, _vp,
                                   ctypes.POINTER(_sz)], _i32),
    "fgx_geodesic_bwd_params": ([_i32, _vp, _vp, _vp, _vp, _sz, _vp, _vp, _vp, _vp, _vp, _vp,
                                 _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32, _i32, _vp, _sz,
                                 _vp, _vp], _i32),
    "fgx_euclidean2d": ([_vp, _vp, _i64, _i64, _i64, _f32, _i32, _vp, _sz, _vp, _vp], _i32),
    "fgx_euclidean3d": ([_vp, _vp, _i64, _i64, _i64, _i64, _vp, _f32, _i32, _vp, _sz, _vp, _vp],
                        _i32),
    "fgx_signed_workspace_size": ([_i32, _i64, _i64, _i64, _i64, _i64, _vp,
                                   ctypes.POINTER(_sz)], _i32),
    "fgx_signed_geodesic2d": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _f32, _f32, _i32, _vp,
                               _sz, _vp, _vp], _i32),
    "fgx_signed_geodesic3d": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32,
                               _i32, _vp, _sz, _vp, _vp], _i32),
    "fgx_gsf_workspace_size": ([_i32, _i64, _i64, _i64, _i64, _i64, _vp, ctypes.POINTER(_sz)],
                               _i32),
    "fgx_gsf2d": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _f32, _f32, _i32, _f32, _f32, _vp, _sz,
                   _vp, _vp], _i32),
    "fgx_gsf3d": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32, _i32, _f32,
                   _f32, _vp, _sz, _vp, _vp], _i32),
    "fgx_batched_workspace_size": ([_vp, _i32, _vp, ctypes.POINTER(_sz)], _i32),
    "fgx_geodesic_batched": ([_vp, _i32, _vp, _sz, _vp, _vp], _i32),
    "fgx_batched_prepare": ([_vp, _i32, _vp, _sz, _vp, _vp, _vp], _i32),
    "fgx_batched_run": ([_vp, _vp], _i32),
    "fgx_batched_autotune": ([_vp, _i32, _vp, _sz, _vp, _i32, _i32, ctypes.POINTER(_i32),
                              ctypes.POINTER(_f32), _vp], _i32),
    "fgx_train_saved_size": ([_i32, _i64, _i64, _i64, _i64, _i32, ctypes.POINTER(_sz)], _i32),
    "fgx_geodesic2d_fwd_train": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _f32, _f32, _i32, _vp,
                                  _sz, _vp, _sz, _vp, _vp], _i32),
    "fgx_geodesic3d_fwd_train": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _f32, _f32,
                                  _i32, _vp, _sz, _vp, _sz, _vp, _vp], _i32),
    "fgx_backward_workspace_size": ([_i32, _i64, _i64, _i64, _i64, _i64, _i32, _vp,
                                     ctypes.POINTER(_sz)], _i32),
    "fgx_geodesic2d_bwd": ([_vp, _vp, _vp, _sz, _vp, _vp, _i64, _i64, _i64, _i64, _f32, _f32,
                            _i32, _vp, _sz, _vp, _vp], _i32),
    "fgx_geodesic3d_bwd": ([_vp, _vp, _vp, _sz, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp,
                            _f32, _f32, _i32, _vp, _sz, _vp, _vp], _i32),
    "fgx_checkpoint_saved_size": ([_i64, _i64, _i64, _i64, _i32, _i32, ctypes.POINTER(_sz)],
                                  _i32),
    "fgx_checkpoint_workspace_size": ([_i64, _i64, _i64, _i64, _i64, _i32, _i32, _vp,
                                       ctypes.POINTER(_sz)], _i32),
    "fgx_geodesic3d_fwd_checkpoint": ([_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _f32,
                                       _f32, _i32, _i32, _vp, _sz, _vp, _sz, _vp, _vp], _i32),
    "fgx_geodesic3d_bwd_checkpoint": ([_vp, _vp, _vp, _vp, _sz, _vp, _vp, _i64, _i64, _i64,
                                       _i64, _i64, _vp, _f32, _f32, _i32, _i32, _vp, _sz, _vp,
                                       _vp], _i32),
    "fgx_noalloc_status": ([_vp], _i32),
}


def lib():
    """Loads the CUDA library (built by ``build.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library not built: {LIB_PATH} is missing; run "
                    "paper_2208_00001_gb300.build.build() (there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().fgx_status_string(int(status)).decode()


def _check(st, where):
    if st != OK:
        raise FgxError(st, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _opt(options):
    if options is None:
        return None
    if isinstance(options, dict):
        options = Options(**options)
    return ctypes.byref(options)


def _check_tensor(t, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _shape(image, mask, ndim):
    _check_tensor(image, "image")
    _check_tensor(mask, "mask")
    if image.dim() != ndim + 2 or mask.dim() != ndim + 2:
        raise ValueError(f"expected {ndim + 2}-d image and mask")
    B, C = image.shape[:2]
    if mask.shape[0] != B or mask.shape[1] != 1 or mask.shape[2:] != image.shape[2:]:
        raise ValueError(f"mask shape {tuple(mask.shape)} does not match image "
                         f"{tuple(image.shape)}")
    if image.device != mask.device:
        raise ValueError("image and mask on different devices")
    spatial = tuple(image.shape[2:])
    if ndim == 2:
        return B, C, 1, spatial[0], spatial[1]
    return (B, C) + spatial


def workspace_size(ndim, B, C, D, H, W, options=None):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_geodesic_workspace_size(ndim, B, C, D, H, W, _opt(options),
                                             ctypes.byref(n)), "workspace size")
    return n.value


def workspace_status(ws):
    """Synchronises the current stream and returns the device status word."""
    return lib().fgx_workspace_status(_ptr(ws), _stream())


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# Tile geometries the 2D autotuner tries: (lines between ring refreshes,
# owned columns) with 4 * 32 = 128 region columns per tile; the first is the
# default.  Long single images favour long refresh blocks, many concurrent
# tiles (batches) shorter ones with wider owned parts.
TILE_CANDIDATES_2D = ((0, 0), (32, 64), (24, 80), (16, 96), (8, 112))
# 3D: ring widths of the plane-tile kernel (0: the planner's per-pass choice,
# 4: every pass narrow, 8: every pass wide where its tiles fit the grid).
RING_CANDIDATES_3D = (0, 4, 8)
# Batches of 2D and 3D instances: SM shares of the 2D launch tried beside the
# library's estimate (0) and one launch after the other (-1), as fractions of
# the SM count.
SPLIT_FRACTIONS = (0.2, 0.26, 0.32, 0.4)
_tuned = {}


def autotune(image, mask, v, lam, iterations, spacing=None, reps=3, candidates=None):
    """Times the tile geometries on these inputs (fgx_autotune) and returns
    the fastest as an options dict (None: the default), cached per shape,
    channel count, lambda = 0 or not and iterations: 2D the ring width and
    owned columns of the line tiles, 3D the ring width of the plane tiles."""
    ndim = image.dim() - 2
    B, C, D, H, W = _shape(image, mask, ndim)
    key = (ndim, B, C, D, H, W, float(lam) == 0.0, int(iterations), image.device.index)
    if key in _tuned:
        return _tuned[key]
    if ndim == 2:
        cands = candidates or TILE_CANDIDATES_2D
        opts = [Options(tile_lines=k, tile_width=t) for k, t in cands]
    else:
        cands = [(k, 0) for k in (candidates or RING_CANDIDATES_3D)]
        opts = [Options(tile_lines=k) for k, _ in cands]
    opts = (Options * len(cands))(*opts)
    dev = image.device
    with torch.cuda.device(dev):
        need = 0
        for o in opts:  # a candidate that cannot be planned is skipped by the tuner
            try:
                need = max(need, workspace_size(ndim, B, C, D, H, W, o))
            except FgxError:
                pass
        ws = _workspace(need, dev)
        out = torch.empty_like(mask)
        best = ctypes.c_int32(-1)
        ms = ctypes.c_float(0.0)
        _check(lib().fgx_autotune(ndim, _ptr(image), _ptr(mask), _ptr(out), B, C, D, H, W,
                                  _spacing(spacing) if ndim == 3 else None, float(v), float(lam),
                                  int(iterations), _ptr(ws), ws.numel(),
                                  ctypes.cast(opts, ctypes.c_void_p), len(cands), int(reps),
                                  ctypes.byref(best), ctypes.byref(ms), _stream()),
               "fgx_autotune")
    k, t = cands[best.value]
    if (k, t) == (0, 0):
        _tuned[key] = None
    else:
        _tuned[key] = dict(tile_lines=k, tile_width=t) if ndim == 2 else dict(tile_lines=k)
    return _tuned[key]


def _resolve(options, image, mask, v, lam, iterations, spacing=None):
    if isinstance(options, str):
        if options != "auto":
            raise ValueError(f"options: a dict, Options, None or 'auto', not {options!r}")
        return autotune(image, mask, v, lam, iterations, spacing)
    return options


def geodesic2d(image, mask, v, lam, iterations, out=None, options=None, workspace=None,
               check=False):
    """2D transform.  image (B,C,H,W), mask (B,1,H,W), float32 CUDA tensors.
    Returns dist (B,1,H,W).  check=True synchronises and raises on a device
    timeout.  options='auto' uses the autotuned tile geometry for this shape."""
    options = _resolve(options, image, mask, v, lam, iterations)
    B, C, D, H, W = _shape(image, mask, 2)
    dev = image.device
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty_like(mask)
        ws = workspace if workspace is not None else _workspace(
            workspace_size(2, B, C, 1, H, W, options), dev)
        _check(lib().fgx_geodesic2d(_ptr(image), _ptr(mask), _ptr(out), B, C, H, W, float(v),
                                    float(lam), int(iterations), _ptr(ws), ws.numel(),
                                    _opt(options), _stream()), "fgx_geodesic2d")
        if check:
            _check(workspace_status(ws), "fgx_geodesic2d (device)")
    return out


def _spacing(spacing):
    sp = (ctypes.c_float * 3)(*[float(s) for s in (spacing or (1.0, 1.0, 1.0))])
    return sp


def geodesic3d(image, mask, spacing, v, lam, iterations, out=None, options=None, workspace=None,
               check=False):
    """3D transform.  image (B,C,D,H,W), mask (B,1,D,H,W); spacing (sD,sH,sW)."""
    options = _resolve(options, image, mask, v, lam, iterations, spacing)
    B, C, D, H, W = _shape(image, mask, 3)
    dev = image.device
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty_like(mask)
        ws = workspace if workspace is not None else _workspace(
            workspace_size(3, B, C, D, H, W, options), dev)
        _check(lib().fgx_geodesic3d(_ptr(image), _ptr(mask), _ptr(out), B, C, D, H, W,
                                    _spacing(spacing), float(v), float(lam), int(iterations),
                                    _ptr(ws), ws.numel(), _opt(options), _stream()),
               "fgx_geodesic3d")
        if check:
            _check(workspace_status(ws), "fgx_geodesic3d (device)")
    return out


def backward_params(grad_dist, image, mask, saved, v, lam, iterations, spacing=None,
                    need_image=False, need_mask=False, options=None, check=False):
    """Gradients with respect to lambda and v through the saved codes:
    returns (grad_lambda, grad_v, lambda_terms, v_terms, grad_image,
    grad_mask).  The two scalars are float64 0-d tensors on the device (sums
    of the per-element float32 terms by a fixed tree); grad_image and
    grad_mask are None unless asked for."""
    ndim = image.dim() - 2
    B, C, D, H, W = _shape(image, mask, ndim)
    _check_tensor(grad_dist, "grad_dist")
    dev = image.device
    with torch.cuda.device(dev):
        n = ctypes.c_size_t(0)
        _check(lib().fgx_params_workspace_size(ndim, B, C, D, H, W, int(iterations),
                                               _opt(options), ctypes.byref(n)),
               "params workspace size")
        ws = _workspace(n.value, dev)
        lt = torch.empty_like(mask)
        vt = torch.empty_like(mask)
        sums = torch.zeros(2, dtype=torch.float64, device=dev)
        gi = torch.empty_like(image) if need_image else None
        gm = torch.empty_like(mask) if need_mask else None
        _check(lib().fgx_geodesic_bwd_params(
            ndim, _ptr(grad_dist), _ptr(image), _ptr(mask), _ptr(saved), saved.numel(),
            _ptr(gi) if gi is not None else None, _ptr(gm) if gm is not None else None,
            _ptr(lt), _ptr(vt), ctypes.c_void_p(sums.data_ptr()),
            ctypes.c_void_p(sums.data_ptr() + 8), B, C, D, H, W,
            _spacing(spacing) if ndim == 3 else None, float(v), float(lam), int(iterations),
            _ptr(ws), ws.numel(), _opt(options), _stream()), "fgx_geodesic_bwd_params")
        if check:
            _check(workspace_status(ws), "fgx_geodesic_bwd_params (device)")
    return sums[0], sums[1], lt, vt, gi, gm


def euclidean(mask, v, iterations, spacing=None, out=None, options=None, workspace=None,
              check=False):
    """Euclidean-only transform (lambda = 0, no image): mask (B,1,H,W) or
    (B,1,D,H,W); spacing (sD,sH,sW) in 3D."""
    _check_tensor(mask, "mask")
    ndim = mask.dim() - 2
    if ndim not in (2, 3) or mask.shape[1] != 1:
        raise ValueError("expected a (B,1,H,W) or (B,1,D,H,W) mask")
    B = mask.shape[0]
    D, H, W = (1,) + tuple(mask.shape[2:]) if ndim == 2 else tuple(mask.shape[2:])
    dev = mask.device
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty_like(mask)
        ws = workspace if workspace is not None else _workspace(
            workspace_size(ndim, B, 1, D, H, W, options), dev)
        if ndim == 2:
            st = lib().fgx_euclidean2d(_ptr(mask), _ptr(out), B, H, W, float(v), int(iterations),
                                       _ptr(ws), ws.numel(), _opt(options), _stream())
        else:
            st = lib().fgx_euclidean3d(_ptr(mask), _ptr(out), B, D, H, W, _spacing(spacing),
                                       float(v), int(iterations), _ptr(ws), ws.numel(),
                                       _opt(options), _stream())
        _check(st, "fgx_euclidean")
        if check:
            _check(workspace_status(ws), "fgx_euclidean (device)")
    return out


def signed_workspace_size(ndim, B, C, D, H, W, options=None):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_signed_workspace_size(ndim, B, C, D, H, W, _opt(options), ctypes.byref(n)),
           "signed workspace size")
    return n.value


def signed_geodesic(image, mask, v, lam, iterations, spacing=None, out=None, options=None,
                    workspace=None, check=False):
    """Signed transform GDT(mask) - GDT(1 - mask): negative inside the region
    mask = 0, positive where mask = 1.  2D or 3D by the image rank."""
    ndim = image.dim() - 2
    B, C, D, H, W = _shape(image, mask, ndim)
    dev = image.device
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty_like(mask)
        ws = workspace if workspace is not None else _workspace(
            signed_workspace_size(ndim, B, C, D, H, W, options), dev)
        if ndim == 2:
            st = lib().fgx_signed_geodesic2d(_ptr(image), _ptr(mask), _ptr(out), B, C, H, W,
                                             float(v), float(lam), int(iterations), _ptr(ws),
                                             ws.numel(), _opt(options), _stream())
        else:
            st = lib().fgx_signed_geodesic3d(_ptr(image), _ptr(mask), _ptr(out), B, C, D, H, W,
                                             _spacing(spacing), float(v), float(lam),
                                             int(iterations), _ptr(ws), ws.numel(),
                                             _opt(options), _stream())
        _check(st, "fgx_signed_geodesic")
        if check:
            _check(workspace_status(ws), "fgx_signed_geodesic (device)")
    return out


def gsf_workspace_size(ndim, B, C, D, H, W, options=None):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_gsf_workspace_size(ndim, B, C, D, H, W, _opt(options), ctypes.byref(n)),
           "gsf workspace size")
    return n.value


def gsf(image, indicator, v, lam, iterations, theta_d, theta_e, spacing=None, out=None,
        options=None, workspace=None, check=False):
    """Geodesic symmetric filtering of a segmentation indicator (1 = object):
    erosion by theta_e and dilation by theta_d in geodesic distance, combined
    symmetrically; returns 1.0 / 0.0 floats of the indicator's shape."""
    ndim = image.dim() - 2
    B, C, D, H, W = _shape(image, indicator, ndim)
    dev = image.device
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty_like(indicator)
        ws = workspace if workspace is not None else _workspace(
            gsf_workspace_size(ndim, B, C, D, H, W, options), dev)
        if ndim == 2:
            st = lib().fgx_gsf2d(_ptr(image), _ptr(indicator), _ptr(out), B, C, H, W, float(v),
                                 float(lam), int(iterations), float(theta_d), float(theta_e),
                                 _ptr(ws), ws.numel(), _opt(options), _stream())
        else:
            st = lib().fgx_gsf3d(_ptr(image), _ptr(indicator), _ptr(out), B, C, D, H, W,
                                 _spacing(spacing), float(v), float(lam), int(iterations),
                                 float(theta_d), float(theta_e), _ptr(ws), ws.numel(),
                                 _opt(options), _stream())
        _check(st, "fgx_gsf")
        if check:
            _check(workspace_status(ws), "fgx_gsf (device)")
    return out


def geodesic(image, mask, v, lam, iterations, spacing=None, **kw):
    """Dispatches on the image rank: (B,C,H,W) -> 2D, (B,C,D,H,W) -> 3D."""
    if image.dim() == 4:
        return geodesic2d(image, mask, v, lam, iterations, **kw)
    return geodesic3d(image, mask, spacing, v, lam, iterations, **kw)


def saved_size(ndim, B, D, H, W, iterations):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_train_saved_size(ndim, B, D, H, W, iterations, ctypes.byref(n)),
           "saved size")
    return n.value


def forward_train(image, mask, v, lam, iterations, spacing=None, options=None, check=False):
    """Forward that records parent codes.  Returns (dist, saved uint8 tensor
    [iterations*passes, B, D*H*W]).  options='auto': the autotuned geometry."""
    options = _resolve(options, image, mask, v, lam, iterations, spacing)
    ndim = image.dim() - 2
    B, C, D, H, W = _shape(image, mask, ndim)
    dev = image.device
    npass = 6 if ndim == 3 else 4
    with torch.cuda.device(dev):
        dist = torch.empty_like(mask)
        saved = torch.empty((iterations * npass, B, D * H * W), dtype=torch.uint8, device=dev)
        ws = _workspace(workspace_size(ndim, B, C, D, H, W, options), dev)
        if ndim == 2:
            st = lib().fgx_geodesic2d_fwd_train(_ptr(image), _ptr(mask), _ptr(dist), B, C, H, W,
                                                float(v), float(lam), int(iterations),
                                                _ptr(saved), saved.numel(), _ptr(ws), ws.numel(),
                                                _opt(options), _stream())
        else:
            st = lib().fgx_geodesic3d_fwd_train(_ptr(image), _ptr(mask), _ptr(dist), B, C, D, H,
                                                W, _spacing(spacing), float(v), float(lam),
                                                int(iterations), _ptr(saved), saved.numel(),
                                                _ptr(ws), ws.numel(), _opt(options), _stream())
        _check(st, "forward_train")
        if check:
            _check(workspace_status(ws), "forward_train (device)")
    return dist, saved


def workspace_timeline(ws):
    """Phase timestamps (ns, device globaltimer) recorded by the persistent
    kernels in the workspace header: [start of first barrier, after it, after
    each pass ...]; zeros where nothing was recorded."""
    torch.cuda.synchronize()
    hdr = ws[128:256].cpu().view(torch.int64)
    return [int(x) for x in hdr.tolist()]


def backward_workspace_size(ndim, B, C, D, H, W, iterations, options=None):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_backward_workspace_size(ndim, B, C, D, H, W, int(iterations), _opt(options),
                                             ctypes.byref(n)), "backward workspace size")
    return n.value


def backward(grad_dist, image, saved, v, lam, iterations, spacing=None, need_image=True,
             need_mask=True, options=None, check=False):
    """Reverse sweep through the codes recorded by :func:`forward_train`.
    Returns (grad_image or None, grad_mask or None)."""
    ndim = image.dim() - 2
    _check_tensor(grad_dist, "grad_dist")
    B, C, D, H, W = _shape(image, grad_dist, ndim)
    dev = image.device
    with torch.cuda.device(dev):
        gi = torch.empty_like(image) if need_image else None
        gm = torch.empty_like(grad_dist) if need_mask else None
        if gi is None and gm is None:
            return None, None
        ws = _workspace(backward_workspace_size(ndim, B, C, D, H, W, iterations, options), dev)
        if ndim == 2:
            st = lib().fgx_geodesic2d_bwd(_ptr(grad_dist), _ptr(image), _ptr(saved),
                                          saved.numel(), _ptr(gi), _ptr(gm), B, C, H, W,
                                          float(v), float(lam), int(iterations), _ptr(ws),
                                          ws.numel(), _opt(options), _stream())
        else:
            st = lib().fgx_geodesic3d_bwd(_ptr(grad_dist), _ptr(image), _ptr(saved),
                                          saved.numel(), _ptr(gi), _ptr(gm), B, C, D, H, W,
                                          _spacing(spacing), float(v), float(lam),
                                          int(iterations), _ptr(ws), ws.numel(), _opt(options),
                                          _stream())
        _check(st, "backward")
        if check:
            _check(workspace_status(ws), "backward (device)")
    return gi, gm


def checkpoint_saved_size(B, D, H, W, iterations, interval):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_checkpoint_saved_size(B, D, H, W, int(iterations), int(interval),
                                           ctypes.byref(n)), "checkpoint saved size")
    return n.value


def checkpoint_workspace_size(B, C, D, H, W, iterations, interval, options=None):
    n = ctypes.c_size_t(0)
    _check(lib().fgx_checkpoint_workspace_size(B, C, D, H, W, int(iterations), int(interval),
                                               _opt(options), ctypes.byref(n)),
           "checkpoint workspace size")
    return n.value


def forward_checkpoint(image, mask, v, lam, iterations, interval, spacing=None, options=None,
                       check=False):
    """3D forward that keeps the distance map at the start of every
    `interval`-th iteration instead of parent codes.  Returns (dist, saved
    float32 tensor [checkpoints, B, D*H*W], possibly empty)."""
    if image.dim() != 5:
        raise ValueError("checkpointed training is 3D: image (B, C, D, H, W)")
    B, C, D, H, W = _shape(image, mask, 3)
    dev = image.device
    with torch.cuda.device(dev):
        dist = torch.empty_like(mask)
        nbytes = checkpoint_saved_size(B, D, H, W, iterations, interval)
        saved = torch.empty((nbytes // 4 // max(B * D * H * W, 1), B, D * H * W),
                            dtype=torch.float32, device=dev)
        ws = _workspace(checkpoint_workspace_size(B, C, D, H, W, iterations, interval, options),
                        dev)
        st = lib().fgx_geodesic3d_fwd_checkpoint(
            _ptr(image), _ptr(mask), _ptr(dist), B, C, D, H, W, _spacing(spacing), float(v),
            float(lam), int(iterations), int(interval), _ptr(saved) if saved.numel() else None,
            saved.numel() * 4, _ptr(ws), ws.numel(), _opt(options), _stream())
        _check(st, "forward_checkpoint")
        if check:
            _check(workspace_status(ws), "forward_checkpoint (device)")
    return dist, saved


def backward_checkpoint(grad_dist, image, mask, saved, v, lam, iterations, interval,
                        spacing=None, need_image=True, need_mask=True, options=None,
                        check=False):
    """Reverse sweep through the checkpoints of :func:`forward_checkpoint`
    (each segment replayed once).  Returns (grad_image or None, grad_mask or
    None), equal bit for bit to :func:`backward`'s."""
    _check_tensor(grad_dist, "grad_dist")
    B, C, D, H, W = _shape(image, grad_dist, 3)
    dev = image.device
    with torch.cuda.device(dev):
        gi = torch.empty_like(image) if need_image else None
        gm = torch.empty_like(grad_dist) if need_mask else None
        if gi is None and gm is None:
            return None, None
        ws = _workspace(checkpoint_workspace_size(B, C, D, H, W, iterations, interval, options),
                        dev)
        st = lib().fgx_geodesic3d_bwd_checkpoint(
            _ptr(grad_dist), _ptr(image), _ptr(mask), _ptr(saved) if saved.numel() else None,
            saved.numel() * 4, _ptr(gi), _ptr(gm), B, C, D, H, W, _spacing(spacing), float(v),
            float(lam), int(iterations), int(interval), _ptr(ws), ws.numel(), _opt(options),
            _stream())
        _check(st, "backward_checkpoint")
        if check:
            _check(workspace_status(ws), "backward_checkpoint (device)")
    return gi, gm


class GeodesicFn(torch.autograd.Function):
    """Differentiable transform: the forward records argmin parent codes, the
    backward runs the reverse sweep through them (dL/dimage, dL/dmask, and
    dL/dv, dL/dlambda when v or lam is a tensor that requires grad).  3D with
    checkpoint=k: the forward keeps the distance map every k iterations
    instead of the codes and the backward replays each segment (image and
    mask gradients only)."""

    @staticmethod
    def forward(ctx, image, mask, v, lam, iterations, spacing=None, options=None,
                checkpoint=None):
        vf, lf = float(v), float(lam)
        if checkpoint:
            if any(torch.is_tensor(x) and x.requires_grad for x in (v, lam)):
                raise ValueError("checkpointed training gives image and mask gradients only")
            dist, saved = forward_checkpoint(image.detach().contiguous(),
                                             mask.detach().contiguous(), vf, lf, iterations,
                                             int(checkpoint), spacing=spacing, options=options)
        else:
            dist, saved = forward_train(image.detach().contiguous(), mask.detach().contiguous(),
                                        vf, lf, iterations, spacing=spacing, options=options)
        ctx.save_for_backward(image.detach(), mask.detach(), saved)
        ctx.params = (vf, lf, iterations, spacing, options, checkpoint)
        ctx.scalar_like = (v, lam)
        return dist

    @staticmethod
    def backward(ctx, grad_dist):
        image, mask, saved = ctx.saved_tensors
        v, lam, iterations, spacing, options, checkpoint = ctx.params
        need_i, need_m, need_v, need_l = ctx.needs_input_grad[:4]
        gv = gl = None
        if checkpoint:
            gi, gm = backward_checkpoint(grad_dist.contiguous(), image, mask, saved, v, lam,
                                         iterations, int(checkpoint), spacing=spacing,
                                         need_image=need_i, need_mask=need_m, options=options)
        elif need_v or need_l:
            dl, dv, _, _, gi, gm = backward_params(grad_dist.contiguous(), image, mask, saved, v,
                                                   lam, iterations, spacing=spacing,
                                                   need_image=need_i, need_mask=need_m,
                                                   options=options)
            tv, tl = ctx.scalar_like
            if need_v:
                gv = dv.to(tv.dtype).reshape(tv.shape)
            if need_l:
                gl = dl.to(tl.dtype).reshape(tl.shape)
        else:
            gi, gm = backward(grad_dist.contiguous(), image, saved, v, lam, iterations,
                              spacing=spacing, need_image=need_i, need_mask=need_m,
                              options=options)
        return gi, gm, gv, gl, None, None, None, None


def geodesic_autograd(image, mask, v, lam, iterations, spacing=None, options=None,
                      checkpoint=None):
    """Autograd entry point: dist = GeodesicFn(image, mask, ...); v and lam
    may be floats or 0-d tensors (then their gradients are returned too).
    checkpoint=k (3D): keep distance maps every k iterations instead of codes."""
    return GeodesicFn.apply(image, mask, v, lam, iterations, spacing, options, checkpoint)


class BatchedPlan:
    """A prepared batched launch over instances of uneven shapes (2D and 3D
    mixed).  ``instances`` is a list of (image, mask, v, lam, iterations,
    spacing) with image (1, C, ...) and mask (1, 1, ...) CUDA float32
    tensors.  :meth:`run` launches the persistent kernels (2D line chains and
    3D plane tiles side by side on disjoint SM shares; replayable, also
    inside a captured CUDA graph); results are in :attr:`outputs`."""

    def __init__(self, instances, options=None):
        self.instances = list(instances)
        if isinstance(options, str):
            if options != "auto":
                raise ValueError("options: a dict, Options, None or 'auto'")
            # the 2D line-tile geometry (the library keeps the plane tiles of
            # the 3D instances whatever 2D geometry the options carry); with
            # 2D and 3D instances jointly with the SM share of the 2D launch
            # running beside the 3D one, since the best geometry on a share
            # of the SMs need not be the best on all of them
            i2 = [inst for inst in self.instances if inst[0].dim() == 4]
            has3 = len(i2) < len(self.instances)
            options = {}
            geos = [dict(tile_lines=k, tile_width=t) if (k, t) != (0, 0) else {}
                    for k, t in TILE_CANDIDATES_2D]
            if i2 and has3:
                dev = self.instances[0][0].device
                sms = torch.cuda.get_device_properties(dev).multi_processor_count
                splits = [0, -1] + [max(1, round(f * sms)) for f in SPLIT_FRACTIONS]
                cands = [dict(geo, split_sms=x) for geo in geos for x in splits]
                options = cands[self._tune(self.instances, cands)]
            elif i2:
                options = geos[self._tune(i2, geos)]
            options = options or None
        self.options = options
        self.outputs = []
        arr = (Instance * max(1, len(self.instances)))()
        dev = None
        for i, (img, m, v, lam, its, sp) in enumerate(self.instances):
            ndim = img.dim() - 2
            B, C, D, H, W = _shape(img, m, ndim)
            if B != 1:
                raise ValueError("batched instances have B = 1")
            out = torch.empty_like(m)
            self.outputs.append(out)
            dev = img.device
            sp3 = (1.0, 1.0, 1.0) if ndim == 2 else tuple(float(x) for x in sp)
            arr[i] = Instance(ndim, C, D, H, W, img.data_ptr(), m.data_ptr(), out.data_ptr(),
                              (ctypes.c_float * 3)(*sp3), float(v), float(lam), int(its))
        self._arr = arr
        self._opt = options if not isinstance(options, dict) else Options(**options)
        n = ctypes.c_size_t(0)
        _check(lib().fgx_batched_workspace_size(ctypes.byref(arr), len(self.instances),
                                                _opt(self._opt), ctypes.byref(n)),
               "batched workspace size")
        dev = dev or torch.device("cuda")
        self.workspace = _workspace(n.value, dev)
        self.plan = BatchedPlanC()
        with torch.cuda.device(dev):
            _check(lib().fgx_batched_prepare(ctypes.byref(arr), len(self.instances),
                                             _ptr(self.workspace), self.workspace.numel(),
                                             _opt(self._opt), ctypes.byref(self.plan), _stream()),
                   "fgx_batched_prepare")
        self.device = dev

    @staticmethod
    def _tune(instances, cands, reps=2):
        """Index of the fastest option set of `cands` (dicts) for this batch
        (fgx_batched_autotune)."""
        opts = (Options * len(cands))(*[Options(**c) for c in cands])
        arr = (Instance * max(1, len(instances)))()
        outs = []
        dev = None
        for i, (img, m, v, lam, its, sp) in enumerate(instances):
            ndim = img.dim() - 2
            B, C, D, H, W = _shape(img, m, ndim)
            out = torch.empty_like(m)
            outs.append(out)
            dev = img.device
            sp3 = (1.0, 1.0, 1.0) if ndim == 2 else tuple(float(x) for x in sp)
            arr[i] = Instance(ndim, C, D, H, W, img.data_ptr(), m.data_ptr(), out.data_ptr(),
                              (ctypes.c_float * 3)(*sp3), float(v), float(lam), int(its))
        need = 0
        for o in opts:
            n = ctypes.c_size_t(0)
            if lib().fgx_batched_workspace_size(ctypes.byref(arr), len(instances), ctypes.byref(o),
                                                ctypes.byref(n)) == OK:
                need = max(need, n.value)
        dev = dev or torch.device("cuda")
        ws = _workspace(need, dev)
        best = ctypes.c_int32(-1)
        ms = ctypes.c_float(0.0)
        with torch.cuda.device(dev):
            _check(lib().fgx_batched_autotune(ctypes.byref(arr), len(instances), _ptr(ws),
                                              ws.numel(), ctypes.cast(opts, ctypes.c_void_p),
                                              len(cands), int(reps), ctypes.byref(best),
                                              ctypes.byref(ms), _stream()),
                   "fgx_batched_autotune")
        return best.value

    def status(self):
        """Synchronises and returns the device status of the last run."""
        return workspace_status(self.workspace)

    def run(self, check=False):
        with torch.cuda.device(self.device):
            _check(lib().fgx_batched_run(ctypes.byref(self.plan), _stream()), "fgx_batched_run")
            if check:
                _check(workspace_status(self.workspace), "fgx_batched_run (device)")
        return self.outputs


def geodesic_batched(instances, options=None, check=False):
    """Prepares and runs one batched plan over all instances; returns their
    distance maps."""
    plan = BatchedPlan(instances, options)
    return plan.run(check=check)
