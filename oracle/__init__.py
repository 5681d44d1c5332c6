"""Oracle for the generalised geodesic distance transform (raster-scan passes).

TEST INFRASTRUCTURE ONLY.  Plain, slow, sequential CPU code (``gdt_oracle.c``)
that restates the method of FastGeodis (Implementation section: four passes in
2D, six in 3D, each line updated from the already-updated previous line; the
generalised GDT with soft seeds D0 = v*M and the geodesic/Euclidean mixture of
the Summary).  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this package.  It shares no code with the CUDA
library and never imports it.

Functions here are ctypes wrappers taking and returning numpy arrays:

* :func:`gdt` - forward transform in float32 (the bit-exact reference for the
  CUDA path) or float64, optionally recording parent codes.
* :func:`gdt_schedule` - float64 forward with any pass schedule, optionally
  iterated to its fixed point.
* :func:`backward` - reverse sweep through recorded codes (dL/dI, dL/dM).
* :func:`param_terms` / :func:`param_grads` - the gradients with respect to
  lambda and v through recorded codes.
* :func:`euclidean` - the transform at lambda = 0 (no image term).
* :func:`signed_gdt` - signed transform GDT(M) - GDT(1 - M) (the paper names
  signed geodesic distance among the applications without defining it; this
  is the reading the library implements).
* :func:`gsf` - geodesic symmetric filtering of a segmentation indicator (the
  paper names GSF among the applications without defining it; the reading
  composes signed transforms into an erosion, a dilation and their
  symmetric combination).

Parity status: forward pinned (Dijkstra at the fixed point, chamfer and
total-variation closed forms, 1D brute force, invariants); backward pinned by
float64 central differences; the signed transform pinned by its half-plane
closed form and its antisymmetry; GSF pinned by half-plane preservation, the
removal of objects thinner than the erosion and of holes narrower than the
dilation, the identity at zero thresholds and its exact complement symmetry.
The paper itself prints no numeric example, so no value of the paper's own is
pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gdt_oracle.c")
_INC = os.path.join(_HERE, "gdt_core.inc")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_gdt.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
          "-shared"]

PASSES_2D = ((1, +1), (1, -1), (2, +1), (2, -1))            # TB BT LR RL
PASSES_3D = ((0, +1), (0, -1), (1, +1), (1, -1), (2, +1), (2, -1))  # FB BF TB BT LR RL


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_INC))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32 = ctypes.c_int64, ctypes.c_int
            vp = ctypes.c_void_p
            lib.oracle_gdt_f32.argtypes = [vp, vp, vp, i32, i64, i64, i64, i64, i64, vp,
                                           ctypes.c_float, ctypes.c_float, i32, vp, i32]
            lib.oracle_gdt_f64.argtypes = [vp, vp, vp, i32, i64, i64, i64, i64, i64, vp,
                                           ctypes.c_double, ctypes.c_double, i32, vp]
            lib.oracle_gdt_sched_f64.argtypes = [vp, vp, vp, i32, i64, i64, i64, i64, i64, vp,
                                                 ctypes.c_double, ctypes.c_double, vp, i32, i32,
                                                 vp]
            lib.oracle_backward_f32.argtypes = [vp, vp, vp, vp, vp, i32, i64, i64, i64, i64, i64,
                                                vp, ctypes.c_float, ctypes.c_float, i32, vp, vp,
                                                vp]
            lib.oracle_backward_f64.argtypes = [vp, vp, vp, vp, vp, i32, i64, i64, i64, i64, i64,
                                                vp, ctypes.c_double, ctypes.c_double, i32, vp, vp,
                                                vp]
            for f in (lib.oracle_gdt_f32, lib.oracle_gdt_f64, lib.oracle_gdt_sched_f64,
                      lib.oracle_backward_f32, lib.oracle_backward_f64):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _shape(image, mask):
    """Returns (ndim, B, C, D, H, W) for image (B,C,H,W)/(B,C,D,H,W) and mask
    (B,1,...)."""
    if image.ndim == 4:
        B, C, H, W = image.shape
        if mask.shape != (B, 1, H, W):
            raise ValueError(f"mask shape {mask.shape} != {(B, 1, H, W)}")
        return 2, B, C, 1, H, W
    if image.ndim == 5:
        B, C, D, H, W = image.shape
        if mask.shape != (B, 1, D, H, W):
            raise ValueError(f"mask shape {mask.shape} != {(B, 1, D, H, W)}")
        return 3, B, C, D, H, W
    raise ValueError("image must be (B,C,H,W) or (B,C,D,H,W)")


def num_passes(ndim: int) -> int:
    return 6 if ndim == 3 else 4


def gdt(image, mask, v, lam, iterations, spacing=None, dtype=np.float32,
        return_codes=False, threads=1):
    """Forward transform.  Returns dist shaped like mask (and the codes array
    [iterations*passes, B, D*H*W] uint8 if return_codes)."""
    lib = _load()
    dt = np.dtype(dtype)
    image = np.ascontiguousarray(image, dtype=dt)
    mask = np.ascontiguousarray(mask, dtype=dt)
    ndim, B, C, D, H, W = _shape(image, mask)
    if spacing is None:
        spacing = (1.0, 1.0, 1.0)
    elif ndim == 2:
        spacing = (1.0, *spacing)
    sp = np.ascontiguousarray(spacing, dtype=dt)
    dist = np.empty_like(mask)
    codes = None
    if return_codes:
        codes = np.zeros((iterations * num_passes(ndim), B, D * H * W), dtype=np.uint8)
    if dt == np.float32:
        r = lib.oracle_gdt_f32(_ptr(image), _ptr(mask), _ptr(dist), ndim, B, C, D, H, W, _ptr(sp),
                               float(np.float32(v)), float(np.float32(lam)), int(iterations),
                               _ptr(codes), int(threads))
    elif dt == np.float64:
        r = lib.oracle_gdt_f64(_ptr(image), _ptr(mask), _ptr(dist), ndim, B, C, D, H, W, _ptr(sp),
                               float(v), float(lam), int(iterations), _ptr(codes))
    else:
        raise TypeError(dtype)
    if r != 0:
        raise ValueError(f"oracle_gdt failed ({r})")
    return (dist, codes) if return_codes else dist


def gdt_schedule(image, mask, v, lam, schedule, iterations=-1, spacing=None):
    """float64 forward with a given list of (axis, direction) passes.  With
    iterations < 0 it runs to the fixed point.  Returns (dist, iterations_run)."""
    lib = _load()
    image = np.ascontiguousarray(image, dtype=np.float64)
    mask = np.ascontiguousarray(mask, dtype=np.float64)
    ndim, B, C, D, H, W = _shape(image, mask)
    if spacing is None:
        spacing = (1.0, 1.0, 1.0)
    elif ndim == 2:
        spacing = (1.0, *spacing)
    sp = np.ascontiguousarray(spacing, dtype=np.float64)
    sched = np.ascontiguousarray(np.array(schedule, dtype=np.int32).reshape(-1))
    dist = np.empty_like(mask)
    its = ctypes.c_int(0)
    r = lib.oracle_gdt_sched_f64(_ptr(image), _ptr(mask), _ptr(dist), ndim, B, C, D, H, W,
                                 _ptr(sp), float(v), float(lam), _ptr(sched), len(schedule),
                                 int(iterations), ctypes.byref(its))
    if r != 0:
        raise ValueError(f"oracle_gdt_sched failed ({r})")
    return dist, its.value


def fixed_point(image, mask, v, lam, spacing=None):
    """float64 passes (paper order) repeated until nothing changes."""
    ndim = 3 if np.ndim(image) == 5 else 2
    return gdt_schedule(image, mask, v, lam, PASSES_3D if ndim == 3 else PASSES_2D, -1,
                        spacing)


def backward(grad_dist, image, codes, v, lam, iterations, spacing=None, dtype=np.float32,
             need_image=True, need_mask=True):
    """Reverse sweep through codes recorded by :func:`gdt`.  Returns
    (grad_image or None, grad_mask or None)."""
    lib = _load()
    dt = np.dtype(dtype)
    image = np.ascontiguousarray(image, dtype=dt)
    grad_dist = np.ascontiguousarray(grad_dist, dtype=dt)
    ndim, B, C, D, H, W = _shape(image, grad_dist)
    if spacing is None:
        spacing = (1.0, 1.0, 1.0)
    elif ndim == 2:
        spacing = (1.0, *spacing)
    sp = np.ascontiguousarray(spacing, dtype=dt)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    if codes.shape != (iterations * num_passes(ndim), B, D * H * W):
        raise ValueError("codes shape mismatch")
    gi = np.empty_like(image) if need_image else None
    gm = np.empty_like(grad_dist) if need_mask else None
    f = lib.oracle_backward_f32 if dt == np.float32 else lib.oracle_backward_f64
    r = f(_ptr(grad_dist), _ptr(image), _ptr(codes), _ptr(gi), _ptr(gm), ndim, B, C, D, H, W,
          _ptr(sp), dt.type(v).item(), dt.type(lam).item(), int(iterations), None, None, None)
    if r != 0:
        raise ValueError(f"oracle_backward failed ({r})")
    return gi, gm


def param_terms(grad_dist, image, mask, codes, v, lam, iterations, spacing=None,
                dtype=np.float32):
    """Per-element terms of the parameter gradients through recorded codes:
    (lambda_terms, v_terms), each shaped like mask.  lambda_terms holds, per
    element and over the pass applications in reverse order, the element's
    adjoint times d c / d lambda = (di2 - s2) / (2c) of its own parent edge
    (c^2 = (1 - lambda) s2 + lambda di2; 0 where c = 0); v_terms = M * G0 with
    G0 the adjoint of D0 = v M.  dL/dlambda and dL/dv are their sums
    (:func:`param_grads`)."""
    lib = _load()
    dt = np.dtype(dtype)
    image = np.ascontiguousarray(image, dtype=dt)
    grad_dist = np.ascontiguousarray(grad_dist, dtype=dt)
    mask = np.ascontiguousarray(mask, dtype=dt)
    ndim, B, C, D, H, W = _shape(image, grad_dist)
    if spacing is None:
        spacing = (1.0, 1.0, 1.0)
    elif ndim == 2:
        spacing = (1.0, *spacing)
    sp = np.ascontiguousarray(spacing, dtype=dt)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    if codes.shape != (iterations * num_passes(ndim), B, D * H * W):
        raise ValueError("codes shape mismatch")
    lt = np.empty_like(grad_dist)
    vt = np.empty_like(grad_dist)
    f = lib.oracle_backward_f32 if dt == np.float32 else lib.oracle_backward_f64
    r = f(_ptr(grad_dist), _ptr(image), _ptr(codes), None, None, ndim, B, C, D, H, W,
          _ptr(sp), dt.type(v).item(), dt.type(lam).item(), int(iterations), _ptr(mask),
          _ptr(lt), _ptr(vt))
    if r != 0:
        raise ValueError(f"oracle_backward failed ({r})")
    return lt, vt


def param_grads(grad_dist, image, mask, codes, v, lam, iterations, spacing=None):
    """(dL/dlambda, dL/dv): the float32 per-element terms of
    :func:`param_terms` summed in float64 (numpy's pairwise order)."""
    lt, vt = param_terms(grad_dist, image, mask, codes, v, lam, iterations, spacing)
    return (float(np.sum(lt.astype(np.float64).ravel(), dtype=np.float64)),
            float(np.sum(vt.astype(np.float64).ravel(), dtype=np.float64)))


def euclidean(mask, v, iterations, spacing=None, threads=1):
    """The transform at lambda = 0: every step costs its spacing-weighted
    length; the image term has no weight, so a zero image stands in."""
    mask = np.ascontiguousarray(mask, np.float32)
    image = np.zeros(mask.shape, np.float32)
    return gdt(image, mask, v, 0.0, iterations, spacing=spacing, threads=threads)


def signed_gdt(image, mask, v, lam, iterations, spacing=None, threads=1):
    """Signed transform GDT(M) - GDT(1 - M) in float32: the transform seeded
    by the region M = 0 minus the one seeded by M = 1, so negative inside the
    region M = 0 and positive where M = 1.  The complement and the difference
    are rounded to float32."""
    m = np.ascontiguousarray(mask, np.float32)
    comp = (np.float32(1.0) - m).astype(np.float32)
    a = gdt(image, m, v, lam, iterations, spacing=spacing, threads=threads)
    b = gdt(image, comp, v, lam, iterations, spacing=spacing, threads=threads)
    return (a - b).astype(np.float32)


def gsf(image, indicator, v, lam, iterations, theta_d, theta_e, spacing=None, threads=1):
    """Geodesic symmetric filtering in float32 of an indicator F in [0, 1]
    (1 = object).  With S(X) = GDT(1 - X) - GDT(X) the signed distance of the
    object of X (negative inside; ``signed_gdt`` of the mask 1 - X):
    erosion F_e = [S(F) < -theta_e], dilation F_d = [S(F) < theta_d], and the
    result [(S(F_e) + S(F_d)) + (theta_d - theta_e) < 0] as 1.0 / 0.0, every
    complement, difference and sum rounded to float32."""
    f = np.ascontiguousarray(indicator, np.float32)
    td, te = np.float32(theta_d), np.float32(theta_e)

    def signed_of_object(x):
        comp = (np.float32(1.0) - x).astype(np.float32)
        return signed_gdt(image, comp, v, lam, iterations, spacing=spacing, threads=threads)

    s = signed_of_object(f)
    f_e = (s < -te).astype(np.float32)
    f_d = (s < td).astype(np.float32)
    total = (signed_of_object(f_e) + signed_of_object(f_d)).astype(np.float32)
    c = np.float32(td - te)
    return ((total + c).astype(np.float32) < 0).astype(np.float32)
