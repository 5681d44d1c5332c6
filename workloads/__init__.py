"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and shapes only; it holds none of the
transform's arithmetic.  Every input is float32, contiguous, and generated with
numpy's PCG64 ``default_rng(seed)``; blurs use
``scipy.ndimage.gaussian_filter(sigma, mode='reflect', truncate=4.0)``.

The paper measures on unspecified "3D volume data" and on "common 2D/3D data
input sizes" kept in its documentation (Summary; Implementation).  Neither is
available, so these generators stand in for them with the shapes and value
structure below (smooth noise, sharp-edged objects, small seed regions):

* ``plain2d``   1x1x256x256, blurred U[0,1] noise, one 5x5 zero seed block.
* ``large2d``   1x3x2048x2048, per-channel blurred noise + 8 constant
  rectangles (sides 128..512), mask = 1 except 3 disks of radius 4.
* ``volume3d``  1x1x128x256x256, blurred U[-1000,1000] + 5 constant
  ellipsoids (semi-axes 8..48), one 3x3x3 seed block.
* ``batched``   64 2D (sides 128..1024) + 16 3D (sides 64..192) instances,
  1-3 seed blocks each, lambda ~ U[0,1].
* ``diff2d`` / ``diff3d``  soft masks in [0,1] with zero seed blocks and a
  loss weight w ~ U[0,1].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _blur(x, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(x, sigma=sigma, mode="reflect", truncate=4.0)


def blurred_noise(rng, shape, lo=0.0, hi=1.0, sigma=3.0):
    """Uniform noise on [lo, hi) smoothed by a Gaussian of `sigma` px."""
    x = rng.uniform(lo, hi, size=shape)
    return _blur(x, sigma).astype(np.float32)


def seed_block_mask(rng, spatial, block, count=1):
    """Mask of ones with `count` zero cubes of side `block` at uniform spots."""
    m = np.ones(spatial, dtype=np.float32)
    for _ in range(count):
        sl = []
        for n in spatial:
            b = min(block, n)
            o = int(rng.integers(0, n - b + 1))
            sl.append(slice(o, o + b))
        m[tuple(sl)] = 0.0
    return m


@dataclass
class Case:
    """One instance of the transform: inputs and parameters."""
    name: str
    image: np.ndarray            # (B,C,H,W) or (B,C,D,H,W) float32
    mask: np.ndarray             # (B,1,...) float32
    v: float
    lam: float
    iterations: int
    spacing: tuple | None = None  # (sD,sH,sW) in 3D; None = unit
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return self.image.ndim - 2

    @property
    def voxels(self):
        return int(np.prod(self.mask.shape))


def plain2d(seed=0, lam=1.0, iterations=2, size=256):
    rng = np.random.default_rng(seed)
    img = blurred_noise(rng, (size, size))
    m = seed_block_mask(rng, (size, size), 5)
    return Case("2D plain", img[None, None], m[None, None], 1e10, lam, iterations)


def large2d(seed=1, lam=0.5, iterations=2, size=2048, channels=3):
    rng = np.random.default_rng(seed)
    img = np.stack([blurred_noise(rng, (size, size)) for _ in range(channels)])
    for _ in range(8):
        hs, ws = (int(rng.integers(128, 513)) for _ in range(2))
        hs, ws = min(hs, size), min(ws, size)
        h0 = int(rng.integers(0, size - hs + 1))
        w0 = int(rng.integers(0, size - ws + 1))
        img[:, h0:h0 + hs, w0:w0 + ws] = rng.uniform(0, 1, size=(channels, 1, 1))
    m = np.ones((size, size), dtype=np.float32)
    yy, xx = np.mgrid[0:size, 0:size]
    for _ in range(3):
        cy, cx = (int(rng.integers(0, size)) for _ in range(2))
        m[(yy - cy) ** 2 + (xx - cx) ** 2 <= 16] = 0.0
    return Case("2D large", img[None].astype(np.float32), m[None, None], 1e10, lam, iterations)


def _ellipsoids(rng, vol, count, lo, hi):
    D, H, W = vol.shape
    zz, yy, xx = np.ogrid[0:D, 0:H, 0:W]
    for _ in range(count):
        c = [rng.uniform(0, n) for n in (D, H, W)]
        r = rng.uniform(8, 48, size=3)
        val = rng.uniform(lo, hi)
        inside = (((zz - c[0]) / r[0]) ** 2 + ((yy - c[1]) / r[1]) ** 2
                  + ((xx - c[2]) / r[2]) ** 2) <= 1.0
        vol[inside] = val
    return vol


def volume3d(seed=2, lam=1.0, iterations=4, shape=(128, 256, 256), spacing=(2.5, 1.0, 1.0)):
    rng = np.random.default_rng(seed)
    vol = blurred_noise(rng, shape, -1000.0, 1000.0)
    vol = _ellipsoids(rng, vol, 5, -1000.0, 1000.0).astype(np.float32)
    m = seed_block_mask(rng, shape, 3)
    return Case("3D volume", vol[None, None], m[None, None], 1e10, lam, iterations,
                tuple(spacing))


def batched(seed=3, n2d=64, n3d=16, side2d=(128, 1024), side3d=(64, 192), iterations=2):
    """Uneven instances; each is a Case with B = 1, C = 1, unit spacing."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n2d):
        H, W = (int(rng.integers(side2d[0], side2d[1] + 1)) for _ in range(2))
        img = blurred_noise(rng, (H, W))
        m = seed_block_mask(rng, (H, W), 3, count=int(rng.integers(1, 4)))
        out.append(Case(f"batched 2D #{i}", img[None, None], m[None, None], 1e10,
                        float(np.float32(rng.uniform(0, 1))), iterations))
    for i in range(n3d):
        shp = tuple(int(rng.integers(side3d[0], side3d[1] + 1)) for _ in range(3))
        vol = blurred_noise(rng, shp)
        m = seed_block_mask(rng, shp, 3, count=int(rng.integers(1, 4)))
        out.append(Case(f"batched 3D #{i}", vol[None, None], m[None, None], 1e10,
                        float(np.float32(rng.uniform(0, 1))), iterations, (1.0, 1.0, 1.0)))
    return out


def _soft_mask(rng, spatial, block, count):
    m = rng.uniform(0, 1, size=spatial).astype(np.float32)
    hard = seed_block_mask(rng, spatial, block, count)
    m[hard == 0] = 0.0
    return m


def diff2d(seed=4, batch=8, size=512, lam=0.75, iterations=2, v=1e10):
    rng = np.random.default_rng(seed)
    img = np.stack([blurred_noise(rng, (size, size)) for _ in range(batch)])[:, None]
    m = np.stack([_soft_mask(rng, (size, size), 5, 1) for _ in range(batch)])[:, None]
    w = rng.uniform(0, 1, size=m.shape).astype(np.float32)
    return Case("differentiable 2D", img, m, v, lam, iterations, extra={"w": w})


def diff3d(seed=4, shape=(96, 160, 160), lam=0.75, iterations=2, v=1e10):
    rng = np.random.default_rng(seed + 1000)
    vol = blurred_noise(rng, shape)
    m = _soft_mask(rng, shape, 3, 1)
    w = rng.uniform(0, 1, size=(1, 1) + tuple(shape)).astype(np.float32)
    return Case("differentiable 3D", vol[None, None], m[None, None], v, lam, iterations,
                (1.0, 1.0, 1.0), extra={"w": w})


def random_case(rng, ndim, shape, channels=1, lam=None, iterations=2, v=1e10, soft=False,
                spacing=None, seeds=1):
    """Small random instance for property and edge-case tests."""
    spatial = tuple(shape)
    img = rng.uniform(0, 1, size=(1, channels) + spatial).astype(np.float32)
    if soft:
        m = rng.uniform(0, 1, size=spatial).astype(np.float32)
    else:
        m = np.ones(spatial, dtype=np.float32)
    for _ in range(seeds):
        idx = tuple(int(rng.integers(0, n)) for n in spatial)
        m[idx] = 0.0
    if lam is None:
        lam = float(np.float32(rng.uniform(0, 1)))
    return Case(f"random {ndim}D {spatial}", img, m[None, None], v, lam, iterations, spacing)
