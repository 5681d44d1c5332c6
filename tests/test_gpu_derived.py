"""Parity of the derived transforms with the oracle (GPU): the Euclidean
entry points (lambda = 0, no image), the signed transform GDT(M) - GDT(1 - M)
and geodesic symmetric filtering, bit for bit in float32."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def fgx():
    from paper_2208_00001_gb300 import build
    build.build()
    import paper_2208_00001_gb300 as m
    return m


def _bits(got, want, what):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    assert got.shape == want.shape, what
    bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
    assert bad.size == 0, f"{what}: {bad.size} of {got.size} differ"


@pytest.mark.parametrize("shape,spacing,its", [
    ((2, 1, 300, 700), None, 2),          # several line tiles and segments
    ((1, 1, 45, 71), None, 1),
    ((1, 1, 40, 90, 70), (2.5, 1.0, 1.0), 2),
    ((2, 1, 17, 30, 33), (1.0, 0.5, 2.0), 1),
])
def test_euclidean_bit_exact(fgx, shape, spacing, its):
    rng = np.random.default_rng(sum(shape))
    m = rng.uniform(0, 1, shape).astype(np.float32)
    m[(0, 0) + tuple(n // 3 for n in shape[2:])] = 0.0
    want = oracle.euclidean(m, 7.0, its, spacing=spacing, threads=THREADS)
    got = fgx.euclidean(torch.from_numpy(m).cuda(), 7.0, its, spacing=spacing, check=True)
    _bits(got.cpu().numpy(), want, f"euclidean {shape}")


@pytest.mark.parametrize("B,C,spatial,lam,its,spacing", [
    (1, 3, (700, 900), 0.5, 2, None),
    (2, 1, (130, 257), 1.0, 3, None),
    (1, 2, (36, 70, 55), 0.6, 2, (2.5, 1.0, 1.0)),
    (2, 1, (20, 33, 41), 0.0, 1, (1.0, 1.0, 1.0)),
    (2, 2, (24, 40, 44), 0.5, 2, (1.5, 1.0, 1.0)),   # tensor-copy staging, 4 transforms
])
def test_signed_bit_exact(fgx, B, C, spatial, lam, its, spacing):
    rng = np.random.default_rng(B * 100 + C + sum(spatial))
    img = np.stack([np.stack([workloads.blurred_noise(rng, spatial) for _ in range(C)])
                    for _ in range(B)]).astype(np.float32)
    m = np.ones((B, 1) + spatial, np.float32)
    sl = tuple(slice(n // 4, n // 2) for n in spatial)
    m[(slice(None), 0) + sl] = 0.0
    m[0, 0][tuple(n - 1 for n in spatial)] = 0.25  # one soft value
    want = oracle.signed_gdt(img, m, 1e10, lam, its, spacing=spacing, threads=THREADS)
    got = fgx.signed_geodesic(torch.from_numpy(img).cuda(), torch.from_numpy(m).cuda(), 1e10,
                              lam, its, spacing=spacing, check=True)
    _bits(got.cpu().numpy(), want, "signed")
    assert np.all(want[m == 0] < 0) and np.all(want[m == 1] >= 0)


def test_signed_in_place_on_mask(fgx):
    rng = np.random.default_rng(8)
    img = rng.uniform(0, 1, (1, 1, 50, 61)).astype(np.float32)
    m = np.ones((1, 1, 50, 61), np.float32)
    m[0, 0, 10:20, 30:40] = 0.0
    want = oracle.signed_gdt(img, m, 1e10, 0.5, 2, threads=THREADS)
    mt = torch.from_numpy(m).cuda()
    got = fgx.signed_geodesic(torch.from_numpy(img).cuda(), mt, 1e10, 0.5, 2, out=mt,
                              check=True)
    assert got.data_ptr() == mt.data_ptr()
    _bits(mt.cpu().numpy(), want, "signed in place")


def test_image_required_unless_euclidean(fgx):
    L = fgx.lib()
    m = torch.ones((1, 1, 8, 8), device="cuda")
    d = torch.empty_like(m)
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    assert L.fgx_geodesic2d(None, P(m), P(d), 1, 1, 8, 8, 1.0, 0.5, 1, P(ws), ws.numel(), None,
                            s) == fgx.ERR_ARG
    assert L.fgx_geodesic2d(None, P(m), P(d), 1, 1, 8, 8, 1.0, 0.0, 1, P(ws), ws.numel(), None,
                            s) == fgx.OK
    torch.cuda.synchronize()
    assert torch.all(d == oracle_free_expected(m))


def oracle_free_expected(m):
    # all-ones mask without seeds: every value stays v * M = 1
    return torch.ones_like(m)


def test_signed_with_tile_options_bit_exact(fgx):
    """The tiled engine serves the batched pair too (both transforms read the
    same image)."""
    rng = np.random.default_rng(12)
    img = rng.uniform(0, 1, (2, 2, 15, 27, 22)).astype(np.float32)
    m = np.ones((2, 1, 15, 27, 22), np.float32)
    m[0, 0, 3, 4, 5] = 0.0
    m[1, 0, 10:12, 20:25, 1:4] = 0.0
    want = oracle.signed_gdt(img, m, 1e10, 0.7, 2, spacing=(1.0, 1.5, 0.5), threads=THREADS)
    got = fgx.signed_geodesic(torch.from_numpy(img).cuda(), torch.from_numpy(m).cuda(), 1e10,
                              0.7, 2, spacing=(1.0, 1.5, 0.5),
                              options=dict(tile_width=8, tile_height=6, tile_lines=3),
                              check=True)
    _bits(got.cpu().numpy(), want, "signed, tile options")


def _objects(rng, shape, B):
    """Indicators (1 = object) of blobs of several sizes with small holes."""
    f = np.zeros((B, 1) + shape, np.float32)
    for b in range(B):
        for _ in range(6):
            lo = [int(rng.integers(0, max(n - 4, 1))) for n in shape]
            size = [int(rng.integers(2, max(n // 3, 3))) for n in shape]
            f[(b, 0) + tuple(slice(l, l + z) for l, z in zip(lo, size))] = 1.0
        holes = tuple(rng.integers(0, n, 20) for n in shape)
        f[(b, 0) + holes] = 0.0
    return f


@pytest.mark.parametrize("B,C,spatial,lam,its,spacing,td,te,opts", [
    (2, 3, (300, 410), 0.5, 2, None, 2.5, 1.5, None),
    (1, 1, (257, 130), 0.0, 1, None, 3.0, 3.0, None),
    (2, 1, (24, 40, 44), 0.8, 2, (2.0, 1.0, 1.0), 1.7, 2.2, None),   # tensor-copy staging
    (1, 2, (19, 35, 31), 0.4, 2, (1.0, 1.0, 1.5), 2.0, 0.5, None),
    (1, 1, (14, 26, 23), 0.6, 1, (1.0, 1.0, 1.0), 1.5, 0.6,
     dict(tile_width=8, tile_height=6, tile_lines=3)),
])
def test_gsf_bit_exact(fgx, B, C, spatial, lam, its, spacing, td, te, opts):
    rng = np.random.default_rng(B * 10 + C + sum(spatial))
    img = np.stack([np.stack([workloads.blurred_noise(rng, spatial) for _ in range(C)])
                    for _ in range(B)]).astype(np.float32)
    f = _objects(rng, spatial, B)
    want = oracle.gsf(img, f, 1e10, lam, its, td, te, spacing=spacing, threads=THREADS)
    got = fgx.gsf(torch.from_numpy(img).cuda(), torch.from_numpy(f).cuda(), 1e10, lam, its, td,
                  te, spacing=spacing, options=opts, check=True)
    _bits(got.cpu().numpy(), want, "gsf")
    assert 0 < want.sum() < want.size


def test_gsf_in_place_and_argument_checks(fgx):
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 1, (1, 1, 60, 70)).astype(np.float32)
    f = _objects(rng, (60, 70), 1)
    want = oracle.gsf(img, f, 1e10, 0.5, 2, 1.5, 1.5, threads=THREADS)
    ft = torch.from_numpy(f).cuda()
    got = fgx.gsf(torch.from_numpy(img).cuda(), ft, 1e10, 0.5, 2, 1.5, 1.5, out=ft, check=True)
    assert got.data_ptr() == ft.data_ptr()
    _bits(ft.cpu().numpy(), want, "gsf in place")
    with pytest.raises(fgx.FgxError):
        fgx.gsf(torch.from_numpy(img).cuda(), ft, 1e10, 0.5, 2, -1.0, 1.5)
