"""Parity of the CUDA forward path with the oracle (GPU).

The bar is bit-exact float32 equality with the sequential oracle (IEEE
square root, no fused multiply-add), element by element, on the seeded
workloads at full size and on edge cases: ragged and tiny extents, several
tiles with rings and inter-tile waits, multi-channel images, every lambda
regime, zero iterations, in-place use and error paths.
"""
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


def gpu_run(fgx, case, options=None, out=None):
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    if case.ndim == 2:
        d = fgx.geodesic2d(img, m, case.v, case.lam, case.iterations, options=options,
                           check=True, out=out)
    else:
        d = fgx.geodesic3d(img, m, case.spacing, case.v, case.lam, case.iterations,
                           options=options, check=True, out=out)
    return d.cpu().numpy()


def oracle_run(case):
    return oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                      spacing=case.spacing, threads=THREADS)


def assert_bit_exact(got, want):
    assert got.shape == want.shape
    bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{bad.size} of {got.size} elements differ; first at flat index "
                             f"{i}: gpu {got.reshape(-1)[i]!r} oracle {want.reshape(-1)[i]!r}")


# ---------------------------------------------------------- seeded workloads

def test_plain2d_bit_exact(fgx):
    case = workloads.plain2d()
    assert_bit_exact(gpu_run(fgx, case), oracle_run(case))


@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("its", [2, 4])
def test_large2d_bit_exact(fgx, lam, its):
    case = workloads.large2d(lam=lam, iterations=its)
    assert_bit_exact(gpu_run(fgx, case), oracle_run(case))


def test_volume3d_bit_exact(fgx):
    case = workloads.volume3d()
    assert_bit_exact(gpu_run(fgx, case), oracle_run(case))


def test_differentiable_configs_forward_bit_exact(fgx):
    for case in (workloads.diff2d(), workloads.diff3d()):
        assert_bit_exact(gpu_run(fgx, case), oracle_run(case))


# ------------------------------------------------------------------ edges

SIDES = [1, 2, 31, 32, 33, 127, 129, 1000]


@pytest.mark.parametrize("H", SIDES)
def test_edge_shapes_2d(fgx, H):
    rng = np.random.default_rng(H)
    for W in SIDES:
        if H * W > 200_000:
            continue
        C = int(rng.integers(1, 5))
        lam = [0.0, 0.3, 1.0][int(rng.integers(0, 3))]
        case = workloads.random_case(rng, 2, (H, W), channels=C, lam=lam,
                                     iterations=int(rng.integers(1, 3)), soft=bool(H % 2),
                                     v=1e10 if W % 2 else 7.5)
        want = oracle_run(case)
        assert_bit_exact(gpu_run(fgx, case), want)
        # many small tiles: rings and neighbour waits on every block
        assert_bit_exact(gpu_run(fgx, case, options=dict(tile_width=8, tile_lines=3)), want)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 7), (6, 1, 9), (7, 8, 1), (9, 17, 33),
                                   (33, 31, 2), (16, 40, 24)])
def test_edge_shapes_3d(fgx, shape):
    rng = np.random.default_rng(sum(shape))
    for C, lam in [(1, 1.0), (2, 0.4), (3, 0.0)]:
        sp = tuple(float(x) for x in rng.uniform(0.5, 3.0, size=3))
        case = workloads.random_case(rng, 3, shape, channels=C, lam=lam, iterations=2,
                                     soft=True, v=20.0, spacing=sp)
        want = oracle_run(case)
        assert_bit_exact(gpu_run(fgx, case), want)
        assert_bit_exact(gpu_run(fgx, case, options=dict(tile_width=4, tile_height=3,
                                                          tile_lines=2)), want)


@pytest.mark.parametrize("lam,tiny", [(1.0, False), (1.0, True), (0.0, False)])
def test_plane_tiles_3d_bit_exact(fgx, lam, tiny):
    """3D passes over planes of several 24 x 24 tiles in both directions,
    three volumes (also in waves of blocks), anisotropic spacing; with tiny
    intensities the |d| cost takes its checked path."""
    rng = np.random.default_rng(31)
    shape = (30, 75, 53)
    img = rng.uniform(-50, 50, (3, 1) + shape).astype(np.float32)
    if tiny:
        img[1, 0, ::3] *= np.float32(1e-30)  # differences below 2^-63 occur
    m = np.ones((3, 1) + shape, np.float32)
    m[0, 0, 3, 4, 5] = 0
    m[1, 0, 29, 74, 52] = 0
    m[2, 0, 15, 37, 26] = 0
    m[2, 0, 0, 0, 0] = 0.5
    case = workloads.Case("tiles3d", img, m, 1e5, lam, 2, (2.0, 0.75, 1.25))
    want = oracle_run(case)
    assert_bit_exact(gpu_run(fgx, case), want)
    assert_bit_exact(gpu_run(fgx, case, options=dict(max_blocks=20)), want)


@pytest.mark.parametrize("shape", [(20, 36, 44), (19, 35, 45)])
@pytest.mark.parametrize("opts", [None, dict(max_blocks=10)])
def test_plane_tiles_3d_rings_and_staging(fgx, shape, opts):
    """Two volumes of three channels (general cost, lambda = 0.6): rows that
    are multiples of 4 floats are staged by tensor copies, others by
    per-lane copies; with the whole grid the planner takes the 8-wide ring
    (16 x 16 owned tiles), with 10 blocks the 4-wide one in waves."""
    rng = np.random.default_rng(sum(shape))
    img = rng.uniform(0, 1, (2, 3) + shape).astype(np.float32)
    m = rng.uniform(0, 1, (2, 1) + shape).astype(np.float32)
    m[0, 0, 2, 3, 4] = 0
    m[1, 0, -1, -2, -3] = 0
    case = workloads.Case("rings3d", img, m, 50.0, 0.6, 2, (1.5, 1.0, 0.5))
    assert_bit_exact(gpu_run(fgx, case, options=opts), oracle_run(case))


def test_batch_of_images_bit_exact(fgx):
    rng = np.random.default_rng(7)
    img = rng.uniform(0, 1, (5, 2, 70, 90)).astype(np.float32)
    m = rng.uniform(0, 1, (5, 1, 70, 90)).astype(np.float32)
    m[:, :, 10, 20] = 0
    case = workloads.Case("batch", img, m, 3.0, 0.6, 3)
    want = oracle_run(case)
    assert_bit_exact(gpu_run(fgx, case), want)
    # few resident blocks: instances run in waves
    assert_bit_exact(gpu_run(fgx, case, options=dict(tile_width=16, tile_lines=4,
                                                     max_blocks=12)), want)


def test_zero_iterations_returns_v_times_mask(fgx):
    case = workloads.plain2d(iterations=0)
    got = gpu_run(fgx, case)
    assert_bit_exact(got, (np.float32(case.v) * case.mask).astype(np.float32))


def test_in_place_on_mask(fgx):
    case = workloads.plain2d()
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    d = fgx.geodesic2d(img, m, case.v, case.lam, case.iterations, out=m, check=True)
    assert d.data_ptr() == m.data_ptr()
    assert_bit_exact(m.cpu().numpy(), oracle_run(case))


def test_empty_inputs(fgx):
    for shape in [(0, 1, 8, 8), (1, 1, 0, 8), (1, 1, 8, 0)]:
        img = torch.zeros(shape, device="cuda")
        m = torch.zeros((shape[0], 1) + shape[2:], device="cuda")
        d = fgx.geodesic2d(img, m, 1.0, 0.5, 2, check=True)
        assert d.shape == m.shape


def test_repeated_calls_are_identical(fgx):
    case = workloads.volume3d(shape=(40, 50, 60))
    a = gpu_run(fgx, case)
    b = gpu_run(fgx, case)
    assert_bit_exact(a, b)


def test_fwd_train_codes_match_oracle(fgx):
    for case in (workloads.diff2d(batch=2, size=96), workloads.diff3d(shape=(20, 24, 28))):
        img = torch.from_numpy(case.image).cuda()
        m = torch.from_numpy(case.mask).cuda()
        d, saved = fgx.forward_train(img, m, case.v, case.lam, case.iterations,
                                     spacing=case.spacing, check=True)
        want_d, want_codes = oracle.gdt(case.image, case.mask, case.v, case.lam,
                                        case.iterations, spacing=case.spacing,
                                        return_codes=True, threads=THREADS)
        assert_bit_exact(d.cpu().numpy(), want_d)
        np.testing.assert_array_equal(saved.cpu().numpy(), want_codes)


@pytest.mark.parametrize("lam,opts", [
    (0.75, None),                                             # rows and columns of 3 tiles
    (0.0, None),                                              # constant costs
    (1.0, dict(tile_width=16, tile_lines=8)),                 # many narrow tiles
    (0.5, dict(tile_width=24, tile_lines=16, max_blocks=14)),  # images in waves
])
def test_fwd_train_codes_2d_multi_tile(fgx, lam, opts):
    """2D parent codes of every pass application equal the oracle's, also
    with tiles, ring refreshes and several waves of images."""
    rng = np.random.default_rng(17)
    img = rng.uniform(0, 1, (3, 2, 150, 301)).astype(np.float32)
    m = np.ones((3, 1, 150, 301), np.float32)
    m[0, 0, 7, 9] = 0
    m[1, 0, 140, 290] = 0
    m[2, 0, 75, 150] = 0
    m[2, 0, 0, 300] = 0.25
    case = workloads.Case("codes2d", img, m, 3.0, lam, 2)
    d, saved = fgx.forward_train(torch.from_numpy(img).cuda(), torch.from_numpy(m).cuda(),
                                 case.v, lam, 2, options=opts, check=True)
    want_d, want_codes = oracle.gdt(img, m, case.v, lam, 2, return_codes=True, threads=THREADS)
    assert_bit_exact(d.cpu().numpy(), want_d)
    np.testing.assert_array_equal(saved.cpu().numpy(), want_codes)


@pytest.mark.parametrize("B,C,H,W,lam,its,segs,soft", [
    (1, 3, 700, 900, 0.5, 2, 3, False),   # converged second iteration: no re-runs
    (1, 1, 1000, 300, 1.0, 3, 5, False),  # five row segments, four column segments
    (2, 1, 512, 640, 0.0, 2, 4, False),   # two images, constant costs
    (1, 2, 400, 400, 0.3, 1, 6, True),    # soft mask: start lines change, re-runs
    (1, 1, 300, 2000, 0.8, 2, 8, True),   # short columns: fewer column segments
    (1, 1, 1500, 500, 0.5, 2, 3, True),   # long segments: re-runs that stop early
])
def test_speculative_segments_2d(fgx, B, C, H, W, lam, its, segs, soft):
    """Passes split into line segments that run at once from the old start
    lines, re-run in order where a start line changed: bit-exact to the
    oracle, and equal to the unsegmented kernel."""
    rng = np.random.default_rng(B * 1000 + H + W)
    img = np.stack([np.stack([workloads.blurred_noise(rng, (H, W)) for _ in range(C)])
                    for _ in range(B)])
    if soft:
        m = rng.uniform(0, 1, (B, 1, H, W)).astype(np.float32)
    else:
        m = np.stack([workloads.seed_block_mask(rng, (H, W), 5, 3)[None] for _ in range(B)])
    case = workloads.Case("segments", img.astype(np.float32), m.astype(np.float32),
                          10.0 if soft else 1e10, lam, its)
    want = oracle_run(case)
    assert_bit_exact(gpu_run(fgx, case, options=dict(segments=segs)), want)
    assert_bit_exact(gpu_run(fgx, case, options=dict(segments=1)), want)


# ----------------------------------------------------------------- errors

def test_error_codes(fgx):
    L = fgx.lib()
    dev = torch.zeros((1, 1, 8, 8), device="cuda")
    host = torch.zeros((1, 1, 8, 8))
    WS = fgx.workspace_size(2, 1, 1, 1, 8, 8)
    ws = torch.zeros(WS, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731

    def call(img, m, d, lam=0.5, v=1.0, its=2, wsb=None, H=8, W=8):
        wsb = WS if wsb is None else wsb
        return L.fgx_geodesic2d(P(img), P(m), P(d), 1, 1, H, W, v, lam, its, P(ws), wsb, None, s)

    out = torch.zeros_like(dev)
    assert call(dev, dev, out) == fgx.OK
    assert call(host, dev, out) == fgx.ERR_NOT_DEVICE_PTR
    assert call(dev, dev, out, lam=1.5) == fgx.ERR_ARG
    assert call(dev, dev, out, lam=float("nan")) == fgx.ERR_ARG
    assert call(dev, dev, out, v=0.0) == fgx.ERR_ARG
    assert call(dev, dev, out, v=float("inf")) == fgx.ERR_ARG
    assert call(dev, dev, out, its=-1) == fgx.ERR_ARG
    assert call(dev, dev, out, wsb=8) == fgx.ERR_WORKSPACE
    assert call(dev, dev, dev) == fgx.ERR_ARG  # dist aliases image
    assert call(dev, dev, out, H=-1) == fgx.ERR_SHAPE
    assert L.fgx_geodesic2d(None, P(dev), P(out), 1, 1, 8, 8, 1.0, 0.5, 1, P(ws), WS, None,
                            s) == fgx.ERR_ARG
    bad = fgx.Options()
    bad.size = 3
    assert L.fgx_geodesic2d(P(dev), P(dev), P(out), 1, 1, 8, 8, 1.0, 0.5, 1, P(ws), WS,
                            ctypes.byref(bad), s) == fgx.ERR_ARG
    sp = (ctypes.c_float * 3)(1.0, 0.0, 1.0)
    d3 = torch.zeros((1, 1, 2, 8, 8), device="cuda")
    o3 = torch.zeros_like(d3)
    assert L.fgx_geodesic3d(P(d3), P(d3), P(o3), 1, 1, 2, 8, 8, sp, 1.0, 0.5, 1, P(ws), WS,
                            None, s) == fgx.ERR_ARG
    torch.cuda.synchronize()


@pytest.mark.parametrize("shape,C", [((20, 36, 44), 1), ((17, 40, 28), 2), ((9, 64, 96), 3),
                                     ((15, 37, 29), 1), ((11, 30, 45), 2)])
def test_cost_tables_3d(fgx, shape, C):
    """The general 3D cost read from the per-call edge-cost tables and
    computed in every pass (no_cost_tables) both equal the oracle bit for
    bit, also with a forced ring width and with parent codes; W or H not a
    multiple of 4 runs on pitched working copies."""
    rng = np.random.default_rng(sum(shape) + C)
    sp = tuple(float(x) for x in rng.uniform(0.5, 3.0, size=3))
    case = workloads.random_case(rng, 3, shape, channels=C, lam=0.65, iterations=2, soft=True,
                                 v=20.0, spacing=sp)
    want = oracle_run(case)
    for opts in (None, dict(no_cost_tables=1), dict(tile_lines=8), dict(tile_lines=4)):
        assert_bit_exact(gpu_run(fgx, case, options=opts), want)
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    d, saved = fgx.forward_train(img, m, case.v, case.lam, case.iterations, spacing=case.spacing)
    dw, cw = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                        spacing=case.spacing, return_codes=True, threads=THREADS)
    assert_bit_exact(d.cpu().numpy(), dw)
    assert np.array_equal(saved.cpu().numpy().reshape(cw.shape), cw)
