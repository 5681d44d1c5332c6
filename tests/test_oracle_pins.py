"""Pins of the oracle against references other than itself (CPU only).

The oracle restates the raster-scan method of FastGeodis (Implementation
section) with the generalised-GDT cost of the Summary.  These tests tie it to:
shortest paths (the passes iterated to their fixed point compute multi-source
shortest paths on the 8/26-connected grid), closed forms (chamfer distance at
lambda = 0, total variation at lambda = 1), 1D brute force in float32,
invariants of the method, and hand-derived fixtures.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import pins

RTOL_FIXED_POINT = 1e-9


def _rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30)))


def _rand_case(rng, spatial, C, lam, soft, v):
    img = rng.uniform(0, 1, size=(1, C) + spatial)
    if soft:
        m = rng.uniform(0, 1, size=spatial)
    else:
        m = np.ones(spatial)
    m[tuple(int(rng.integers(0, n)) for n in spatial)] = 0.0
    return img, m[None, None], v, lam


# ---------------------------------------------------------------- P1 Dijkstra

@pytest.mark.parametrize("shape,C,lam,soft", [
    ((32, 32), 1, 1.0, False), ((32, 32), 3, 0.5, False), ((24, 31), 2, 0.0, False),
    ((17, 32), 1, 0.3, True), ((32, 9), 3, 0.75, True), ((1, 29), 1, 0.6, False),
])
def test_fixed_point_is_dijkstra_2d(shape, C, lam, soft):
    rng = np.random.default_rng(hash((shape, C, lam, soft)) % 2**32)
    img, m, v, lam = _rand_case(rng, shape, C, lam, soft, v=3.0 if soft else 1e10)
    d, its = oracle.fixed_point(img, m, v, lam)
    ref = pins.dijkstra_distance(img[0], m[0, 0], v, lam)
    assert its >= 1
    assert _rel_err(d[0, 0], ref) < RTOL_FIXED_POINT


@pytest.mark.parametrize("shape,C,lam,spacing", [
    ((12, 12, 12), 1, 1.0, (2.5, 1.0, 1.0)), ((9, 11, 13), 2, 0.5, (1.0, 1.0, 1.0)),
    ((10, 8, 7), 1, 0.0, (2.5, 1.0, 1.0)), ((6, 13, 9), 1, 0.0, (0.7, 1.3, 2.1)),
    ((8, 8, 8), 3, 0.75, (1.0, 2.0, 0.5)),
])
def test_fixed_point_is_dijkstra_3d(shape, C, lam, spacing):
    rng = np.random.default_rng(hash((shape, C, lam)) % 2**32)
    img, m, v, lam = _rand_case(rng, shape, C, lam, False, v=1e10)
    d, _ = oracle.fixed_point(img, m, v, lam, spacing=spacing)
    ref = pins.dijkstra_distance(img[0], m[0, 0], v, lam, spacing)
    assert _rel_err(d[0, 0], ref) < RTOL_FIXED_POINT


def test_fixed_point_is_dijkstra_on_plain_config_crop():
    """32x32 crop of the 2D plain workload centred on its seed block."""
    case = workloads.plain2d()
    m = case.mask[0, 0]
    ys, xs = np.nonzero(m == 0)
    cy, cx = int(ys.mean()), int(xs.mean())
    y0 = int(np.clip(cy - 16, 0, m.shape[0] - 32))
    x0 = int(np.clip(cx - 16, 0, m.shape[1] - 32))
    img = case.image[:, :, y0:y0 + 32, x0:x0 + 32]
    mc = case.mask[:, :, y0:y0 + 32, x0:x0 + 32]
    assert (mc == 0).sum() == 25
    d, _ = oracle.fixed_point(img, mc, case.v, case.lam)
    ref = pins.dijkstra_distance(img[0], mc[0, 0], case.v, case.lam)
    assert _rel_err(d[0, 0], ref) < RTOL_FIXED_POINT


@pytest.mark.parametrize("shape,lam", [((3, 3), 0.5), ((3, 3), 1.0), ((2, 4), 0.0),
                                       ((2, 2, 2), 0.4)])
def test_fixed_point_is_brute_force_minimum(shape, lam):
    rng = np.random.default_rng(len(shape) * 7 + int(lam * 10))
    img = rng.uniform(0, 1, size=(1, 1) + shape)
    m = rng.uniform(0, 1, size=shape)[None, None]
    v = 4.0
    d, _ = oracle.fixed_point(img, m, v, lam)
    ref = pins.brute_force_paths(img[0], m[0, 0], v, lam)
    assert _rel_err(d[0, 0], ref) < RTOL_FIXED_POINT


# ---------------------------------------------------------------- P2 chamfer

@pytest.mark.parametrize("shape,seed", [((40, 33), (7, 20)), ((16, 64), (15, 0)),
                                        ((1, 20), (0, 5))])
def test_lambda0_one_iteration_is_chamfer_2d(shape, seed):
    img = np.random.default_rng(0).uniform(0, 1, size=(1, 1) + shape)
    m = np.ones(shape)
    m[seed] = 0
    d = oracle.gdt(img, m[None, None], 1e10, 0.0, 1, dtype=np.float64)[0, 0]
    hh, ww = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    a = np.abs(hh - seed[0])
    b = np.abs(ww - seed[1])
    ref = np.sqrt(2.0) * np.minimum(a, b) + (np.maximum(a, b) - np.minimum(a, b))
    np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-12)


def test_lambda0_one_iteration_is_chamfer_3d():
    shape, seed = (9, 14, 11), (3, 10, 2)
    img = np.random.default_rng(1).uniform(0, 1, size=(1, 2) + shape)
    m = np.ones(shape)
    m[seed] = 0
    d = oracle.gdt(img, m[None, None], 1e10, 0.0, 1, dtype=np.float64)[0, 0]
    g = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    dd = np.sort(np.stack([np.abs(g[i] - seed[i]) for i in range(3)]), axis=0)
    ref = (np.sqrt(3.0) * dd[0] + np.sqrt(2.0) * (dd[1] - dd[0]) + (dd[2] - dd[1]))
    np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-12)


def test_lambda0_float32_within_summation_error_of_chamfer():
    shape, seed = (128, 96), (40, 70)
    m = np.ones(shape)
    m[seed] = 0
    img = np.zeros((1, 1) + shape)
    d = oracle.gdt(img, m[None, None], 1e10, 0.0, 1, dtype=np.float32)[0, 0]
    hh, ww = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    a, b = np.abs(hh - seed[0]), np.abs(ww - seed[1])
    ref = np.sqrt(2.0) * np.minimum(a, b) + (np.maximum(a, b) - np.minimum(a, b))
    steps = np.maximum(a, b)
    # sequential float32 sums of `steps` terms: relative error <= steps * 2^-24
    assert np.all(np.abs(d - ref) <= (steps + 1) * 2.0**-24 * np.maximum(ref, 1) + 1e-7)


# ------------------------------------------------------- P3 total variation

def test_lambda1_monotone_rows_give_total_variation():
    H, W, w0 = 23, 41, 17
    f = np.cumsum(np.random.default_rng(2).uniform(0.01, 1.0, size=W))
    img = np.broadcast_to(f, (H, W))[None, None].copy()
    m = np.ones((H, W))
    m[:, w0] = 0
    d = oracle.gdt(img, m[None, None], 1e10, 1.0, 1, dtype=np.float64)[0, 0]
    ref = np.broadcast_to(np.abs(f - f[w0]), (H, W))
    np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-12)


def test_lambda1_flat_region_is_exactly_zero():
    """Piecewise-constant image: distance is exactly 0 on the seed's
    8-connected flat region and positive elsewhere."""
    from scipy.ndimage import label
    rng = np.random.default_rng(3)
    levels = rng.integers(0, 3, size=(6, 6)).repeat(4, 0).repeat(4, 1).astype(np.float64)
    m = np.ones(levels.shape)
    m[5, 5] = 0
    d, _ = oracle.fixed_point(levels[None, None], m[None, None], 1e10, 1.0)
    lab, _ = label(levels == levels[5, 5], structure=np.ones((3, 3)))
    region = lab == lab[5, 5]
    assert np.all(d[0, 0][region] == 0.0)
    assert np.all(d[0, 0][~region] > 0.0)
    d32 = oracle.gdt(levels[None, None].astype(np.float32), m[None, None].astype(np.float32),
                     1e10, 1.0, 50)
    assert np.all(d32[0, 0][region] == 0.0)


# -------------------------------------------------- 1D brute force (float32)

@pytest.mark.parametrize("n,C,lam,soft", [(37, 1, 1.0, False), (50, 3, 0.5, True),
                                          (9, 2, 0.0, True), (64, 1, 0.25, True)])
@pytest.mark.parametrize("axis", ["H", "W"])
def test_line_inputs_match_brute_force_bit_exact_2d(n, C, lam, soft, axis):
    rng = np.random.default_rng(n * 31 + C)
    img = rng.uniform(0, 1, size=(C, n)).astype(np.float32)
    m = (rng.uniform(0, 1, size=n) if soft else np.ones(n)).astype(np.float32)
    m[int(rng.integers(0, n))] = 0
    v = 7.0 if soft else 1e10
    ref = pins.line_brute_force_f32(img, m, v, lam)
    shp = (n, 1) if axis == "H" else (1, n)
    d = oracle.gdt(img.reshape((1, C) + shp), m.reshape((1, 1) + shp), v, lam, 1)
    np.testing.assert_array_equal(d.reshape(-1), ref)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_inputs_match_brute_force_bit_exact_3d(axis):
    n, C, lam = 33, 2, 0.7
    spacing = (2.5, 1.25, 0.75)
    rng = np.random.default_rng(axis)
    img = rng.uniform(0, 1, size=(C, n)).astype(np.float32)
    m = rng.uniform(0, 1, size=n).astype(np.float32)
    m[5] = 0
    ref = pins.line_brute_force_f32(img, m, 9.0, lam, step_spacing=spacing[axis])
    shp = [1, 1, 1]
    shp[axis] = n
    d = oracle.gdt(img.reshape([1, C] + shp), m.reshape([1, 1] + shp), 9.0, lam, 1,
                   spacing=spacing)
    np.testing.assert_array_equal(d.reshape(-1), ref)


# -------------------------------------------------------------- P4 invariants

def _small_configs():
    p = workloads.plain2d()
    yield p.image, p.mask, p.v, p.lam, None
    L = workloads.large2d(size=160)
    yield L.image, L.mask, L.v, L.lam, None
    V = workloads.volume3d(shape=(20, 24, 28))
    yield V.image, V.mask, V.v, V.lam, V.spacing
    Df = workloads.diff2d(batch=2, size=48)
    yield Df.image, Df.mask, Df.v, Df.lam, None


@pytest.mark.parametrize("k", range(4))
def test_invariants(k):
    img, m, v, lam, sp = list(_small_configs())[k]
    prev = None
    for it in range(0, 4):
        d = oracle.gdt(img, m, v, lam, it, spacing=sp)
        v0 = (np.float32(v) * m.astype(np.float32))
        assert np.all(d >= 0)
        assert np.all(d <= v0)
        assert np.all(d[m == 0] == 0)
        if it == 0:
            np.testing.assert_array_equal(d, v0)
        if prev is not None:
            assert np.all(d <= prev)
        prev = d


def test_fixed_point_does_not_depend_on_pass_order():
    rng = np.random.default_rng(5)
    img, m, v, lam = _rand_case(rng, (20, 23), 2, 0.6, True, 5.0)
    a, _ = oracle.gdt_schedule(img, m, v, lam, oracle.PASSES_2D, -1)
    b, _ = oracle.gdt_schedule(img, m, v, lam, [(2, -1), (1, +1), (2, +1), (1, -1)], -1)
    assert _rel_err(a, b) < 1e-12
    img3, m3, v3, lam3 = _rand_case(rng, (7, 9, 8), 1, 0.4, True, 5.0)
    a3, _ = oracle.gdt_schedule(img3, m3, v3, lam3, oracle.PASSES_3D, -1, (2.0, 1.0, 1.0))
    b3, _ = oracle.gdt_schedule(img3, m3, v3, lam3, list(reversed(oracle.PASSES_3D)), -1,
                                (2.0, 1.0, 1.0))
    assert _rel_err(a3, b3) < 1e-12


def test_float32_close_to_float64():
    case = workloads.large2d(size=96)
    d32 = oracle.gdt(case.image, case.mask, case.v, case.lam, 2)
    d64 = oracle.gdt(case.image, case.mask, case.v, case.lam, 2, dtype=np.float64)
    assert _rel_err(d32, d64) < 1e-4


def test_threads_do_not_change_results():
    case = workloads.volume3d(shape=(16, 20, 24))
    a = oracle.gdt(case.image, case.mask, case.v, case.lam, 2, spacing=case.spacing)
    b = oracle.gdt(case.image, case.mask, case.v, case.lam, 2, spacing=case.spacing,
                   threads=4)
    np.testing.assert_array_equal(a, b)


def test_degenerate_shapes():
    for shape in [(1, 1), (1, 7), (7, 1), (0, 5)]:
        img = np.ones((1, 1) + shape, np.float32)
        m = np.ones((1, 1) + shape, np.float32)
        if m.size:
            m.reshape(-1)[0] = 0
        d = oracle.gdt(img, m, 1e10, 0.5, 2)
        assert d.shape == m.shape
    # zero iterations return v*M
    m = np.random.default_rng(0).uniform(0, 1, (1, 1, 5, 6)).astype(np.float32)
    d = oracle.gdt(np.zeros((1, 1, 5, 6), np.float32), m, 3.0, 0.5, 0)
    np.testing.assert_array_equal(d, np.float32(3.0) * m)


# ----------------------------------------------------------------- fixtures

@pytest.mark.parametrize("name", ["chamfer_3x3_centre.txt", "tv_row_lambda1.txt",
                                  "mixture_row_lambda_half.txt", "spacing_3x3x3_centre.txt"])
def test_golden_fixtures(name):
    g = pins.load_golden(name)
    shape = tuple(int(s) for s in (g["shape"] if isinstance(g["shape"], list) else [g["shape"]]))
    C = int(g["channels"])
    img = np.array(g["image"], np.float32).reshape((1, C) + shape)
    m = np.array(g["mask"], np.float32).reshape((1, 1) + shape)
    sp = tuple(g["spacing"]) if "spacing" in g else None
    d = oracle.gdt(img, m, g["v"], g["lambda"], int(g["iterations"]), spacing=sp)
    np.testing.assert_array_equal(d.reshape(-1), np.array(g["expect"], np.float32))


# ------------------------------------------------------------ codes (argmin)

def test_codes_name_a_parent_that_realises_the_value():
    """In the last pass (right-left) every element with a non-zero code holds
    exactly D[parent] + c(parent, x) in float32, with the parent on its right;
    seeds (M = 0) never record a parent."""
    f = np.float32
    rng = np.random.default_rng(9)
    H, W, lam = 13, 17, f(0.6)
    img = rng.uniform(0, 1, (1, 2, H, W)).astype(f)
    m = rng.uniform(0, 1, (1, 1, H, W)).astype(f)
    m[0, 0, 3, 4] = 0
    d, codes = oracle.gdt(img, m, 5.0, lam, 1, return_codes=True)
    assert codes.shape == (4, 1, H * W) and codes.max() <= 3
    last = codes[-1, 0].reshape(H, W)
    D = d[0, 0]
    checked = 0
    for h in range(H):
        for w in range(W - 1):
            k = int(last[h, w])
            if k == 0:
                continue
            ph, pw = h + (k - 2), w + 1
            s2 = f(f(1) + f((k - 2) * (k - 2)))
            di2 = f(0)
            for ch in range(2):
                dd = f(img[0, ch, h, w] - img[0, ch, ph, pw])
                di2 = f(di2 + f(dd * dd))
            c = f(np.sqrt(f(f(f(1) - lam) * s2) + f(lam * di2)))
            assert D[h, w] == f(D[ph, pw] + c)
            checked += 1
    assert checked > 0
    assert np.all(codes[:, :, np.flatnonzero(m.reshape(-1) == 0)] == 0)
