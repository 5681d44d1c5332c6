"""Pins of the oracle's derived transforms (CPU only): the Euclidean
transform (lambda = 0) and the signed transform GDT(M) - GDT(1 - M).

The paper names signed geodesic distance among the applications of the
transform without a definition; the reading pinned here is the difference of
the transforms seeded by the region M = 0 and by M = 1.  Pins: the
half-plane closed form (at lambda = 0 the distance to a half-plane of seeds
is the number of steps times the spacing along that axis), exact
antisymmetry under M -> 1 - M, and the Euclidean transform's single-seed
chamfer closed form.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("H,W,x0", [(9, 14, 6), (1, 7, 1), (12, 5, 4)])
def test_signed_half_plane_closed_form_2d(H, W, x0):
    # seeds of GDT(M): columns < x0 (M = 0); of GDT(1 - M): columns >= x0
    m = np.ones((1, 1, H, W), np.float32)
    m[..., :x0] = 0.0
    img = np.random.default_rng(0).uniform(0, 1, (1, 1, H, W)).astype(np.float32)
    got = oracle.signed_gdt(img, m, 1e10, 0.0, 1)
    x = np.arange(W, dtype=np.float64)
    want = np.where(x >= x0, x - x0 + 1, -(x0 - x))
    np.testing.assert_array_equal(got[0, 0], np.broadcast_to(want, (H, W)).astype(np.float32))


def test_signed_half_space_closed_form_3d_anisotropic():
    # split along D with spacing 2.5: distances are multiples of 2.5
    D, H, W, d0 = 7, 5, 6, 3
    m = np.ones((1, 1, D, H, W), np.float32)
    m[:, :, :d0] = 0.0
    img = np.zeros((1, 1, D, H, W), np.float32)
    got = oracle.signed_gdt(img, m, 1e10, 0.0, 1, spacing=(2.5, 1.0, 1.0))
    d = np.arange(D, dtype=np.float64)
    want = np.where(d >= d0, (d - d0 + 1) * 2.5, -(d0 - d) * 2.5)
    np.testing.assert_array_equal(got[0, 0], np.broadcast_to(want[:, None, None], (D, H, W)))


@pytest.mark.parametrize("lam,its", [(0.5, 2), (1.0, 1), (0.0, 3)])
def test_signed_antisymmetric(lam, its):
    # masks whose complement is exact in float32 (binary and k/8 values)
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 1, (2, 2, 13, 17)).astype(np.float32)
    m = (rng.integers(0, 9, (2, 1, 13, 17)) / 8.0).astype(np.float32)
    m[0, 0, 3, 4] = 0.0
    m[1, 0, 10, 2] = 1.0
    a = oracle.signed_gdt(img, m, 5.0, lam, its)
    b = oracle.signed_gdt(img, (1 - m).astype(np.float32), 5.0, lam, its)
    np.testing.assert_array_equal(a, -b)


def test_signed_sign_on_binary_mask():
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, (1, 1, 20, 23)).astype(np.float32)
    m = np.ones((1, 1, 20, 23), np.float32)
    m[..., 5:11, 7:15] = 0.0
    s = oracle.signed_gdt(img, m, 1e10, 0.7, 2)
    assert np.all(s[m == 0] <= 0) and np.all(s[m == 1] >= 0)
    assert np.all(s[m == 0] < 0)  # the complement's seeds are at least one step away


def test_euclidean_single_seed_chamfer():
    # one iteration of the four passes gives the 8-neighbour chamfer distance
    # (max - min) + sqrt(2) * min from a single seed
    H, W, (sy, sx) = 15, 19, (6, 11)
    m = np.ones((1, 1, H, W), np.float32)
    m[0, 0, sy, sx] = 0.0
    got = oracle.euclidean(m, 1e10, 1)[0, 0].astype(np.float64)
    dy = np.abs(np.arange(H)[:, None] - sy)
    dx = np.abs(np.arange(W)[None, :] - sx)
    want = np.maximum(dy, dx) - np.minimum(dy, dx) + np.sqrt(2.0) * np.minimum(dy, dx)
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=0)


def test_euclidean_ignores_the_image():
    rng = np.random.default_rng(5)
    m = rng.uniform(0, 1, (1, 1, 11, 9)).astype(np.float32)
    img = rng.uniform(0, 1, (1, 3, 11, 9)).astype(np.float32)
    np.testing.assert_array_equal(oracle.euclidean(m, 3.0, 2),
                                  oracle.gdt(img, m, 3.0, 0.0, 2))


def test_signed_golden_fixture():
    from tests import pins
    g = pins.load_golden("signed_3x3_centre.txt")
    img = np.array(g["image"], np.float32).reshape(1, 1, 3, 3)
    m = np.array(g["mask"], np.float32).reshape(1, 1, 3, 3)
    got = oracle.signed_gdt(img, m, g["v"], g["lambda"], int(g["iterations"]))
    np.testing.assert_array_equal(got.reshape(-1), np.array(g["expect"], np.float32))


# ------------------------------------------------ geodesic symmetric filtering
# The reading (the paper names GSF without defining it): S(X) = GDT(1 - X) -
# GDT(X) for an indicator X (1 = object), erosion [S(F) < -theta_e],
# dilation [S(F) < theta_d], result [(S(F_e) + S(F_d)) + theta_d - theta_e < 0].

@pytest.mark.parametrize("td,te", [(1.5, 2.5), (2.5, 1.5), (0.7, 0.7), (3.2, 0.0)])
def test_gsf_keeps_a_half_plane(td, te):
    """At lambda = 0 a half-plane object stays the same half-plane: erosion
    and dilation shift its edge by whole steps in opposite directions and
    the symmetric combination puts it back (a wrong sign of either term or
    of theta_d - theta_e moves the edge)."""
    H, W, x0 = 6, 16, 7
    f = np.zeros((1, 1, H, W), np.float32)
    f[..., x0:] = 1.0
    img = np.random.default_rng(1).uniform(0, 1, (1, 1, H, W)).astype(np.float32)
    np.testing.assert_array_equal(oracle.gsf(img, f, 1e10, 0.0, 2, td, te), f)


def test_gsf_keeps_a_half_space_3d_anisotropic():
    D, H, W, d0 = 9, 4, 5, 4
    f = np.zeros((1, 1, D, H, W), np.float32)
    f[:, :, d0:] = 1.0
    img = np.zeros((1, 1, D, H, W), np.float32)
    got = oracle.gsf(img, f, 1e10, 0.0, 2, 5.5, 3.0, spacing=(2.5, 1.0, 1.0))
    np.testing.assert_array_equal(got, f)


def test_gsf_removes_thin_objects_and_fills_narrow_holes():
    """A 3 x 3 object vanishes under an erosion of 2.5 (its centre is 2 steps
    from the background); a one-pixel hole in a large object closes under a
    dilation of 1.5; both survive smaller thresholds."""
    img = np.zeros((1, 1, 30, 30), np.float32)
    f = np.zeros((1, 1, 30, 30), np.float32)
    f[..., 3:6, 3:6] = 1.0          # small object
    f[..., 12:28, 10:28] = 1.0      # large object ...
    f[..., 20, 19] = 0.0            # ... with a one-pixel hole
    out = oracle.gsf(img, f, 1e10, 0.0, 2, 1.5, 2.5)
    assert out[..., 3:6, 3:6].sum() == 0
    assert out[0, 0, 20, 19] == 1.0
    assert out[..., 14:26, 12:26].min() == 1.0
    kept = oracle.gsf(img, f, 1e10, 0.0, 2, 0.5, 0.5)
    assert kept[..., 4, 4] == 1.0 and kept[0, 0, 20, 19] == 0.0


@pytest.mark.parametrize("lam", [0.0, 0.4, 0.9])
def test_gsf_with_zero_thresholds_is_the_identity(lam):
    """With positive step costs (lambda < 1) S(F) < 0 exactly inside a binary
    object and > 0 outside, so zero thresholds reproduce F."""
    rng = np.random.default_rng(7)
    img = rng.uniform(0, 1, (2, 2, 15, 19)).astype(np.float32)
    f = (rng.uniform(0, 1, (2, 1, 15, 19)) < 0.4).astype(np.float32)
    np.testing.assert_array_equal(oracle.gsf(img, f, 1e10, lam, 2, 0.0, 0.0), f)


@pytest.mark.parametrize("lam", [0.3, 1.0])
def test_gsf_complement_symmetry(lam):
    """Filtering the background with the thresholds swapped gives the
    complement: S(1 - F) = -S(F) exactly, so erosion and dilation trade
    places and every sum changes sign (thresholds chosen off the distances
    that occur, so no comparison ties)."""
    rng = np.random.default_rng(8)
    img = rng.uniform(0, 1, (1, 1, 21, 24)).astype(np.float32)
    f = (rng.uniform(0, 1, (1, 1, 21, 24)) < 0.5).astype(np.float32)
    a = oracle.gsf(img, f, 1e10, lam, 2, 1.23456, 0.87654)
    b = oracle.gsf(img, (1 - f).astype(np.float32), 1e10, lam, 2, 0.87654, 1.23456)
    np.testing.assert_array_equal(a, 1 - b)
