"""Parity of the CUDA reverse sweep with the oracle's (GPU).

The GPU records parent codes in the forward (checked equal to the oracle's
codes in the forward tests) and runs the adjoint through them; with identical
codes the float32 gradients must match the oracle's float32 reverse sweep bit
for bit (same accumulation order: children in offset order, parent-side image
terms before the child-side term).
"""
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


def _bits_equal(got, want, what):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    assert got.shape == want.shape, what
    bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size}/{got.size} differ; first {i}: "
                             f"gpu {got.reshape(-1)[i]!r} oracle {want.reshape(-1)[i]!r}")


def _run(fgx, case, w, options=None, need_image=True, need_mask=True):
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    d, saved = fgx.forward_train(img, m, case.v, case.lam, case.iterations,
                                 spacing=case.spacing, options=options, check=True)
    g = torch.from_numpy(w).cuda()
    gi, gm = fgx.backward(g, img, saved, case.v, case.lam, case.iterations,
                          spacing=case.spacing, need_image=need_image, need_mask=need_mask,
                          options=options, check=True)
    return (d.cpu().numpy(), saved.cpu().numpy(), None if gi is None else gi.cpu().numpy(),
            None if gm is None else gm.cpu().numpy())


def _oracle(case, w, codes):
    return oracle.backward(w, case.image, codes, case.v, case.lam, case.iterations,
                           spacing=case.spacing)


@pytest.mark.parametrize("v", [1e10, 10.0])
def test_backward_2d_bit_exact(fgx, v):
    case = workloads.diff2d(batch=2, size=96, v=v)
    w = case.extra["w"]
    d, codes, gi, gm = _run(fgx, case, w)
    want_d, want_codes = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                                    return_codes=True, threads=THREADS)
    np.testing.assert_array_equal(codes, want_codes)
    wi, wm = _oracle(case, w, want_codes)
    _bits_equal(gi, wi, "grad_image")
    _bits_equal(gm, wm, "grad_mask")
    assert np.abs(gi).sum() > 0


def test_backward_2d_many_tiles_and_channels(fgx):
    rng = np.random.default_rng(21)
    img = rng.uniform(0, 1, (3, 2, 45, 70)).astype(np.float32)
    m = rng.uniform(0, 1, (3, 1, 45, 70)).astype(np.float32)
    m[:, :, 10, 20] = 0
    case = workloads.Case("mc", img, m, 5.0, 0.6, 2)
    w = rng.uniform(0, 1, m.shape).astype(np.float32)
    for opts in (None, dict(tile_width=8, tile_lines=3), dict(tile_width=16, tile_lines=5,
                                                             max_blocks=12)):
        d, codes, gi, gm = _run(fgx, case, w, options=opts)
        wi, wm = _oracle(case, w, codes)
        _bits_equal(gi, wi, f"grad_image {opts}")
        _bits_equal(gm, wm, f"grad_mask {opts}")


@pytest.mark.parametrize("C,lam", [(3, 0.6), (5, 0.3), (1, 0.0)])
def test_backward_2d_multi_tile_bit_exact(fgx, C, lam):
    """Reverse sweep over rows and columns of several line tiles (default
    geometry, ring refreshes), three or five channels, constant costs; also
    the call that asks for dL/dM only."""
    rng = np.random.default_rng(40 + C)
    img = rng.uniform(0, 1, (2, C, 140, 290)).astype(np.float32)
    m = rng.uniform(0, 1, (2, 1, 140, 290)).astype(np.float32)
    m[0, 0, 5:9, 200:204] = 0
    m[1, 0, 120, 7] = 0
    case = workloads.Case("bwd2d", img, m, 7.0, lam, 2)
    w = rng.uniform(-1, 1, m.shape).astype(np.float32)
    d, codes, gi, gm = _run(fgx, case, w)
    wi, wm = _oracle(case, w, codes)
    _bits_equal(gi, wi, "grad_image")
    _bits_equal(gm, wm, "grad_mask")
    _, _, gi2, gm2 = _run(fgx, case, w, need_image=False)
    assert gi2 is None
    _bits_equal(gm2, wm, "grad_mask alone")


def test_backward_3d_bit_exact(fgx):
    case = workloads.diff3d(shape=(14, 19, 23), v=10.0)
    w = case.extra["w"]
    for opts in (None, dict(tile_width=4, tile_height=3, tile_lines=2)):
        d, codes, gi, gm = _run(fgx, case, w, options=opts)
        wi, wm = _oracle(case, w, codes)
        _bits_equal(gi, wi, f"grad_image {opts}")
        _bits_equal(gm, wm, f"grad_mask {opts}")


def test_backward_3d_anisotropic_multichannel(fgx):
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (1, 2, 9, 12, 10)).astype(np.float32)
    m = rng.uniform(0, 1, (1, 1, 9, 12, 10)).astype(np.float32)
    m[0, 0, 4, 5, 6] = 0
    case = workloads.Case("3d", img, m, 4.0, 0.3, 2, (2.5, 1.0, 0.75))
    w = rng.uniform(0, 1, m.shape).astype(np.float32)
    d, codes, gi, gm = _run(fgx, case, w)
    wi, wm = _oracle(case, w, codes)
    _bits_equal(gi, wi, "grad_image")
    _bits_equal(gm, wm, "grad_mask")


@pytest.mark.parametrize("C,lam,spacing,opts", [
    (1, 1.0, (1.0, 1.0, 1.0), None),
    (2, 0.4, (2.5, 1.0, 0.75), None),
    (3, 0.0, (1.0, 2.0, 1.0), dict(max_blocks=18)),
    (1, 0.7, (1.5, 1.0, 1.0), dict(max_blocks=16)),
])
def test_backward_3d_multi_tile_bit_exact(fgx, C, lam, spacing, opts):
    """Reverse sweep over planes of several plane tiles along both in-plane
    axes (ring refreshes), three instances, waves of instances when the grid
    is capped; also the call that asks for dL/dM only."""
    rng = np.random.default_rng(60 + C)
    img = rng.uniform(0, 1, (3, C, 30, 50, 61)).astype(np.float32)
    m = rng.uniform(0, 1, (3, 1, 30, 50, 61)).astype(np.float32)
    m[0, 0, 3:6, 40:44, 10:12] = 0
    m[1, 0, 29, 0, 60] = 0
    m[2, 0, 15, 25, 30] = 0
    case = workloads.Case("bwd3d", img, m, 6.0, lam, 2, spacing)
    w = rng.uniform(-1, 1, m.shape).astype(np.float32)
    d, codes, gi, gm = _run(fgx, case, w, options=opts)
    wi, wm = _oracle(case, w, codes)
    _bits_equal(gi, wi, "grad_image")
    _bits_equal(gm, wm, "grad_mask")
    _, _, gi2, gm2 = _run(fgx, case, w, options=opts, need_image=False)
    assert gi2 is None
    _bits_equal(gm2, wm, "grad_mask alone")


@pytest.mark.parametrize("which", ["image", "mask"])
def test_backward_single_output(fgx, which):
    case = workloads.diff2d(batch=1, size=40, v=10.0)
    w = case.extra["w"]
    d, codes, gi, gm = _run(fgx, case, w, need_image=which == "image",
                            need_mask=which == "mask")
    wi, wm = _oracle(case, w, codes)
    if which == "image":
        assert gm is None
        _bits_equal(gi, wi, "grad_image")
    else:
        assert gi is None
        _bits_equal(gm, wm, "grad_mask")


def test_backward_zero_iterations(fgx):
    case = workloads.diff2d(batch=1, size=24, iterations=0)
    w = case.extra["w"]
    d, codes, gi, gm = _run(fgx, case, w)
    assert np.all(gi == 0)
    _bits_equal(gm, (np.float32(case.v) * w).astype(np.float32), "grad_mask")


def test_differentiable_configs_full_size(fgx):
    """The differentiable workloads at their stated sizes (8x512x512 2D batch,
    96x160x160 volume): gradients bit-exact to the oracle."""
    for case in (workloads.diff2d(), workloads.diff3d()):
        w = case.extra["w"]
        d, codes, gi, gm = _run(fgx, case, w)
        want_d, want_codes = oracle.gdt(case.image, case.mask, case.v, case.lam,
                                        case.iterations, spacing=case.spacing,
                                        return_codes=True, threads=THREADS)
        _bits_equal(d, want_d, "dist")
        np.testing.assert_array_equal(codes, want_codes)
        wi, wm = _oracle(case, w, codes)
        _bits_equal(gi, wi, "grad_image")
        _bits_equal(gm, wm, "grad_mask")


def test_autograd_function(fgx):
    case = workloads.diff2d(batch=2, size=48, v=10.0)
    img = torch.from_numpy(case.image).cuda().requires_grad_(True)
    m = torch.from_numpy(case.mask).cuda().requires_grad_(True)
    w = torch.from_numpy(case.extra["w"]).cuda()
    d = fgx.geodesic_autograd(img, m, case.v, case.lam, case.iterations)
    loss = (w * d).sum()
    loss.backward()
    _, codes = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                          return_codes=True)
    wi, wm = _oracle(case, case.extra["w"], codes)
    _bits_equal(img.grad.cpu().numpy(), wi, "autograd grad_image")
    _bits_equal(m.grad.cpu().numpy(), wm, "autograd grad_mask")
    # forward value equals the plain forward
    plain = fgx.geodesic2d(img.detach(), m.detach(), case.v, case.lam, case.iterations)
    _bits_equal(d.detach().cpu().numpy(), plain.cpu().numpy(), "autograd forward")


# ------------------------------------------------------- checkpointed 3D training

def _ckpt_case(C=2, lam=0.6, iterations=3, shape=(18, 33, 41)):
    rng = np.random.default_rng(77 + C)
    img = rng.uniform(0, 1, (2, C) + shape).astype(np.float32)
    m = rng.uniform(0, 1, (2, 1) + shape).astype(np.float32)
    m[0, 0, 2, 3, 4] = 0
    m[1, 0, -2, -3, -4] = 0
    w = rng.uniform(-1, 1, m.shape).astype(np.float32)
    return workloads.Case("ckpt3d", img, m, 8.0, lam, iterations, (2.0, 1.0, 0.75)), w


@pytest.mark.parametrize("interval", [1, 2, 3, 5])
@pytest.mark.parametrize("C,lam", [(2, 0.6), (1, 1.0)])
def test_checkpointed_backward_equals_oracle(fgx, interval, C, lam):
    """Forward keeping distance maps every `interval` iterations, backward
    replaying each segment: the distances equal the plain forward's and the
    gradients equal the oracle's reverse sweep bit for bit (3 iterations: 3,
    2, 1 and 1 segments)."""
    case, w = _ckpt_case(C, lam)
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    d, saved = fgx.forward_checkpoint(img, m, case.v, case.lam, case.iterations, interval,
                                      spacing=case.spacing, check=True)
    nseg = -(-case.iterations // interval)
    assert saved.shape[0] == nseg - 1
    want_d, want_codes = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                                    spacing=case.spacing, return_codes=True, threads=THREADS)
    _bits_equal(d.cpu().numpy(), want_d, "dist")
    gi, gm = fgx.backward_checkpoint(torch.from_numpy(w).cuda(), img, m, saved, case.v,
                                     case.lam, case.iterations, interval, spacing=case.spacing,
                                     check=True)
    wi, wm = _oracle(case, w, want_codes)
    _bits_equal(gi.cpu().numpy(), wi, "grad_image")
    _bits_equal(gm.cpu().numpy(), wm, "grad_mask")


def test_checkpointed_autograd_matches_codes_mode(fgx):
    """GeodesicFn with checkpoint=1 and without: same forward, same image and
    mask gradients (the differentiable 3D workload's generator, smaller)."""
    case = workloads.diff3d(shape=(20, 36, 44), v=10.0)
    w = torch.from_numpy(case.extra["w"]).cuda()
    grads = []
    for ck in (None, 1):
        img = torch.from_numpy(case.image).cuda().requires_grad_(True)
        m = torch.from_numpy(case.mask).cuda().requires_grad_(True)
        d = fgx.geodesic_autograd(img, m, case.v, case.lam, case.iterations,
                                  spacing=case.spacing, checkpoint=ck)
        (w * d).sum().backward()
        grads.append((d.detach().cpu().numpy(), img.grad.cpu().numpy(), m.grad.cpu().numpy()))
    for a, b, what in zip(grads[0], grads[1], ("dist", "grad_image", "grad_mask")):
        _bits_equal(b, a, what)


def test_backward_3d_scratch_does_not_grow_with_iterations(fgx):
    """The 3D reverse sweep keeps the adjoint of one pass application, not of
    every one: its scratch is the same for 1 and 8 iterations, and the
    checkpointed kept buffer is 4/interval bytes per voxel and iteration."""
    B, C, D, H, W = 1, 1, 64, 64, 64
    n = D * H * W
    s1 = fgx.backward_workspace_size(3, B, C, D, H, W, 1)
    s8 = fgx.backward_workspace_size(3, B, C, D, H, W, 8)
    assert s1 == s8
    assert s8 < 16 * n
    assert fgx.saved_size(3, B, D, H, W, 8) == 8 * 6 * n
    assert fgx.checkpoint_saved_size(B, D, H, W, 8, 2) == 3 * 4 * n
    assert fgx.checkpoint_saved_size(B, D, H, W, 8, 8) == 0
