"""Gradients with respect to lambda and v (GPU) against the oracle.

The per-element terms (float32, fixed operation order) must equal the
oracle's bit for bit; the two sums are float64 over the same terms in
another order, so they must agree within the bound of two float64
summations: |a - b| <= 2 (n - 1) 2^-53 sum |t|.
"""
import os

import numpy as np
import pytest
import torch

import oracle

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


def _sum_close(got, terms, what):
    t = terms.astype(np.float64).ravel()
    want = float(np.sum(t))
    bound = 2 * max(t.size - 1, 1) * 2.0 ** -53 * float(np.sum(np.abs(t)))
    assert abs(float(got) - want) <= bound, (what, float(got), want, bound)


@pytest.mark.parametrize("shape,lam,its,spacing", [
    ((2, 2, 140, 290), 0.75, 2, None),
    ((1, 1, 64, 64), 0.3, 3, None),
    ((2, 1, 30, 50, 61), 0.6, 2, (2.5, 1.0, 0.75)),
    ((1, 3, 20, 24, 28), 0.75, 1, (1.0, 1.0, 1.0)),
])
def test_param_grads_match_oracle(fgx, shape, lam, its, spacing):
    rng = np.random.default_rng(sum(shape) + its)
    img = rng.uniform(0, 1, shape).astype(np.float32)
    m = rng.uniform(0, 1, (shape[0], 1) + shape[2:]).astype(np.float32)
    m.reshape(shape[0], -1)[:, 5] = 0.0
    w = rng.uniform(-1, 1, m.shape).astype(np.float32)
    v = 6.0
    ti, tm, tw = (torch.from_numpy(x).cuda() for x in (img, m, w))
    d, saved = fgx.forward_train(ti, tm, v, lam, its, spacing=spacing, check=True)
    codes = saved.cpu().numpy()
    want_lt, want_vt = oracle.param_terms(w, img, m, codes, v, lam, its, spacing=spacing)
    gl, gv, lt, vt, gi, gm = fgx.backward_params(tw, ti, tm, saved, v, lam, its,
                                                 spacing=spacing, need_image=True,
                                                 need_mask=True, check=True)
    _bits(lt.cpu().numpy(), want_lt, "lambda terms")
    _bits(vt.cpu().numpy(), want_vt, "v terms")
    _sum_close(gl.item(), want_lt, "dL/dlambda")
    _sum_close(gv.item(), want_vt, "dL/dv")
    wi, wm = oracle.backward(w, img, codes, v, lam, its, spacing=spacing)
    _bits(gi.cpu().numpy(), wi, "grad_image")
    _bits(gm.cpu().numpy(), wm, "grad_mask")
    assert abs(gl.item()) > 0 and abs(gv.item()) > 0
    # the sums are the same bits on every run
    gl2, gv2, *_ = fgx.backward_params(tw, ti, tm, saved, v, lam, its, spacing=spacing)
    assert gl2.item() == gl.item() and gv2.item() == gv.item()


def test_param_grads_zero_iterations(fgx):
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, (1, 1, 33, 47)).astype(np.float32)
    m = rng.uniform(0, 1, (1, 1, 33, 47)).astype(np.float32)
    w = rng.uniform(-1, 1, m.shape).astype(np.float32)
    ti, tm, tw = (torch.from_numpy(x).cuda() for x in (img, m, w))
    d, saved = fgx.forward_train(ti, tm, 3.0, 0.5, 0)
    gl, gv, lt, vt, _, _ = fgx.backward_params(tw, ti, tm, saved, 3.0, 0.5, 0, check=True)
    assert gl.item() == 0.0 and torch.all(lt == 0)
    _bits(vt.cpu().numpy(), (m * w).astype(np.float32), "v terms")
    _sum_close(gv.item(), (m * w).astype(np.float32), "dL/dv")


def test_param_grads_refuse_3d_tile_options(fgx):
    rng = np.random.default_rng(3)
    img = torch.from_numpy(rng.uniform(0, 1, (1, 1, 12, 14, 16)).astype(np.float32)).cuda()
    m = torch.ones((1, 1, 12, 14, 16), device="cuda")
    m[0, 0, 5, 5, 5] = 0
    opts = dict(tile_width=8, tile_height=4, tile_lines=3)
    d, saved = fgx.forward_train(img, m, 2.0, 0.5, 1, spacing=(1.0, 1.0, 1.0), options=opts)
    with pytest.raises(fgx.FgxError):
        fgx.backward_params(torch.ones_like(m), img, m, saved, 2.0, 0.5, 1,
                            spacing=(1.0, 1.0, 1.0), options=opts)


def test_param_grads_2d_tile_options(fgx):
    """The 2D reverse sweep honours tile options and still gives the terms."""
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, (1, 2, 40, 70)).astype(np.float32)
    m = np.ones((1, 1, 40, 70), np.float32)
    m[0, 0, 5, 5] = 0
    w = rng.uniform(0, 1, m.shape).astype(np.float32)
    opts = dict(tile_width=16, tile_lines=8)
    ti, tm, tw = (torch.from_numpy(x).cuda() for x in (img, m, w))
    d, saved = fgx.forward_train(ti, tm, 2.0, 0.5, 2, options=opts)
    gl, gv, lt, vt, _, _ = fgx.backward_params(tw, ti, tm, saved, 2.0, 0.5, 2, options=opts,
                                               check=True)
    want_lt, want_vt = oracle.param_terms(w, img, m, saved.cpu().numpy(), 2.0, 0.5, 2)
    _bits(lt.cpu().numpy(), want_lt, "lambda terms")
    _bits(vt.cpu().numpy(), want_vt, "v terms")


def test_autograd_lambda_and_v(fgx):
    """GeodesicFn returns dL/dv and dL/dlambda for tensor parameters (float64
    sums cast to the parameters' dtype) next to the image and mask gradients."""
    rng = np.random.default_rng(9)
    img = rng.uniform(0, 1, (1, 1, 48, 60)).astype(np.float32)
    m = rng.uniform(0, 1, (1, 1, 48, 60)).astype(np.float32)
    m[0, 0, 10, 10] = 0
    w = rng.uniform(0, 1, m.shape).astype(np.float32)
    ti = torch.from_numpy(img).cuda().requires_grad_(True)
    tm = torch.from_numpy(m).cuda().requires_grad_(True)
    tv = torch.tensor(5.0, dtype=torch.float64, device="cuda", requires_grad=True)
    tl = torch.tensor(0.6, dtype=torch.float64, device="cuda", requires_grad=True)
    d = fgx.geodesic_autograd(ti, tm, tv, tl, 2)
    (torch.from_numpy(w).cuda() * d).sum().backward()
    _, codes = oracle.gdt(img, m, 5.0, np.float32(0.6), 2, return_codes=True)
    lt, vt = oracle.param_terms(w, img, m, codes, 5.0, np.float32(0.6), 2)
    _sum_close(tl.grad.item(), lt, "autograd dL/dlambda")
    _sum_close(tv.grad.item(), vt, "autograd dL/dv")
    wi, wm = oracle.backward(w, img, codes, 5.0, np.float32(0.6), 2)
    _bits(ti.grad.cpu().numpy(), wi, "autograd grad_image")
    _bits(tm.grad.cpu().numpy(), wm, "autograd grad_mask")


def test_derived_entries_on_empty_inputs(fgx):
    img = torch.empty((0, 1, 8, 8), device="cuda")
    m = torch.empty((0, 1, 8, 8), device="cuda")
    assert fgx.signed_geodesic(img, m, 1.0, 0.5, 2).numel() == 0
    assert fgx.euclidean(m, 1.0, 2).numel() == 0
    d, saved = fgx.forward_train(img, m, 1.0, 0.5, 2)
    gl, gv, lt, vt, _, _ = fgx.backward_params(torch.empty_like(m), img, m, saved, 1.0, 0.5, 2)
    assert gl.item() == 0.0 and gv.item() == 0.0
