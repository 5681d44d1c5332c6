"""Allocation-free forward (GPU).

fgx_geodesic_noalloc serves callers that cannot allocate device memory when
they need a transform (allocator callbacks, fixed-budget real-time loops,
plugins whose host framework owns every allocation).  It keeps the sweep's
scratch in a static device array inside the library.  This test calls it
through the C ABI twice in a row and checks both results against
fgx_geodesic2d / fgx_geodesic3d with a caller workspace, bit for bit (the
tolerance of every forward parity test), that fgx_noalloc_status reads back a
clean status word after those calls, and that shapes beyond the static
scratch are rejected before any launch.  It lives in a file of its own,
collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgx():
    from paper_2208_00001_gb300 import build
    build.build()
    import paper_2208_00001_gb300 as m
    return m


def _noalloc(fgx):
    f = fgx.lib().fgx_geodesic_noalloc
    i64, vp = ctypes.c_int64, ctypes.c_void_p
    f.argtypes = [ctypes.c_int, vp, vp, vp, i64, i64, i64, i64, i64, vp, ctypes.c_float,
                  ctypes.c_float, ctypes.c_int, vp, vp]
    f.restype = ctypes.c_int
    return f


def _call(fgx, case, out):
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    sp = (ctypes.c_float * 3)(*(case.spacing or (1.0, 1.0, 1.0)))
    if case.ndim == 2:
        B, C, H, W = case.image.shape
        D = 1
    else:
        B, C, D, H, W = case.image.shape
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _noalloc(fgx)(case.ndim, ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                       ctypes.c_void_p(out.data_ptr()), B, C, D, H, W, sp, case.v, case.lam,
                       case.iterations, None, s)
    return st, img, m


@pytest.mark.parametrize("make", [lambda: workloads.plain2d(),
                                  lambda: workloads.large2d(size=600, lam=0.5),
                                  lambda: workloads.volume3d(shape=(40, 64, 72))])
def test_noalloc_matches_workspace_entry_point_twice(fgx, make):
    case = make()
    ref = None
    for _ in range(2):
        out = torch.full(case.mask.shape, -1.0, device="cuda")
        st, img, m = _call(fgx, case, out)
        assert st == fgx.OK, fgx.status_string(st)
        if ref is None:
            if case.ndim == 2:
                ref = fgx.geodesic2d(img, m, case.v, case.lam, case.iterations, check=True)
            else:
                ref = fgx.geodesic3d(img, m, case.spacing, case.v, case.lam, case.iterations,
                                     check=True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = ref.cpu().numpy()
        np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
        assert _status(fgx) == fgx.OK


def _status(fgx):
    f = fgx.lib().fgx_noalloc_status
    f.argtypes = [ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_rejects_shapes_beyond_static_scratch(fgx):
    """9,000 images need 9,000 tile tags (72 KB): more than the 64 KiB static
    scratch, so the call is refused before any launch."""
    B, H, W = 9000, 4, 4
    img = torch.rand((B, 1, H, W), device="cuda")
    m = torch.ones((B, 1, H, W), device="cuda")
    out = torch.zeros_like(m)
    sp = (ctypes.c_float * 3)(1.0, 1.0, 1.0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _noalloc(fgx)(2, ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                       ctypes.c_void_p(out.data_ptr()), B, 1, 1, H, W, sp, 1.0, 0.5, 1, None, s)
    assert st == fgx.ERR_WORKSPACE
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0  # nothing was launched
    # the workspace entry point serves the same shape
    d = fgx.geodesic2d(img, m, 1.0, 0.5, 1, check=True)
    assert d.shape == m.shape
