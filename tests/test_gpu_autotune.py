"""The autotuner (GPU): it picks one of the candidate tile geometries by
timing them on the caller's inputs, caches the choice per shape, and every
choice gives the oracle's bits (the geometry never changes the result)."""
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
    bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
    assert bad.size == 0, f"{what}: {bad.size} of {got.size} differ"


def test_autotune_2d_picks_a_candidate_and_caches(fgx):
    case = workloads.diff2d(batch=3, size=300)
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    opts = fgx.autotune(img, m, case.v, case.lam, case.iterations)
    cands = [None] + [dict(tile_lines=k, tile_width=t) for k, t in fgx.TILE_CANDIDATES_2D[1:]]
    assert opts in cands
    assert fgx.autotune(img, m, case.v, case.lam, case.iterations) is opts  # cached
    got = fgx.geodesic2d(img, m, case.v, case.lam, case.iterations, options="auto", check=True)
    want = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations, threads=THREADS)
    _bits(got.cpu().numpy(), want, "auto options")


def test_autotune_c_abi_skips_unsupported_candidates(fgx):
    rng = np.random.default_rng(1)
    img = torch.from_numpy(rng.uniform(0, 1, (1, 1, 64, 700)).astype(np.float32)).cuda()
    m = torch.ones((1, 1, 64, 700), device="cuda")
    m[0, 0, 3, 3] = 0
    out = torch.empty_like(m)
    # the first candidate cannot hold a pass's tiles at once (max_blocks = 1)
    opts = (fgx.Options * 2)(fgx.Options(max_blocks=1, tile_width=16, tile_lines=8),
                             fgx.Options())
    ws = torch.zeros(fgx.workspace_size(2, 1, 1, 1, 64, 700), dtype=torch.uint8, device="cuda")
    best, ms = ctypes.c_int32(-1), ctypes.c_float(0)
    st = fgx.lib().fgx_autotune(2, ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), 1, 1, 1, 64, 700, None, 1e10,
                                0.5, 2, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                ctypes.cast(opts, ctypes.c_void_p), 2, 2, ctypes.byref(best),
                                ctypes.byref(ms), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fgx.OK and best.value == 1 and ms.value > 0


def test_batched_auto_options_match_plain_calls(fgx):
    cases = workloads.batched(n2d=10, n3d=2, side2d=(128, 400), side3d=(24, 40))
    dev = torch.device("cuda")
    inst = [(torch.from_numpy(c.image).to(dev), torch.from_numpy(c.mask).to(dev), c.v, c.lam,
             c.iterations, c.spacing or (1.0, 1.0, 1.0)) for c in cases]
    plan = fgx.BatchedPlan(inst, options="auto")
    # 2D and 3D instances: the tuner also chose the SM share of the 2D launch
    assert "split_sms" in plan.options
    outs = plan.run(check=True)
    for c, o in zip(cases, outs):
        want = oracle.gdt(c.image, c.mask, c.v, c.lam, c.iterations, spacing=c.spacing,
                          threads=THREADS)
        _bits(o.cpu().numpy(), want, c.name)


@pytest.mark.parametrize("shape", [(12, 14, 16), (40, 72, 64)])
def test_autotune_3d_ring_width(fgx, shape):
    """The 3D tuner picks a ring width of the plane-tile kernel; every
    candidate (the planner's choice, all passes narrow, all wide) gives the
    oracle's result bit for bit."""
    case = workloads.diff3d(shape=shape)
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    choice = fgx.autotune(img, m, case.v, case.lam, case.iterations, spacing=case.spacing)
    assert choice in (None, dict(tile_lines=4), dict(tile_lines=8))
    want = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                      spacing=case.spacing, threads=THREADS)
    for opts in (choice, dict(tile_lines=4), dict(tile_lines=8)):
        got = fgx.geodesic(img, m, case.v, case.lam, case.iterations, spacing=case.spacing,
                           options=opts, check=True)
        _bits(got.cpu().numpy(), want, f"3D ring option {opts}")
