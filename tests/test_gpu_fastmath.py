"""Fast-math variant of the forward (GPU): edge costs by a fused multiply-add
and the approximate square root.  Every forward configuration stays within
1e-5 relative of the oracle (a minimum over paths moves by at most the
relative error of its step costs, about 2^-22, plus summation rounding);
where the general cost formula applies the results must differ from the
exact ones somewhere (the option is not ignored), and where it does not
apply (lambda = 0; lambda = 1 with one channel) they stay bit-exact."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
RTOL = 1e-5


@pytest.fixture(scope="module")
def fgx():
    from paper_2208_00001_gb300 import build
    build.build()
    import paper_2208_00001_gb300 as m
    return m


def _fast(fgx, case, extra=None):
    opts = dict(fast_math=1, **(extra or {}))
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    return fgx.geodesic(img, m, case.v, case.lam, case.iterations, spacing=case.spacing,
                        options=opts, check=True).cpu().numpy()


def _check(got, want, general):
    assert got.shape == want.shape
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    bound = RTOL * np.abs(want.astype(np.float64))
    assert np.all(err <= bound), f"max relative error {np.max(err / np.maximum(bound / RTOL, 1e-30)):.3g}"
    differs = np.any(got.view(np.uint32) != want.view(np.uint32))
    assert differs == general, "fast math applied where it should not, or not at all"


CONFIGS = [
    ("2D plain 256", lambda: workloads.plain2d(), False),
    ("2D large lambda=0.5", lambda: workloads.large2d(lam=0.5), True),
    ("2D large lambda=1 (3 channels)", lambda: workloads.large2d(lam=1.0), True),
    ("2D large lambda=0", lambda: workloads.large2d(lam=0.0), False),
    ("3D volume", lambda: workloads.volume3d(), False),
    ("differentiable 2D", lambda: workloads.diff2d(), True),
    ("differentiable 3D", lambda: workloads.diff3d(), True),
]


@pytest.mark.parametrize("name,make,general", CONFIGS, ids=[c[0] for c in CONFIGS])
def test_fast_math_within_tolerance(fgx, name, make, general):
    case = make()
    want = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                      spacing=case.spacing, threads=THREADS)
    _check(_fast(fgx, case), want, general)


@pytest.mark.parametrize("ndim", [2, 3])
def test_fast_math_tiled_engine_and_batched(fgx, ndim):
    rng = np.random.default_rng(90 + ndim)
    shape = (70, 90) if ndim == 2 else (17, 30, 26)
    case = workloads.random_case(rng, ndim, shape, channels=2, lam=0.6, iterations=2, soft=True,
                                 v=30.0, spacing=None if ndim == 2 else (1.5, 1.0, 1.0))
    want = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                      spacing=case.spacing, threads=THREADS)
    tiles = dict(tile_width=8, tile_lines=3) if ndim == 2 else dict(tile_width=6,
                                                                    tile_height=5, tile_lines=2)
    _check(_fast(fgx, case, tiles), want, True)
    outs = fgx.geodesic_batched([(torch.from_numpy(case.image).cuda(),
                                  torch.from_numpy(case.mask).cuda(), case.v, case.lam,
                                  case.iterations, case.spacing or (1.0, 1.0, 1.0))],
                                options=dict(fast_math=1), check=True)
    _check(outs[0].cpu().numpy(), want, True)


def test_training_forward_ignores_fast_math(fgx):
    """Recorded codes come from the exact costs: the training forward with the
    option is bit-exact to the oracle, codes included."""
    case = workloads.diff3d(shape=(20, 36, 44), v=10.0)
    img = torch.from_numpy(case.image).cuda()
    m = torch.from_numpy(case.mask).cuda()
    d, saved = fgx.forward_train(img, m, case.v, case.lam, case.iterations,
                                 spacing=case.spacing, options=dict(fast_math=1), check=True)
    want, codes = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                             spacing=case.spacing, return_codes=True, threads=THREADS)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), want.view(np.uint32))
    np.testing.assert_array_equal(saved.cpu().numpy(), codes)
