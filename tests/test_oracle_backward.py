"""Pins of the oracle's reverse sweep (CPU only).

The forward transform is a composition of min and + of smooth edge costs, so
away from ties it is differentiable and its derivative follows the recorded
argmin codes.  The float64 reverse sweep is checked against float64 central
differences (h = 1e-6) of loss = sum(w * D), excluding the elements whose
perturbation changes some code (a kink of the min).
"""
import numpy as np
import pytest

import oracle
import workloads

H_FD = 1e-6


def _loss_and_codes(img, m, v, lam, its, sp, w):
    """Returns the distance map (the loss is sum(w * D)) and the codes."""
    d, codes = oracle.gdt(img, m, v, lam, its, spacing=sp, dtype=np.float64, return_codes=True)
    return d, codes


def _fd_check(img, m, v, lam, its, sp, w, check_image=True, check_mask=True, max_elems=None,
              seed=0):
    _, base_codes = _loss_and_codes(img, m, v, lam, its, sp, w)
    gi, gm = oracle.backward(w, img, base_codes, v, lam, its, spacing=sp, dtype=np.float64)
    rng = np.random.default_rng(seed)
    results = []
    for which, arr, grad in (("image", img, gi), ("mask", m, gm)):
        if (which == "image" and not check_image) or (which == "mask" and not check_mask):
            continue
        flat = np.arange(arr.size)
        if max_elems is not None and arr.size > max_elems:
            flat = rng.choice(arr.size, size=max_elems, replace=False)
        fd, an, kinks = [], [], 0
        for e in flat:
            plus = arr.copy()
            minus = arr.copy()
            plus.reshape(-1)[e] += H_FD
            minus.reshape(-1)[e] -= H_FD
            Lp, cp = _loss_and_codes(*(plus if which == "image" else img,
                                       plus if which == "mask" else m), v, lam, its, sp, w)
            Lm, cm = _loss_and_codes(*(minus if which == "image" else img,
                                       minus if which == "mask" else m), v, lam, its, sp, w)
            if not (np.array_equal(cp, base_codes) and np.array_equal(cm, base_codes)):
                kinks += 1
                continue
            # difference of the two losses summed term by term, so that terms
            # the perturbation does not reach cancel exactly
            fd.append(float(np.sum(w * (Lp - Lm))) / (2 * H_FD))
            an.append(grad.reshape(-1)[e])
        fd, an = np.array(fd), np.array(an)
        results.append((which, fd, an, kinks, len(flat)))
    return results


@pytest.mark.parametrize("lam", [0.75, 0.3])
def test_backward_2d_matches_central_differences(lam):
    case = workloads.diff2d(batch=1, size=32, v=10.0, lam=lam)
    img = case.image.astype(np.float64)
    m = case.mask.astype(np.float64)
    w = case.extra["w"].astype(np.float64)
    for which, fd, an, kinks, n in _fd_check(img, m, case.v, case.lam, case.iterations, None, w):
        assert kinks < 0.05 * n, (which, kinks)
        err = np.linalg.norm(fd - an) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-6, (which, err)
        assert np.linalg.norm(an) > 0


def test_backward_2d_multichannel_matches_central_differences():
    rng = np.random.default_rng(11)
    img = rng.uniform(0, 1, (2, 3, 14, 19))
    m = rng.uniform(0, 1, (2, 1, 14, 19))
    m[:, :, 4, 7] = 0
    w = rng.uniform(0, 1, m.shape)
    for which, fd, an, kinks, n in _fd_check(img, m, 6.0, 0.6, 2, None, w):
        assert kinks < 0.05 * n
        err = np.linalg.norm(fd - an) / np.linalg.norm(fd)
        assert err < 1e-6, (which, err)


def test_backward_3d_matches_central_differences():
    # the 16 x 16 x 16 gradient-check instance of the differentiable workload
    # (anisotropic spacing added so that the spacing terms are exercised too)
    case = workloads.diff3d(shape=(16, 16, 16), v=10.0)
    img = case.image.astype(np.float64)
    m = case.mask.astype(np.float64)
    w = case.extra["w"].astype(np.float64)
    res = _fd_check(img, m, case.v, case.lam, case.iterations, (2.5, 1.0, 1.0), w,
                    max_elems=1200)
    for which, fd, an, kinks, n in res:
        assert kinks < 0.05 * n
        err = np.linalg.norm(fd - an) / np.linalg.norm(fd)
        assert err < 1e-6, (which, err)


def test_backward_float32_close_to_float64():
    case = workloads.diff2d(batch=2, size=40)
    d32, c32 = oracle.gdt(case.image, case.mask, case.v, case.lam, 2, return_codes=True)
    w = case.extra["w"]
    gi32, gm32 = oracle.backward(w, case.image, c32, case.v, case.lam, 2)
    # same codes in float64 arithmetic
    gi64, gm64 = oracle.backward(w.astype(np.float64), case.image.astype(np.float64), c32,
                                 case.v, case.lam, 2, dtype=np.float64)
    assert np.linalg.norm(gi32 - gi64) / np.linalg.norm(gi64) < 1e-4
    assert np.linalg.norm(gm32 - gm64) / np.linalg.norm(gm64) < 1e-5


def test_backward_lambda0_has_no_image_gradient_and_mask_gradient_is_v_times_count():
    """lambda = 0: costs do not depend on I, so dL/dI = 0; dL/dM(x) = v * sum of
    w over the elements whose shortest path starts at x."""
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, (1, 1, 9, 11))
    m = np.ones((1, 1, 9, 11))
    m[0, 0, 2, 3] = 0
    w = np.ones_like(m)
    d, codes = oracle.gdt(img, m, 1e10, 0.0, 2, dtype=np.float64, return_codes=True)
    gi, gm = oracle.backward(w, img, codes, 1e10, 0.0, 2, dtype=np.float64)
    assert np.all(gi == 0)
    # every element is reached from the single seed
    assert gm[0, 0, 2, 3] == pytest.approx(1e10 * m.size)
    assert np.count_nonzero(gm) == 1


# ------------------------------------------------ lambda and v gradients

def _param_fd(img, m, v, lam, its, sp, w, which):
    """Central difference of sum(w * D) in lambda or v (float64), and whether
    the perturbation left every code unchanged."""
    def run(vv, ll):
        return oracle.gdt(img, m, vv, ll, its, spacing=sp, dtype=np.float64, return_codes=True)
    _, base = run(v, lam)
    if which == "lambda":
        (dp, cp), (dm, cm) = run(v, lam + H_FD), run(v, lam - H_FD)
    else:
        (dp, cp), (dm, cm) = run(v + H_FD * v, lam), run(v - H_FD * v, lam)
    stable = np.array_equal(cp, base) and np.array_equal(cm, base)
    h = H_FD if which == "lambda" else H_FD * v
    return float(np.sum(w * (dp - dm))) / (2 * h), stable, base


@pytest.mark.parametrize("shape,C,lam,sp", [
    ((1, 1, 24, 29), 1, 0.75, None),
    ((2, 3, 13, 17), 3, 0.4, None),
    ((1, 2, 9, 11, 10), 2, 0.6, (2.5, 1.0, 0.75)),
])
def test_param_grads_match_central_differences(shape, C, lam, sp):
    """dL/dlambda (each used edge's cost derivative (di2 - s2) / (2c) times
    the element's adjoint) and dL/dv (sum of M * G0) against float64 central
    differences of the forward."""
    rng = np.random.default_rng(sum(shape))
    img = rng.uniform(0, 1, shape)
    m = rng.uniform(0, 1, (shape[0], 1) + shape[2:])
    m.reshape(shape[0], -1)[:, 3] = 0.0
    w = rng.uniform(0, 1, m.shape)
    v = 4.0
    for which in ("lambda", "v"):
        fd, stable, codes = _param_fd(img, m, v, lam, 2, sp, w, which)
        assert stable
        lt, vt = oracle.param_terms(w, img, m, codes, v, lam, 2, spacing=sp, dtype=np.float64)
        an = float(np.sum(lt if which == "lambda" else vt))
        assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-12), (which, an, fd)
        assert abs(an) > 0


def test_param_grads_float32_terms_track_float64():
    """The float32 terms (the GPU's reference) stay close to the float64 ones."""
    case = workloads.diff2d(batch=1, size=40, v=10.0)
    d, codes = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations,
                          return_codes=True)
    g32 = oracle.param_grads(case.extra["w"], case.image, case.mask, codes, case.v, case.lam,
                             case.iterations)
    lt, vt = oracle.param_terms(case.extra["w"], case.image, case.mask, codes, case.v, case.lam,
                                case.iterations, dtype=np.float64)
    g64 = (float(np.sum(lt)), float(np.sum(vt)))
    for a, b in zip(g32, g64):
        assert abs(a - b) <= 1e-4 * abs(b), (a, b)
