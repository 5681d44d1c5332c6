"""Batched launch of uneven instances (GPU).

One prepared plan computes every instance of a mixed 2D/3D list (the 2D line
chains and the 3D plane tiles as two persistent launches side by side, or
one after the other); each result must equal the oracle's bit for bit and the
plain single-instance call bit for bit, also when instances are spread over
several waves, for every SM share, and when the prepared launch is replayed
or captured in a CUDA graph.
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


def _bits(a, b, what):
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    assert a.shape == b.shape, what
    bad = np.flatnonzero(a.view(np.uint32) != b.view(np.uint32))
    assert bad.size == 0, f"{what}: {bad.size} of {a.size} differ"


def _to_gpu(cases):
    out = []
    for c in cases:
        out.append((torch.from_numpy(c.image).cuda(), torch.from_numpy(c.mask).cuda(), c.v,
                    c.lam, c.iterations, c.spacing or (1.0, 1.0, 1.0)))
    return out


def _small_mixed(seed=0):
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(9):
        if i % 3 == 2:
            shp = tuple(int(x) for x in rng.integers(5, 22, size=3))
            sp = tuple(float(x) for x in rng.uniform(0.5, 2.5, size=3))
            cases.append(workloads.random_case(rng, 3, shp, channels=int(rng.integers(1, 3)),
                                               lam=[0.0, 1.0, 0.6][i % 3], iterations=2,
                                               soft=True, v=9.0, spacing=sp))
        else:
            shp = tuple(int(x) for x in rng.integers(3, 200, size=2))
            cases.append(workloads.random_case(rng, 2, shp, channels=int(rng.integers(1, 4)),
                                               lam=[0.0, 0.5, 1.0][i % 3],
                                               iterations=int(rng.integers(1, 4))))
    return cases


@pytest.mark.parametrize("opts", [None, dict(max_blocks=24, tile_width=16, tile_lines=4),
                                  dict(max_blocks=24, tile_width=16, tile_lines=4, tile_height=8)])
def test_batched_small_mixed_bit_exact(fgx, opts):
    cases = _small_mixed()
    outs = fgx.geodesic_batched(_to_gpu(cases), options=opts, check=True)
    for c, o in zip(cases, outs):
        want = oracle.gdt(c.image, c.mask, c.v, c.lam, c.iterations, spacing=c.spacing,
                          threads=THREADS)
        _bits(o.cpu().numpy(), want, c.name)


def test_batched_config_matches_plain_calls(fgx):
    """The batched workload (64 2D images, sides 128..1024, and 16 volumes,
    sides 64..192): one plan equals 80 plain calls and the oracle, bit for
    bit, on every instance."""
    cases = workloads.batched()
    gpu = _to_gpu(cases)
    plan = fgx.BatchedPlan(gpu)
    outs = plan.run(check=True)
    for k, (c, g, o) in enumerate(zip(cases, gpu, outs)):
        plain = fgx.geodesic(g[0], g[1], c.v, c.lam, c.iterations, spacing=c.spacing, check=True)
        _bits(o.cpu().numpy(), plain.cpu().numpy(), c.name)
    for k, c in enumerate(cases):
        want = oracle.gdt(c.image, c.mask, c.v, c.lam, c.iterations, spacing=c.spacing,
                          threads=THREADS)
        _bits(outs[k].cpu().numpy(), want, c.name + " vs oracle")


@pytest.mark.parametrize("split", [-1, 0, 1, 7, 10_000])
def test_batched_concurrent_launches(fgx, split):
    """A batch with 2D and 3D instances runs its line-chain and plane-tile
    launches at the same time on disjoint SM shares (split_sms > 0 sets the
    2D launch's share, clamped so that the largest instance of each launch
    has its tiles resident; 0 estimates it; -1 runs them one after the
    other): every share gives the oracle's results bit for bit, also on
    replay."""
    cases = _small_mixed(seed=5)
    plan = fgx.BatchedPlan(_to_gpu(cases), options=dict(split_sms=split))
    p = plan.plan
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    assert p.n2d > 0 and p.n3d > 0
    assert p.concurrent == (0 if split == -1 else 1)
    if p.concurrent:
        assert p.grid2d + p.grid3d <= sms
        if split == 10_000:
            assert p.grid3d == 1
    for rep in range(2):
        for o in plan.outputs:
            o.fill_(-1.0)
        outs = plan.run(check=True)
        for c, o in zip(cases, outs):
            want = oracle.gdt(c.image, c.mask, c.v, c.lam, c.iterations, spacing=c.spacing,
                              threads=THREADS)
            _bits(o.cpu().numpy(), want, f"{c.name} split {split} run {rep}")


def test_batched_replay_and_graph_capture(fgx):
    cases = _small_mixed(seed=3)
    plan = fgx.BatchedPlan(_to_gpu(cases))
    first = [o.clone() for o in plan.run(check=True)]
    for o in plan.outputs:
        o.fill_(-1.0)
    plan.run(check=True)
    for a, b in zip(first, plan.outputs):
        _bits(a.cpu().numpy(), b.cpu().numpy(), "replay")
    # the run step captured in a CUDA graph
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run()
        torch.cuda.synchronize()
        for o in plan.outputs:
            o.fill_(-1.0)
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert fgx.workspace_status(plan.workspace) == 0
    for a, b in zip(first, plan.outputs):
        _bits(a.cpu().numpy(), b.cpu().numpy(), "graph replay")


def test_batched_empty_and_errors(fgx):
    assert fgx.geodesic_batched([]) == []
    img = torch.rand((1, 1, 8, 8), device="cuda")
    m = torch.ones((1, 1, 8, 8), device="cuda")
    with pytest.raises(fgx.FgxError):
        fgx.geodesic_batched([(img, m, 1.0, 1.5, 2, None)])  # lambda > 1
    with pytest.raises(fgx.FgxError):
        fgx.geodesic_batched([(img, m, -1.0, 0.5, 2, None)])  # v <= 0
    L = fgx.lib()
    arr = (fgx.Instance * 1)()
    host = torch.zeros((1, 1, 8, 8))
    arr[0] = fgx.Instance(2, 1, 1, 8, 8, host.data_ptr(), m.data_ptr(), m.data_ptr(),
                          (ctypes.c_float * 3)(1, 1, 1), 1.0, 0.5, 1)
    ws = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    st = L.fgx_geodesic_batched(ctypes.byref(arr), 1, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fgx.ERR_NOT_DEVICE_PTR
