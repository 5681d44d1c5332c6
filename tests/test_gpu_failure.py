"""Failure detection without a GPU fault (GPU): the library's bounded wait on
a tag that nothing writes gives up after its limit, records FGX_ERR_TIMEOUT in
the workspace status word, and leaves the context usable."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgx():
    from paper_2208_00001_gb300 import build
    build.build()
    import paper_2208_00001_gb300 as m
    return m


def test_bounded_wait_reports_timeout_and_context_stays_usable(fgx):
    L = fgx.lib()
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert L.fgx_probe_wait_timeout(ctypes.c_void_p(ws.data_ptr()), ws.numel(), 50, s) == fgx.OK
    assert fgx.workspace_status(ws) == fgx.ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.045
    # argument checks
    assert L.fgx_probe_wait_timeout(ctypes.c_void_p(ws.data_ptr()), 16, 50, s) == \
        fgx.ERR_WORKSPACE
    assert L.fgx_probe_wait_timeout(ctypes.c_void_p(ws.data_ptr()), ws.numel(), 0, s) == \
        fgx.ERR_ARG
    # the same context still computes exact transforms
    case = workloads.plain2d(size=64)
    d = fgx.geodesic2d(torch.from_numpy(case.image).cuda(), torch.from_numpy(case.mask).cuda(),
                       case.v, case.lam, case.iterations, check=True)
    want = oracle.gdt(case.image, case.mask, case.v, case.lam, case.iterations)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), want.view(np.uint32))
