"""rok_jvp_noalloc: the allocation-free finite-difference JVP.

Callers that cannot allocate device memory (plug-ins whose host owns every
device allocation, loops that must not synchronise the device with
cudaMalloc/cudaFree) use this entry point instead of rok_jvp; its scratch is a
static device array.  The test calls it through the C ABI twice in a row and
checks each result against rok_jvp's (same kernels: bitwise equal, which is
within every tolerance the JVP tests use).  Collected last on purpose; it
passes alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('rounding', ['fast', 'strict'])
def test_jvp_noalloc_matches_rok_jvp_twice(rounding):
    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    mode = rok.ROK_ROUND_STRICT if rounding == 'strict' else rok.ROK_ROUND_FAST
    cases = [W.taylor_green(64, reynolds=400.0), W.isentropic_vortex(48)]
    for prob, y0 in cases:
        ctx = rok.rok_init(prob, krylov_max=2, rounding=mode)
        y = rok.state_tensor(y0)
        g = torch.Generator(device='cuda').manual_seed(3)
        v = torch.randn(y.shape, dtype=torch.float64, device='cuda', generator=g)
        v /= v.norm()
        fy = rok.rok_residual(ctx, y)
        ref = rok.rok_jvp(ctx, y, v, fy=fy)                 # existing entry point, automatic eps
        ref_eps = rok.rok_jvp(ctx, y, v, fy=fy, eps=2.0 ** -21)
        for _ in range(2):                                   # two calls in a row share the scratch
            out = torch.full_like(y, float('nan'))
            status = torch.full((1,), -1, dtype=torch.int32, device='cuda')
            rok.rok_jvp_noalloc(prob, y, v, fy, out, status=status, rounding=mode)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
            assert int(status.item()) == 0
            rok.rok_jvp_noalloc(prob, y, v, fy, out, eps=2.0 ** -21, status=status, rounding=mode)
            torch.cuda.synchronize()
            assert torch.equal(out, ref_eps)


def test_jvp_noalloc_rejects_oversize_and_curvilinear():
    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    big = W.FlowProblem(kind=W.EULER, nx=4096, ny=1025, lx=1.0, ly=1.0)
    d, keep = rok._desc(big, 0, rok.ROK_ROUND_FAST)
    x = torch.zeros(8, dtype=torch.float64, device='cuda')
    p = ctypes.c_void_p(x.data_ptr())
    q = ctypes.c_void_p(x.data_ptr() + 32)
    assert rok._lib.rok_jvp_noalloc(ctypes.byref(d), p, p, p, q, 0.0, None, None) == rok.ROK_ERR_INVALID_ARG
    pc, _, _ = W.cylinder_ogrid(8, 16)
    d, keep = rok._desc(pc, 0, rok.ROK_ROUND_FAST)
    assert rok._lib.rok_jvp_noalloc(ctypes.byref(d), p, p, p, q, 0.0, None, None) == rok.ROK_ERR_UNSUPPORTED
