"""rok_jvp_noalloc: the allocation-free finite-difference JVP.

Callers that cannot allocate device memory (plug-ins whose host owns every
device allocation, loops that must not synchronise the device with
cudaMalloc/cudaFree) use this entry point instead of rok_jvp; its scratch is a
static device array.  The tests call it through the C ABI twice in a row and
check each result against rok_jvp's (same kernels: bitwise equal, which is
within every tolerance the JVP tests use), on uniform grids and on Lorenz-96;
check the status word it writes for a non-finite input; check that repeated
calls leave the device's free memory unchanged; and check its refusals.

The file name sorts last so that pytest collects it after every other test:
a run that stops at the first failure has then run all the others.  Nothing
here depends on that order: each test builds its own inputs, and the file
passes alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _cases():
    from paper_1607_06834_gb300 import workloads as W
    p, y = W.lorenz96(40)
    return [W.taylor_green(64, reynolds=400.0), W.isentropic_vortex(48), (p, y)]


@pytest.mark.parametrize('rounding', ['fast', 'strict'])
def test_jvp_noalloc_matches_rok_jvp_twice(rounding):
    from paper_1607_06834_gb300 import rok
    mode = rok.ROK_ROUND_STRICT if rounding == 'strict' else rok.ROK_ROUND_FAST
    for prob, y0 in _cases():
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
            assert torch.equal(out, ref), prob.name
            assert int(status.item()) == 0
            rok.rok_jvp_noalloc(prob, y, v, fy, out, eps=2.0 ** -21, status=status, rounding=mode)
            torch.cuda.synchronize()
            assert torch.equal(out, ref_eps), prob.name


def test_jvp_noalloc_reports_a_nonfinite_result_then_recovers():
    # the status word of a call is cleared at its start: a NaN in y sets it, the
    # next call on good data reports 0 again (the shared scratch keeps no stale error)
    from paper_1607_06834_gb300 import rok
    from paper_1607_06834_gb300 import workloads as W
    prob, y0 = W.isentropic_vortex(32)
    bad = y0.copy()
    bad[0, 4, 9] = np.nan
    v = rok.state_tensor(np.random.default_rng(5).standard_normal(y0.shape))
    ctx = rok.rok_init(prob, krylov_max=2)
    y = rok.state_tensor(y0)
    fy = rok.rok_residual(ctx, y)
    out = torch.empty_like(y)
    status = torch.full((1,), -1, dtype=torch.int32, device='cuda')
    rok.rok_jvp_noalloc(prob, rok.state_tensor(bad), v, fy, out, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) != 0
    rok.rok_jvp_noalloc(prob, y, v, fy, out, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(out, rok.rok_jvp(ctx, y, v, fy=fy))


def test_jvp_noalloc_allocates_nothing():
    # after a first call (which loads the kernels and resolves the scratch
    # address), further calls leave the device's free memory where it was
    from paper_1607_06834_gb300 import rok
    prob, y0 = _cases()[0]
    ctx = rok.rok_init(prob, krylov_max=2)
    y = rok.state_tensor(y0)
    v = torch.ones_like(y) / float(np.sqrt(y.numel()))
    fy = rok.rok_residual(ctx, y)
    out = torch.empty_like(y)
    status = torch.zeros(1, dtype=torch.int32, device='cuda')
    rok.rok_jvp_noalloc(prob, y, v, fy, out, status=status)
    rok.rok_jvp_noalloc(prob, y, v, fy, out, status=status, rounding=rok.ROK_ROUND_STRICT)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        rok.rok_jvp_noalloc(prob, y, v, fy, out, status=status)
        rok.rok_jvp_noalloc(prob, y, v, fy, out, status=status, rounding=rok.ROK_ROUND_STRICT)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_jvp_noalloc_rejects_oversize_curvilinear_and_exact():
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
    small, _ = W.isentropic_vortex(2)
    d, keep = rok._desc(small, 0, rok.ROK_ROUND_FAST, jvp=rok.ROK_JVP_EXACT)
    assert rok._lib.rok_jvp_noalloc(ctypes.byref(d), p, p, p, q, 0.0, None, None) == rok.ROK_ERR_UNSUPPORTED
    # the binding checks sizes and devices before the call
    prob, y0 = W.isentropic_vortex(16)
    y = rok.state_tensor(y0)
    with pytest.raises(ValueError):
        rok.rok_jvp_noalloc(prob, y, y, y, torch.empty(10, dtype=torch.float64, device='cuda'))
    with pytest.raises(ValueError):
        rok.rok_jvp_noalloc(prob, y, y, y, torch.empty_like(y).cpu())
