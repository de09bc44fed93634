"""Arnoldi breakdown (Sec. 2.2.2: the process stops when h_{j+1,j} vanishes)
inside the persistent Gram-Schmidt kernels, against the CPU oracle.

Lorenz-96 (appendix problem) is invariant under a shift of its index, and its
residual and FD-JVP evaluate the same formula at every index, so from a state
of period p (n = 20) every Krylov vector is exactly p-periodic: the Krylov
space has dimension p and column j = p - 1 breaks down (w is rounding noise
after its projections).  p = 5 ends the column on a single-vector pass and
p = 4 on a two-vector pass of the FMA build's column kernel.  (p = 3 is
degenerate: the advection term vanishes for period 3, J = -I on the
subspace, and the Krylov vectors after the first are FD noise.)  Both builds
must stop at M_eff = p like the oracle, with an orthonormal basis; the strict
build gives the oracle's V and H and ROK4 step bit for bit, the FMA build
agrees to the FD-JVP noise (the quotient amplifies a last-bit difference of f
by 1/eps, eps ~ 6e-8 here).
"""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W
from tests.gpu_common import dev, host

pytestmark = pytest.mark.gpu

M = 8


@pytest.fixture(scope='module')
def rok():
    from paper_1607_06834_gb300 import rok as r
    return r


def _periodic_state(period, n=20):
    prob, y = W.lorenz96(n, seed=3)
    return prob, np.ascontiguousarray(np.tile(y[:period], n // period))


@pytest.mark.parametrize('period', [4, 5])
@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_arnoldi_breaks_down_at_the_krylov_dimension(rok, period, mode):
    prob, y = _periodic_state(period)
    sys_ = core.System(prob)
    eps = I.fd_eps(I.norm(y))
    Vo, Ho, meo = I.arnoldi(sys_, y, sys_.f(y), M, eps)
    assert meo == period
    ctx = rok.rok_init(prob, krylov_max=M, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    V, H, me = rok.rok_arnoldi(ctx, dev(y), M)
    assert me == period
    V, H = host(V), host(H)[:me, :me]
    assert np.abs(V @ V.T - np.eye(me)).max() <= 1e-13
    if mode == 'strict':
        assert np.array_equal(V, Vo) and np.array_equal(H, Ho)
    else:
        assert np.abs(H - Ho).max() <= 1e-6 * np.abs(Ho).max()
        assert np.abs(V - Vo).max() <= 1e-6


@pytest.mark.parametrize('period', [4, 5])
@pytest.mark.parametrize('mode', ['strict', 'fast'])
def test_rok_step_with_breakdown(rok, period, mode):
    prob, y0 = _periodic_state(period)
    h = 0.01
    yo = I.rok_step(core.System(prob), y0, h, M)
    ctx = rok.rok_init(prob, krylov_max=M, rounding=getattr(rok, 'ROK_ROUND_' + mode.upper()))
    y = dev(y0)
    info = rok.rok_step(ctx, y, h, M, info=True)
    assert info['m_eff'] == period
    y = host(y)
    if mode == 'strict':
        assert np.array_equal(y, yo)
    else:
        assert np.abs(y - yo).max() <= 1e-9 * np.abs(yo).max()
    # the step stays in the invariant subspace
    assert np.array_equal(y, np.tile(y[:period], 20 // period))

