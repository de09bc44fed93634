"""GPU adaptive time stepping (embedded ROK4 estimate, DOPRI5 comparator)
against the oracle's controller, through the C ABI.

Bar: under strict rounding the GPU takes exactly the oracle's sequence of
accepted and rejected steps and ends on the same bits (the step, the error
norm and the controller are the same operations in the same order); the FMA
build ends within the tolerance the integration was run at."""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W
from tests.gpu_common import dev, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def rok():
    from paper_1607_06834_gb300 import rok as r
    return r


def _case():
    prob, y0 = W.taylor_green(24, reynolds=300.0)
    y0 = np.ascontiguousarray(y0 + 0.01 * W.random_smooth_state(prob, seed=4))
    h1 = I.dt_from_cfl(prob, y0, 1.0)
    return prob, y0, h1


@pytest.mark.parametrize('method', ['rok', 'dopri5'])
def test_adaptive_strict_matches_oracle_step_sequence(rok, method):
    prob, y0, h1 = _case()
    T, tol, M = 12 * h1, 1e-7, 8
    ctx = rok.rok_init(prob, krylov_max=M, rounding=rok.ROK_ROUND_STRICT)
    y = dev(y0)
    sys_ = core.System(prob)
    if method == 'rok':
        info = rok.rok_integrate(ctx, y, T, M, tol, tol, 2 * h1)
        yo, st = I.rok_integrate(sys_, y0, T, 2 * h1, M, tol, tol)
    else:
        info = rok.dopri5_integrate(ctx, y, T, tol, tol, 2 * h1)
        yo, st = I.dopri5_integrate(sys_, y0, T, 2 * h1, tol, tol)
    assert (info['accepted'], info['rejected']) == (st['accepted'], st['rejected']), (info, st)
    assert info['h_next'] == st['h'] and info['t'] == st['t']
    assert np.array_equal(host(y), yo), rel_l2(host(y), yo)


@pytest.mark.parametrize('method', ['rok', 'dopri5'])
def test_adaptive_fast_within_tolerance(rok, method):
    prob, y0, h1 = _case()
    T, tol, M = 12 * h1, 1e-8, 8
    ctx = rok.rok_init(prob, krylov_max=M)
    y = dev(y0)
    sys_ = core.System(prob)
    if method == 'rok':
        info = rok.rok_integrate(ctx, y, T, M, tol, tol, 2 * h1)
        yo, _ = I.rok_integrate(sys_, y0, T, 2 * h1, M, tol, tol)
    else:
        info = rok.dopri5_integrate(ctx, y, T, tol, tol, 2 * h1)
        yo, _ = I.dopri5_integrate(sys_, y0, T, 2 * h1, tol, tol)
    assert abs(info['t'] - T) <= 1e-12 * T
    assert rel_l2(host(y), yo) <= 10 * tol


def test_adaptive_invalid_options(rok):
    prob, y0, h1 = _case()
    ctx = rok.rok_init(prob, krylov_max=4)
    y = dev(y0)
    with pytest.raises(rok.RokError):
        rok.rok_integrate(ctx, y, 1.0, 4, 1e-6, 1e-6, -1.0)
    with pytest.raises(rok.RokError):
        rok.dopri5_integrate(ctx, y, 1.0, 0.0, 0.0, h1)
    with pytest.raises(rok.RokError) as e:
        rok.dopri5_integrate(ctx, y, 100.0, 1e-6, 1e-6, h1, max_steps=3)
    assert e.value.status == rok.ROK_ERR_NOT_CONVERGED
