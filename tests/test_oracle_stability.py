"""Why ROK4 has a stability ceiling on the stretched O-grid (Sec. 2.2.2; the
paper lists ROK as conditionally stable in the table of Sec. 3.1).

Eq. ROK is the W-method with A = V H V^T: on the Krylov space K_M(J, f(y_n))
it is the implicit Rosenbrock step, and on its complement the stages reduce to
the explicit (alpha, b) part, which here is classical RK4.  A mode of J with
h lambda outside the RK4 stability region is therefore amplified by
|R_RK4(h lambda)| per step unless the Krylov space captures it, and at large
CFL that factor reaches (h |lambda|)^4 / 24.  On a small O-grid with the
cylinder's wall spacing (8 x 16 cells, N = 512, exact Jacobian at the
impulsive start) the linearised step y' = J y shows it: the smallest Krylov
dimension that keeps ROK4 from outgrowing the exact solution rises with the
CFL number, 2 at CFL 10 (48 decaying modes outside the RK4 region), 8 at
CFL 30 (96) and 32 at CFL 100 (112 modes, max |R| ~ 3e6); one step below
each, the iteration blows up or grows well beyond the exact solution.
These tests run the oracle's ROK4 step on that linear system."""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W


def _rk4_r(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


@pytest.fixture(scope='module')
def linear_ogrid():
    prob, y0, _ = W.cylinder_ogrid(8, 16)
    N = y0.size
    J = np.empty((N, N))
    for c in range(N):
        v = np.zeros(N)
        v[c] = 1.0
        J[:, c] = core.jvp_exact(prob, y0, v.reshape(y0.shape)).ravel()
    lam = np.linalg.eigvals(J)

    class Linear:
        shape = (N,)
        jac = J

        def f(self, y):
            return J @ y

        def jvp(self, y, v, f0, eps):
            return J @ v
    return prob, y0, lam, Linear()


def _outside(h, lam):
    """Eigenvalues whose exact modes decay but whose RK4 factor exceeds 1."""
    return (lam.real < 0.0) & (np.abs(_rk4_r(h * lam)) > 1.0 + 1e-12)


def _growth(sys_, h, M, steps):
    x0 = np.random.default_rng(0).standard_normal(sys_.shape)
    x = x0.copy()
    for _ in range(steps):
        x = I.rok_step(sys_, x, h, M)
        g = np.linalg.norm(x) / np.linalg.norm(x0)
        if not np.isfinite(g) or g > 1e6:
            return np.inf
    return g


def _exact_growth(J, t):
    from scipy.linalg import expm
    x0 = np.random.default_rng(0).standard_normal(J.shape[0])
    return np.linalg.norm(expm(J * t) @ x0) / np.linalg.norm(x0)


def test_the_jacobian_is_stiff(linear_ogrid):
    prob, y0, lam, _ = linear_ogrid
    # the impulsive start is not an equilibrium: a few slow modes grow (rate ~4,
    # a few per cent over the integrations below); the stiff part, |lambda| up
    # to ~8e5, is damped
    assert lam.real.max() < 1e-5 * np.abs(lam).max()
    h100 = I.dt_from_cfl(prob, y0, 100.0)
    out = _outside(h100, lam)
    print('\n[stability] 8x16 O-grid: %d eigenvalues, %d outside the RK4 region at CFL 100, max |R| %.2g'
          % (lam.size, out.sum(), np.abs(_rk4_r(h100 * lam)).max()))
    assert out.sum() > 64 and np.abs(_rk4_r(h100 * lam)).max() > 1e6
    assert not _outside(I.dt_from_cfl(prob, y0, 1.0), lam).any()


@pytest.mark.parametrize('cfl, steps, grows, holds', [(10.0, 30, 1, 2), (30.0, 30, 4, 8), (100.0, 60, 16, 32)])
def test_rok4_needs_the_growing_modes_in_its_krylov_space(linear_ogrid, cfl, steps, grows, holds):
    prob, y0, lam, sys_ = linear_ogrid
    h = I.dt_from_cfl(prob, y0, cfl)
    exact = _exact_growth(sys_.jac, steps * h)
    g_small = _growth(sys_, h, grows, steps)
    print('\n[stability] CFL %g: %d eigenvalues outside the RK4 region; over %d steps the exact solution '
          'grows %.3g x, ROK4 with M = %d %.3g x' % (cfl, _outside(h, lam).sum(), steps, exact, grows, g_small))
    assert g_small > 1.3 * exact
    if holds is not None:
        g = _growth(sys_, h, holds, steps)
        print('[stability]   M = %d: %.3g x' % (holds, g))
        assert g <= 1.1 * max(exact, 1.0)
