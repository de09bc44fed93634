"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) against quantities
fixed independently of it: the dense Jacobian built column by column by the
complex step, the exact affinity of the residual in the viscosity, and the
complex-step derivative of the oracle's own ROK4 step map (the analytic
continuation of integrators.rok_step, no difference quotients of the map)."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W


def _cases():
    p, y = W.taylor_green(10, reynolds=300.0)
    p = W.FlowProblem(**{**p.__dict__, 'ny': 12, 'ly': p.ly * 12 / 10})
    y = np.ascontiguousarray(np.concatenate([y, y[:, :2]], axis=1) + 0.01 * W.random_smooth_state(p, seed=3))
    out = [('ns-periodic-10x12', p, y)]
    p, y = W.isentropic_vortex(8)
    out.append(('euler-8x8', p, y))
    p4, y4, _ = W.cylinder_ogrid(6, 16)
    out.append(('ogrid-6x16', p4, np.ascontiguousarray(y4 + 0.02 * W.random_smooth_state(p4, seed=2))))
    # walls on three sides and a far field, Sutherland's law (corner ghosts
    # mirrored across two walls)
    xw, yw = W.perturbed_box_grid(7, 6, 2.0, 1.8, amp=0.3, seed=5)
    p6 = W.FlowProblem(kind=W.NAVIER_STOKES, nx=7, ny=6, xv=xw, yv=yw, mu=0.02, q_inf=(1.0, 0.3, 0.1, 2.5),
                       bc=(W.WALL, W.FARFIELD, W.WALL, W.WALL), sutherland_s=0.4, t_ref=0.5)
    out.append(('box-walls-7x6', p6, W.random_smooth_state(p6, seed=8, amp=0.08)))
    p5, y5 = W.lorenz96(12)
    out.append(('lorenz12', p5, y5))
    return out


def _dense_jacobian(prob, y):
    N = y.size
    J = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        J[:, c] = core.jvp_exact(prob, y, e.reshape(y.shape)).ravel()
    return J


@pytest.mark.parametrize('name,prob,y', _cases(), ids=[c[0] for c in _cases()])
def test_residual_vjp_is_the_dense_jacobian_transpose(name, prob, y):
    u = np.random.default_rng(1).standard_normal(y.shape)
    J = _dense_jacobian(prob, y)
    ref = (J.T @ u.ravel()).reshape(y.shape)
    got = A.residual_vjp(prob, y, u)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(got - ref).max()


def test_residual_vjp_adjoint_identity_larger_grids():
    # <u, J v> = <J^T u, v> with J v the complex-step JVP (periodic sides that
    # 5 does not divide, a Sutherland case, a curvilinear grid)
    rng = np.random.default_rng(4)
    p, y = W.taylor_green(24, reynolds=500.0)
    p = W.FlowProblem(**{**p.__dict__, 'sutherland_s': 0.4, 't_ref': 1.0 / 1.4})
    xv, yv = W.perturbed_box_grid(14, 18, 2.0, 1.8, amp=0.3, seed=4)
    p3 = W.FlowProblem(kind=W.NAVIER_STOKES, nx=14, ny=18, xv=xv, yv=yv, mu=0.02)
    for prob, yy in ((p, y), (p3, W.random_smooth_state(p3, seed=7, amp=0.08))):
        u = rng.standard_normal(yy.shape)
        v = rng.standard_normal(yy.shape)
        lhs = np.sum(u * core.jvp_exact(prob, yy, v))
        rhs = np.sum(A.residual_vjp(prob, yy, u) * v)
        assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(u * core.jvp_exact(prob, yy, np.abs(v)))), (lhs, rhs)


@pytest.mark.parametrize('sutherland', [False, True])
def test_residual_is_affine_in_the_viscosity(sutherland):
    # constant viscosity, and Sutherland's law with mu the viscosity at t_ref
    # (a temperature field away from t_ref, so that g(T) != 1 matters)
    p, y = W.taylor_green(16, reynolds=200.0)
    if sutherland:
        p = W.FlowProblem(**{**p.__dict__, 'sutherland_s': 0.4, 't_ref': 0.5})
    d = A.residual_dmu(p, y)
    pa = W.FlowProblem(**{**p.__dict__, 'mu': 0.05})
    pb = W.FlowProblem(**{**p.__dict__, 'mu': 0.01})
    diff = core.residual(pa, y) - core.residual(pb, y)
    assert np.abs(diff - 0.04 * d).max() <= 1e-11 * np.abs(core.residual(pa, y)).max()
    assert np.abs(d).max() > 0.0
    if sutherland:
        # the derivative differs from the constant-viscosity one (g(T) enters)
        pc = W.FlowProblem(**{**p.__dict__, 'sutherland_s': 0.0})
        assert np.abs(d - A.residual_dmu(pc, y)).max() > 1e-3 * np.abs(d).max()


def _step_derivative_cs(prob, y, h, M, d, c):
    """<c, dPhi(y)/dy d> by the complex step through integrators.rok_step."""
    yc = I.rok_step(core.System(prob), y + 1e-30j * d, h, M)
    return float(np.sum(c * yc.imag) / 1e-30)


@pytest.mark.parametrize('M', [0, 3, 8])
@pytest.mark.parametrize('case', ['tgv', 'tgv-sutherland', 'vortex', 'ogrid', 'lorenz'])
def test_rok_step_vjp_matches_complex_step(case, M):
    if case.startswith('tgv'):
        prob, y = W.taylor_green(16, reynolds=400.0)
        if case == 'tgv-sutherland':
            prob = W.FlowProblem(**{**prob.__dict__, 'sutherland_s': 0.4, 't_ref': 0.5})
        y = np.ascontiguousarray(y + 0.01 * W.random_smooth_state(prob, seed=5))
    elif case == 'ogrid':
        # curvilinear, wall and far field, Sutherland's law
        prob, y, _ = W.cylinder_ogrid(6, 16)
        y = np.ascontiguousarray(y + 0.02 * W.random_smooth_state(prob, seed=2))
    elif case == 'lorenz':
        prob, y = W.lorenz96(12)
    else:
        prob, y = W.isentropic_vortex(16)
    # (CFL 1 on the O-grid: the M = 0 step is explicit RK4 there)
    h = 0.01 if case == 'lorenz' else I.dt_from_cfl(prob, y, 1.0 if case == 'ogrid' else 5.0)
    rng = np.random.default_rng(M)
    d = rng.standard_normal(y.shape)
    c = rng.standard_normal(y.shape)
    fwd = _step_derivative_cs(prob, y, h, M, d, c)
    yb, _ = A.rok_step_vjp(prob, y, h, M, c)
    rev = float(np.sum(yb * d))
    # both are the exact derivative of the same discrete map; they differ by the
    # rounding of the FD quotients' derivatives (relative u / eps ~ 1e-8)
    assert abs(fwd - rev) <= 1e-6 * abs(fwd), (fwd, rev)


def test_rok_step_vjp_state_adjoint_reproduces_the_step_for_M0():
    # M = 0: the step is RK4 on f, its reverse uses residual_vjp only
    prob, y = W.taylor_green(12, reynolds=300.0)
    h = I.dt_from_cfl(prob, y, 1.0)
    rng = np.random.default_rng(9)
    d, c = rng.standard_normal(y.shape), rng.standard_normal(y.shape)
    yb, _ = A.rok_step_vjp(prob, y, h, 0, c)
    fd = (np.sum(c * I.rok_step(core.System(prob), y + 1e-6 * d, h, 0))
          - np.sum(c * I.rok_step(core.System(prob), y - 1e-6 * d, h, 0))) / 2e-6
    assert abs(np.sum(yb * d) - fd) <= 1e-7 * abs(fd)


@pytest.mark.parametrize('M,sutherland', [(0, False), (2, False), (6, False), (2, True)])
def test_rok_step_vjp_viscosity_matches_complex_step(M, sutherland):
    # f is affine in mu (pinned above), so f(y; mu + i d) = f(y; mu) + i d df/dmu(y)
    # continues the residual analytically in mu; the complex step through the
    # oracle's ROK4 step then gives dPhi/dmu exactly.  (Central differences in mu
    # do not converge here: the FD-JVP quotients re-round at every evaluation.)
    prob, y = W.taylor_green(16, reynolds=100.0)
    if sutherland:
        prob = W.FlowProblem(**{**prob.__dict__, 'sutherland_s': 0.4, 't_ref': 0.5})
    y = np.ascontiguousarray(y + 0.01 * W.random_smooth_state(prob, seed=6))
    h = I.dt_from_cfl(prob, y, 2.0)
    c = np.random.default_rng(2).standard_normal(y.shape)
    _, mub = A.rok_step_vjp(prob, y, h, M, c)

    class MuStep(core.System):
        def f(self, yy):
            return core.residual(prob, yy) + 1e-30j * A.residual_dmu(prob, yy)

        def jvp(self, yy, v, f0, eps):
            return (self.f(np.asarray(yy) + eps * np.asarray(v)) - f0) / eps
    yc = I.rok_step(MuStep(prob), y.astype(complex), h, M)
    cs = float(np.sum(c * yc.imag) / 1e-30)
    assert abs(mub - cs) <= 1e-8 * abs(cs), (mub, cs)


def test_multi_step_derivative_conditioning():
    # Evidence for the choice of gradient checks: the derivative of the FD-JVP
    # ROK4 map over several steps is well conditioned on the Euler vortex but
    # moves by O(1e-2 .. 1) under 1e-12 relative changes of the state on the
    # low-Mach Taylor-Green state at CFL 4 (complex-step derivatives of the
    # oracle's own map, no differencing of the map)
    def ke(yy):
        return 0.5 * np.sum((yy[1] ** 2 + yy[2] ** 2) / yy[0])

    def deriv(prob, y0, h, M, K, d):
        yc = y0 + 1e-30j * d
        for _ in range(K):
            yc = I.rok_step(core.System(prob), yc, h, M)
        return float(np.imag(ke(yc)) / 1e-30)

    rng = np.random.default_rng(11)
    out = {}
    for name in ('vortex', 'tgv'):
        if name == 'vortex':
            prob, y0 = W.isentropic_vortex(20)
            cfl = 1.0
        else:
            prob, y0 = W.taylor_green(20, reynolds=200.0)
            y0 = np.ascontiguousarray(y0 + 0.01 * W.random_smooth_state(prob, seed=9))
            cfl = 4.0
        h = I.dt_from_cfl(prob, y0, cfl)
        d = rng.standard_normal(y0.shape)
        a = deriv(prob, y0, h, 6, 4, d)
        b = deriv(prob, y0 * (1 + 1e-12 * rng.standard_normal(y0.shape)), h, 6, 4, d)
        out[name] = abs(a - b) / abs(a)
    assert out['vortex'] < 1e-7, out
    assert out['tgv'] > 1e-4, out
