"""Pins of the oracle residual and FD-JVP against facts fixed by mathematics,
not by the oracle's own formulas (Sec. 3.2 Eq. Nav_Stokes; Sec. 2.3 Eq. matvecFD)."""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W


def _uniform_state(prob, q):
    y = np.empty(prob.shape)
    for k in range(4):
        y[k] = q[k]
    return y


def _phys_flux(Wp, nx, ny, g=1.4):
    r, u, v, p = Wp
    qn = u * nx + v * ny
    E = p / (g - 1) + 0.5 * r * (u * u + v * v)
    return np.array([r * qn, r * u * qn + p * nx, r * v * qn + p * ny, (E + p) * qn])


# ---- free stream, conservation, symmetry ------------------------------------

@pytest.mark.parametrize('kind', [W.EULER, W.NAVIER_STOKES])
def test_free_stream_uniform_periodic(kind):
    prob, _ = W.isentropic_vortex(16)
    prob.kind = kind
    prob.mu = 0.01
    y = _uniform_state(prob, prob.q_inf)
    assert np.abs(core.residual(prob, y)).max() <= 1e-13


def test_free_stream_curvilinear_periodic():
    xv, yv = W.perturbed_box_grid(24, 20, 3.0, 2.0, amp=0.3, seed=3)
    prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=24, ny=20, xv=xv, yv=yv, mu=0.01,
                         q_inf=(1.0, 0.4, -0.3, 3.0))
    y = _uniform_state(prob, prob.q_inf)
    f = core.residual(prob, y)
    assert np.abs(f).max() <= 1e-12


def test_free_stream_ogrid_interior():
    prob, y, ratio = W.cylinder_ogrid(32, 64)
    f = core.residual(prob, y)
    # the wall rows see the no-slip condition; away from them the metric closure
    # makes a uniform stream an exact steady state up to rounding
    scale = np.abs(y).max() * 64
    assert np.abs(f[:, 3:, :]).max() <= 1e-12 * scale
    assert np.abs(f[:, 0, :]).max() > 1.0


@pytest.mark.parametrize('case', ['vortex', 'tgv', 'curv'])
def test_discrete_conservation(case):
    if case == 'vortex':
        prob, y = W.isentropic_vortex(32)
    elif case == 'tgv':
        prob, y = W.taylor_green(32, reynolds=100.0)
    else:
        xv, yv = W.perturbed_box_grid(20, 18, 2.0, 2.0, amp=0.3, seed=1)
        prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=20, ny=18, xv=xv, yv=yv, mu=0.02)
        y = W.random_smooth_state(prob, seed=5, amp=0.1)
    f = core.residual(prob, y)
    vol = core.cell_volumes(prob)
    for k in range(4):
        scale = np.sum(np.abs(vol * f[k])) + 1e-300
        assert abs(np.sum(vol * f[k])) <= 1e-13 * scale * np.sqrt(f[k].size)


def test_euler_limit_of_ns_bitwise():
    prob, y = W.taylor_green(24)
    prob_e = W.FlowProblem(**{**prob.__dict__, 'kind': W.EULER})
    prob_ns0 = W.FlowProblem(**{**prob.__dict__, 'kind': W.NAVIER_STOKES, 'mu': 0.0})
    assert np.array_equal(core.residual(prob_e, y), core.residual(prob_ns0, y))


def test_transpose_symmetry_bitwise():
    prob, y = W.taylor_green(24, reynolds=200.0)
    y = y + 0.01 * W.random_smooth_state(prob, seed=2)
    yt = np.stack([y[0].T, y[2].T, y[1].T, y[3].T])
    f = core.residual(prob, y)
    ft = core.residual(prob, yt)
    assert np.array_equal(ft, np.stack([f[0].T, f[2].T, f[1].T, f[3].T]))


def test_curvilinear_matches_uniform_on_box():
    prob, y = W.taylor_green(20, reynolds=300.0)
    xv, yv = W.perturbed_box_grid(20, 20, prob.lx, prob.ly, amp=0.0)
    pc = W.FlowProblem(**{**prob.__dict__, 'xv': xv, 'yv': yv})
    f = core.residual(prob, y)
    fc = core.residual(pc, y)
    assert np.abs(f - fc).max() <= 1e-11 * np.abs(f).max()


# ---- Roe flux: consistency and upwinding ------------------------------------

@pytest.mark.parametrize('n', [(1.0, 0.0), (0.0, 1.0), (0.6, 0.8), (-0.28, 0.96)])
def test_roe_consistency(n):
    Wp = np.array([1.3, 0.4, -0.7, 0.9])
    F = core.roe_flux(Wp, Wp, n[0], n[1])
    assert np.allclose(F, _phys_flux(Wp, *n), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize('n', [(1.0, 0.0), (0.6, 0.8)])
def test_roe_supersonic_upwinding(n):
    # all four Roe eigenvalues positive (normal Mach ~ 2.5): flux is F(left) exactly;
    # all negative: F(right).  This pins every wave strength and eigenvector.
    nx, ny = n
    WL = np.array([1.0, 3.0 * nx, 3.0 * ny, 1.0])
    WR = np.array([1.2, 2.9 * nx + 0.1 * ny, 2.9 * ny - 0.1 * nx, 1.3])
    F = core.roe_flux(WL, WR, nx, ny, efix=0.0)
    assert np.allclose(F, _phys_flux(WL, nx, ny), rtol=1e-13, atol=1e-13)
    WLm = WL.copy(); WRm = WR.copy()
    WLm[1:3] *= -1; WRm[1:3] *= -1
    F = core.roe_flux(WLm, WRm, nx, ny, efix=0.0)
    assert np.allclose(F, _phys_flux(WRm, nx, ny), rtol=1e-13, atol=1e-13)


def test_roe_property_subsonic():
    # Roe's linearisation: F(R) - F(L) = A_roe (q_R - q_L); with the flux formula
    # F = (F_L + F_R)/2 - |A|dq/2 this means F - F_L = (A - |A|) dq / 2, so for a
    # state jump carried only by right-running waves (a pure shear jump with
    # positive normal velocity) the flux equals F_L.
    WL = np.array([1.0, 0.3, 0.2, 1.0])
    WR = np.array([1.0, 0.3, 0.5, 1.0])
    F = core.roe_flux(WL, WR, 1.0, 0.0, efix=0.0)
    assert np.allclose(F, _phys_flux(WL, 1.0, 0.0), rtol=1e-14, atol=1e-14)


# ---- spatial accuracy against the exact vortex and the heat equation ---------

def test_vortex_spatial_order():
    errs = []
    for n in (32, 64, 128):
        prob, y = W.isentropic_vortex(n)
        d = 1e-5
        dydt = (W.vortex_exact(prob, d) - W.vortex_exact(prob, -d)) / (2 * d)
        f = core.residual(prob, y)
        errs.append(np.sqrt(np.mean((f - dydt) ** 2)))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > 1.8, (errs, slopes)


def test_heat_conduction_at_rest():
    # u = v = 0, uniform p, T = T0 (1 + a sin x): the momentum residual vanishes and
    # dE/dt -> k d2T/dx2 = -k T0 a sin x (Fourier heat flux, Eq. Nav_Stokes q_i)
    errs = []
    for n in (32, 64):
        L = 2 * np.pi
        prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=n, ny=4, lx=L, ly=L * 4 / n, mu=0.05)
        X, _ = W.cell_centres_uniform(n, 4, L, L * 4 / n)
        a, T0, p0 = 0.1, 1.0, 1.0
        T = T0 * (1 + a * np.sin(X))
        rho = p0 / T
        y = np.stack([rho, 0 * X, 0 * X, p0 / 0.4 + 0 * X])
        f = core.residual(prob, y)
        k = prob.mu * prob.gamma / ((prob.gamma - 1) * prob.prandtl)
        exact = -k * T0 * a * np.sin(X)
        assert np.abs(f[1:3]).max() <= 1e-12
        errs.append(np.abs(f[3] - exact).max() / np.abs(exact).max())
    assert errs[1] < 0.3 * errs[0] and errs[1] < 0.01


def test_tgv_viscous_decay_rate():
    # incompressible limit: u ~ exp(-2 nu t), so the viscous part of d(KE)/dt is
    # -4 nu KE at t = 0; the Roe/MUSCL numerical dissipation (Euler part) is O(dx^3)
    def rate(p, y):
        f = core.residual(p, y)
        rho, mx, my = y[0], y[1], y[2]
        u, v = mx / rho, my / rho
        dke = np.mean(u * f[1] + v * f[2] - 0.5 * (u * u + v * v) * f[0])
        return dke / np.mean(0.5 * rho * (u * u + v * v))
    re = 50.0
    inv = []
    for n in (32, 64):
        prob, y = W.taylor_green(n, mach=0.05, reynolds=re)
        pe = W.FlowProblem(**{**prob.__dict__, 'kind': W.EULER})
        r_ns, r_e = rate(prob, y), rate(pe, y)
        inv.append(r_e)
        assert abs((r_ns - r_e) - (-4.0 / re)) <= 0.005 * (4.0 / re), (n, r_ns, r_e)
    assert inv[0] < 0 and inv[1] < 0 and 6.0 < inv[0] / inv[1] < 10.0, inv


# ---- FD JVP ------------------------------------------------------------------

def test_fd_eps_is_power_of_two_near_knoll_keyes():
    for yn in (0.0, 1.0, 37.5, 1e4, 3.3e6):
        e = I.fd_eps(yn)
        m, _ = np.frexp(e)
        assert m == 0.5
        kk = np.sqrt(2.0 ** -52 * (1 + yn))
        assert kk / np.sqrt(2) <= e <= kk * np.sqrt(2)


def test_fd_jvp_first_order_in_eps():
    prob, y = W.isentropic_vortex(16)
    rng = np.random.default_rng(0)
    v = rng.normal(size=y.shape)
    v /= np.linalg.norm(v)
    f0 = core.residual(prob, y)
    hc = 1e-5
    ref = (core.residual(prob, y + hc * v) - core.residual(prob, y - hc * v)) / (2 * hc)
    errs = []
    epss = [2.0 ** -8, 2.0 ** -10, 2.0 ** -12, 2.0 ** -14]
    for e in epss:
        errs.append(np.linalg.norm(core.jvp_fd(prob, y, v, f0, e) - ref))
    slopes = [np.log2(errs[i] / errs[i + 1]) / 2 for i in range(3)]
    assert all(0.85 < s < 1.15 for s in slopes), slopes


def test_fd_jvp_against_dense_jacobian():
    prob, y = W.taylor_green(8, reynolds=100.0)
    N = y.size
    f0 = core.residual(prob, y)
    hc = 1e-6
    J = np.empty((N, N))
    for c in range(N):
        e = np.zeros(N); e[c] = hc
        J[:, c] = ((core.residual(prob, y + e.reshape(y.shape)) - core.residual(prob, y - e.reshape(y.shape))) / (2 * hc)).ravel()
    rng = np.random.default_rng(1)
    v = rng.normal(size=y.shape)
    v /= np.linalg.norm(v)
    eps = I.fd_eps(np.linalg.norm(y))
    w = core.jvp_fd(prob, y, v, f0, eps).ravel()
    assert np.linalg.norm(w - J @ v.ravel()) <= 1e-5 * np.linalg.norm(J @ v.ravel())


def test_cfl_dt_uniform_closed_form():
    prob, y = W.isentropic_vortex(32)
    dt = I.dt_from_cfl(prob, y, 1.0)
    rho = y[0]; u = y[1] / rho; v = y[2] / rho
    p = 0.4 * (y[3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(1.4 * p / rho)
    dx = prob.lx / prob.nx
    assert np.isclose(dt, 1.0 / np.max((np.abs(u) + c) / dx + (np.abs(v) + c) / dx), rtol=1e-13)


# ---- exact JVP (complex step) -------------------------------------------------

@pytest.mark.parametrize('which', ['vortex', 'tgv', 'ogrid'])
def test_complex_step_jvp_matches_dense_jacobian(which):
    if which == 'vortex':
        prob, y = W.isentropic_vortex(8)
    elif which == 'tgv':
        prob, y = W.taylor_green(8, reynolds=100.0)
        prob = W.FlowProblem(**{**prob.__dict__, 'sutherland_s': 0.4, 't_ref': 70.0})
    else:
        prob, y, _ = W.cylinder_ogrid(6, 12)
        y = y + 0.02 * W.random_smooth_state(prob, seed=1)
    N = y.size
    rng = np.random.default_rng(2)
    v = rng.normal(size=y.shape)
    w = core.jvp_exact(prob, y, v)
    # fourth-order central differences, column by column of the dense Jacobian
    hc = 1e-4
    J = np.empty((N, N))
    for c in range(N):
        e = np.zeros(N); e[c] = hc
        e = e.reshape(y.shape)
        J[:, c] = ((-core.residual(prob, y + 2 * e) + 8 * core.residual(prob, y + e)
                    - 8 * core.residual(prob, y - e) + core.residual(prob, y - 2 * e)) / (12 * hc)).ravel()
    ref = J @ v.ravel()
    assert np.linalg.norm(w.ravel() - ref) <= 1e-7 * np.linalg.norm(ref)


def test_complex_step_is_linear_and_matches_fd_limit():
    prob, y = W.taylor_green(16, reynolds=200.0)
    rng = np.random.default_rng(4)
    v1, v2 = rng.normal(size=y.shape), rng.normal(size=y.shape)
    w1, w2 = core.jvp_exact(prob, y, v1), core.jvp_exact(prob, y, v2)
    w12 = core.jvp_exact(prob, y, 2.0 * v1 - 3.0 * v2)
    assert np.abs(w12 - (2.0 * w1 - 3.0 * w2)).max() <= 1e-12 * np.abs(w12).max()
    # the one-sided FD quotient approaches it at first order in eps
    f0 = core.residual(prob, y)
    e = [np.linalg.norm(core.jvp_fd(prob, y, v1, f0, 2.0 ** -k) - w1) for k in (10, 12, 14)]
    assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5


def test_openmp_build_gives_the_same_bits():
    # the CPU-baseline build of the oracle (OpenMP over independent rows) must
    # compute exactly what the plain build computes
    cases = [W.taylor_green(40, reynolds=300.0), W.isentropic_vortex(36)]
    p3, y3, _ = W.cylinder_ogrid(12, 40)
    cases.append((p3, y3 + 0.02 * W.random_smooth_state(p3, seed=2)))
    plain = [core.residual(p, y) for p, y in cases]
    v = np.random.default_rng(3).standard_normal(cases[0][1].shape)
    j_plain = core.jvp_fd(cases[0][0], cases[0][1], v, plain[0], 2.0 ** -20)
    try:
        core.use_parallel_build(4)
        for (p, y), f in zip(cases, plain):
            assert np.array_equal(core.residual(p, y), f)
        assert np.array_equal(core.jvp_fd(cases[0][0], cases[0][1], v, plain[0], 2.0 ** -20), j_plain)
    finally:
        core.use_parallel_build(None)
