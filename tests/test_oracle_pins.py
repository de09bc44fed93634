"""Pins of the parts of the oracle residual that a free-stream, conservation or
order test cannot see: Sutherland's law, the no-slip wall ghosts, the MUSCL
kappa coefficients, the Roe flux against a form built independently of the
oracle's own algebra, and the CFL step on curvilinear grids and with
Sutherland viscosity.

Each pin compares with a closed form or with an invariant that a plausible
mistake (a wrong exponent, a wrong ghost layer, (1 - kappa) and (1 + kappa)
swapped, a dropped or mis-signed wave) would break (Sec. 3.2 Eq. Nav_Stokes;
the discretisation of Sec. 4.2: kappa-MUSCL without limiter, Roe flux,
Sutherland's law)."""
import numpy as np
import pytest

from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W

GAMMA = 1.4


# ---- helpers (inputs and closed forms only) -----------------------------------

def _state(rho, u, v, p, g=GAMMA):
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)]))


def _shear_box(n=32, ny=24, T=1.0, mu=0.02, suth=0.0, t_ref=1.0, wall=False, lx=1.0, ly=2.0, U=0.1):
    """Uniform box, rho and p uniform (temperature T = p/rho), u = U s(y), v = 0.
    Periodic: s = sin(2 pi y / ly).  wall=True: no-slip walls at y = 0 and
    y = ly and s = sin(pi y / ly), which is odd about both walls."""
    bc = (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL) if wall else (W.PERIODIC,) * 4
    prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=n, ny=ny, lx=lx, ly=ly, bc=bc, mu=mu,
                         sutherland_s=suth, t_ref=t_ref)
    _, Y = W.cell_centres_uniform(n, ny, lx, ly)
    k = (np.pi if wall else 2 * np.pi) / ly
    rho = np.ones_like(Y)
    p = T * rho
    u = U * np.sin(k * Y)
    return prob, _state(rho, u, 0 * Y, p), k, U * np.sin(k * Y)


def _mu_effective(prob, y, k, u):
    """Viscosity seen by the residual in a parallel shear flow u(y), v = 0 with
    uniform rho and p: the Roe dissipation vanishes (no pressure, density or
    normal-velocity jump; the shear wave moves at q_n = 0), x-faces carry no
    differences, so f(rho u) = mu (u_{j+1} - 2 u_j + u_{j-1}) / dy^2, and for
    u = U sin(k y) that is mu u_j (2 cos(k dy) - 2) / dy^2 exactly."""
    f = core.residual(prob, y)
    dy = prob.ly / prob.ny
    lam = (2.0 * np.cos(k * dy) - 2.0) / dy ** 2
    big = np.abs(u) > 0.3 * np.abs(u).max()
    mu = f[1][big] / (lam * u[big])
    return mu, f


# ---- Sutherland's law ------------------------------------------------------------

def test_shear_flow_reads_constant_viscosity_exactly():
    prob, y, k, u = _shear_box(mu=0.037)
    mu, f = _mu_effective(prob, y, k, u)
    assert np.abs(mu / 0.037 - 1.0).max() <= 1e-10
    assert np.abs(f[0]).max() <= 1e-15 and np.abs(f[2]).max() <= 1e-12


@pytest.mark.parametrize('t', [1.0, 0.5, 3.0])
def test_sutherland_closed_form(t):
    # mu(T) = mu_ref t^{3/2} (1 + s) / (t + s), t = T / T_ref, s = S / T_ref
    # (Sec. 4.2: Sutherland's law; S = 110.4 K, T_ref = 278 K); at t = 1, mu = mu_ref
    s, mu_ref, t_ref = 110.4 / 278.0, 0.02, 0.8
    prob, y, k, u = _shear_box(T=t * t_ref, mu=mu_ref, suth=s, t_ref=t_ref)
    mu, _ = _mu_effective(prob, y, k, u)
    expect = mu_ref * t ** 1.5 * (1.0 + s) / (t + s)
    assert np.abs(mu / expect - 1.0).max() <= 1e-10, (t, mu.mean(), expect)


@pytest.mark.parametrize('t, ratio, tol', [(1e8, 2.0, 1e-7), (1e-8, 8.0, 1e-6)])
def test_sutherland_asymptotic_exponents(t, ratio, tol):
    # mu ~ t^{1/2} far above S and ~ t^{3/2} far below it: mu(4t)/mu(t) -> 2 and 8.
    # A law with the wrong power of t fails one of the two limits.  The flow keeps
    # T = p/rho = 1 and moves t through T_ref; mu_ref keeps mu near 0.02.
    s = 110.4 / 278.0
    mu_ref = 0.02 / (t ** 0.5 * (1 + s)) if t > 1 else 0.02 * s / (t ** 1.5 * (1 + s))
    mus = []
    for tt in (t, 4 * t):
        prob, y, k, u = _shear_box(T=1.0, mu=mu_ref, suth=s, t_ref=1.0 / tt)
        mus.append(_mu_effective(prob, y, k, u)[0].mean())
    assert abs(mus[1] / mus[0] / ratio - 1.0) <= tol, mus[1] / mus[0]


# ---- no-slip adiabatic wall ------------------------------------------------------

def test_wall_shear_stress_of_odd_profile():
    # channel between no-slip walls, u = U sin(pi y / H): the mirrored ghosts
    # (rho, -u, -v, p) continue the profile oddly through each wall, so the wall
    # rows obey the same discrete relation as the interior, with the wall face
    # carrying the stress mu (u_0 - u_ghost) / dy = 2 mu u_0 / dy
    mu0 = 0.05
    prob, y, k, u = _shear_box(mu=mu0, wall=True)
    f = core.residual(prob, y)
    dy = prob.ly / prob.ny
    lam = (2.0 * np.cos(k * dy) - 2.0) / dy ** 2
    ref = mu0 * lam * u
    scale = np.abs(ref).max()
    assert np.abs(f[1] - ref).max() <= 1e-12 * scale
    for row in (0, -1):   # the wall rows themselves
        assert np.abs(f[1][row] - ref[row]).max() <= 1e-12 * scale
    assert np.abs(f[0]).max() <= 1e-15 and np.abs(f[2]).max() <= 1e-12 * scale


def _wall_cases():
    out = []
    prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=20, ny=16, lx=2.0, ly=1.5,
                         bc=(W.PERIODIC, W.PERIODIC, W.WALL, W.WALL), mu=0.02,
                         sutherland_s=0.4, t_ref=1.0 / 1.4)
    out.append(('channel', prob, W.random_smooth_state(prob, seed=9, amp=0.1)))
    # annulus between two no-slip cylinders: the O-grid generator with walls on both radial ends
    p4, _, _ = W.cylinder_ogrid(12, 40, r_outer=3.0)
    p4 = W.FlowProblem(**{**p4.__dict__, 'bc': (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL)})
    out.append(('annulus', p4, W.random_smooth_state(p4, seed=10, amp=0.1)))
    return out


@pytest.mark.parametrize('case', _wall_cases(), ids=lambda c: c[0])
def test_walls_pass_no_mass_and_no_energy(case):
    # mirrored ghosts make the Riemann problem at the wall symmetric: the Roe
    # averages have zero normal velocity, so no mass or energy crosses the wall;
    # the wall-face velocity is zero (no stress work) and the mirrored temperature
    # gives no normal heat flux (adiabatic).  With periodic i-sides every other
    # face cancels, so total mass and energy are conserved exactly.
    _, prob, y = case
    f = core.residual(prob, y)
    vol = core.cell_volumes(prob)
    for k in (0, 3):
        scale = np.sum(np.abs(vol * f[k]))
        assert abs(np.sum(vol * f[k])) <= 1e-13 * scale * np.sqrt(f[k].size), (case[0], k)
    # momentum is not conserved: the walls push (pressure and shear)
    assert abs(np.sum(vol * f[1])) + abs(np.sum(vol * f[2])) > 1e-6


def test_wall_ghost_layers_are_the_mirror_images():
    # a state symmetric about the lower wall (cells j and -1-j mirrored) is
    # what the ghosts hold: the residual of a periodic box whose lower half is
    # the mirror image of its upper half equals, in the upper half, the residual
    # of the walled channel (both ghost layers enter through MUSCL and the
    # viscous stencil, so a wrong layer or a missing sign breaks the equality)
    n, ny = 16, 12
    pw = W.FlowProblem(kind=W.NAVIER_STOKES, nx=n, ny=ny, lx=1.0, ly=1.0,
                       bc=(W.PERIODIC, W.PERIODIC, W.WALL, W.WALL), mu=0.03)
    yw = W.random_smooth_state(pw, seed=12, amp=0.15)
    # periodic box of height 2: rows -ny..-1 are the mirror of rows 0..ny-1,
    # which makes it symmetric about y = 0 and (by periodicity) about y = 1
    pp = W.FlowProblem(kind=W.NAVIER_STOKES, nx=n, ny=2 * ny, lx=1.0, ly=2.0, mu=0.03)
    mirror = yw[:, ::-1, :].copy()
    mirror[1:3] *= -1.0
    yp = np.ascontiguousarray(np.concatenate([mirror, yw], axis=1))
    fw = core.residual(pw, yw)
    fp = core.residual(pp, yp)[:, ny:, :]
    assert np.abs(fw - fp).max() <= 1e-12 * np.abs(fw).max()


# ---- MUSCL kappa --------------------------------------------------------------------

def _cubic_avg(a, x0, x1):
    """Cell average of a0 + a1 x + a2 x^2 + a3 x^3 over [x0, x1] (antiderivative)."""
    P = lambda x: a[0] * x + a[1] * x ** 2 / 2 + a[2] * x ** 3 / 3 + a[3] * x ** 4 / 4
    return (P(x1) - P(x0)) / (x1 - x0)


@pytest.mark.parametrize('kappa', [1.0 / 3.0, -1.0, 0.0, 1.0])
def test_muscl_kappa_on_cell_averages_of_a_cubic(kappa):
    # supersonic stream along x (every Roe wave runs right, the flux is F(W_L),
    # pinned by test_roe_supersonic_upwinding), uniform u and p, density given as
    # cell averages of a cubic rho(x).  The kappa scheme reconstructs the face
    # value of a quadratic with error h^2 c (3 kappa - 1) / 6 (c its x^2
    # coefficient): exact only for kappa = 1/3.  For a cubic the error's
    # quadratic part varies linearly along x, so the interior mass residual
    # differs from -u (rho(x_{i+1/2}) - rho(x_{i-1/2})) / h by the constant
    # -d u h^2 (3 kappa - 1) / 2 (d the x^3 coefficient); a swap of
    # (1 - kappa) and (1 + kappa) turns kappa = 1/3 into kappa = -1/3.
    n, h = 40, 0.05
    a = (1.0, 0.2, 0.3, 0.25)
    x = np.arange(n + 1) * h - 1.0          # faces, [-1, 1]
    avg = np.array([_cubic_avg(a, x[i], x[i + 1]) for i in range(n)])
    rho = np.tile(avg, (3, 1))
    u0, p0 = 3.0, 1.0 / GAMMA
    prob = W.FlowProblem(kind=W.EULER, nx=n, ny=3, lx=n * h, ly=3 * h, muscl_kappa=kappa, entropy_fix=0.1)
    y = _state(rho, np.full_like(rho, u0), 0 * rho, np.full_like(rho, p0))
    f = core.residual(prob, y)
    rface = a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3
    exact = -u0 * (rface[1:] - rface[:-1]) / h
    err = f[0][1, 3:n - 3] - exact[3:n - 3]            # interior cells (periodic wrap is a jump)
    offset = -a[3] * u0 * h ** 2 * (3 * kappa - 1) / 2
    assert np.abs(err - offset).max() <= 1e-11, (kappa, err.mean(), offset)
    # x-momentum: flux rho u^2 + p, p uniform: the same with a factor u
    errm = f[1][1, 3:n - 3] - u0 * exact[3:n - 3]
    assert np.abs(errm - u0 * offset).max() <= 1e-10


# ---- Roe flux against an eigen-decomposition of the Roe matrix -----------------------

def _cons(Wp, g=GAMMA):
    r, u, v, p = Wp
    return np.array([r, r * u, r * v, p / (g - 1) + 0.5 * r * (u * u + v * v)], dtype=complex)


def _phys_flux_cons(q, nx, ny, g=GAMMA):
    r, mu_, mv, E = q
    u, v = mu_ / r, mv / r
    p = (g - 1) * (E - 0.5 * r * (u * u + v * v))
    qn = u * nx + v * ny
    return np.array([r * qn, mu_ * qn + p * nx, mv * qn + p * ny, (E + p) * qn])


def _roe_textbook(WL, WR, nx, ny, efix, g=GAMMA):
    """1/2 (F(q_L) + F(q_R)) - 1/2 |A| (q_R - q_L), |A| = R |Lambda| R^{-1}, with
    A the flux Jacobian (complex step, column by column) at the Roe-averaged
    state (sqrt(rho)-weighted u, v and total enthalpy H) and Harten's fix on the
    two acoustic eigenvalues.  Also returns the defect of Roe's property
    A (q_R - q_L) = F(q_R) - F(q_L)."""
    qL, qR = _cons(WL), _cons(WR)
    sL, sR = np.sqrt(WL[0]), np.sqrt(WR[0])
    HL = (qL[3].real + WL[3]) / WL[0]
    HR = (qR[3].real + WR[3]) / WR[0]
    ut = (sL * WL[1] + sR * WR[1]) / (sL + sR)
    vt = (sL * WL[2] + sR * WR[2]) / (sL + sR)
    Ht = (sL * HL + sR * HR) / (sL + sR)
    rt = sL * sR
    pt = rt * (g - 1) / g * (Ht - 0.5 * (ut * ut + vt * vt))
    qt = _cons((rt, ut, vt, pt))
    A = np.empty((4, 4))
    hc = 1e-30
    for c in range(4):
        e = np.zeros(4, dtype=complex)
        e[c] = 1j * hc
        A[:, c] = np.imag(_phys_flux_cons(qt + e, nx, ny)) / hc
    # spectrum by numpy.linalg.eig: q_n - c, q_n (twice: entropy and shear
    # waves), q_n + c.  The double eigenvalue makes eig's eigenvector matrix
    # ill-conditioned, so |A| is formed from the spectral projectors
    # P_k = prod_{m != k} (A - l_m I) / (l_k - l_m) over the three distinct
    # eigenvalues (A is diagonalisable, so A = sum_k l_k P_k; asserted below).
    lam = np.sort(np.linalg.eig(A)[0].real)
    ct = np.sqrt((g - 1) * (Ht - 0.5 * (ut * ut + vt * vt)))
    qnt = ut * nx + vt * ny
    assert np.allclose(lam, [qnt - ct, qnt, qnt, qnt + ct], rtol=0, atol=1e-12 * (abs(qnt) + ct))
    ls = [lam[0], 0.5 * (lam[1] + lam[2]), lam[3]]
    E = np.eye(4)
    P = []
    for k in range(3):
        Pk = E.copy()
        for m in range(3):
            if m != k:
                Pk = Pk @ (A - ls[m] * E) / (ls[k] - ls[m])
        P.append(Pk)
    assert np.abs(sum(l * Pk for l, Pk in zip(ls, P)) - A).max() <= 1e-12 * np.abs(A).max()
    delta = efix * (abs(qnt) + ct)
    a = [abs(x) for x in ls]
    for k in (0, 2):       # Harten's fix on the acoustic waves only
        if a[k] < delta:
            a[k] = (a[k] ** 2 + delta ** 2) / (2 * delta)
    absA = sum(ak * Pk for ak, Pk in zip(a, P))
    diss = absA @ (qR - qL).real
    FL = _phys_flux_cons(qL, nx, ny).real
    FR = _phys_flux_cons(qR, nx, ny).real
    roe_prop = np.abs(A @ (qR - qL).real - (FR - FL)).max() / np.abs(FR - FL).max()
    return 0.5 * (FL + FR) - 0.5 * diss, roe_prop


def _random_pairs(seed, n, sonic=False):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        th = rng.uniform(0, 2 * np.pi)
        nx, ny = np.cos(th), np.sin(th)
        WL = np.array([rng.uniform(0.5, 2.0), rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(0.4, 1.5)])
        WR = WL * (1 + rng.uniform(-0.3, 0.3, 4)) + np.array([0, rng.normal(0, 0.2), rng.normal(0, 0.2), 0])
        if sonic:
            # normal velocity near the sound speed: an acoustic eigenvalue near zero
            c = np.sqrt(GAMMA * WL[3] / WL[0])
            for Wp in (WL, WR):
                Wp[1] += (c * rng.uniform(0.9, 1.1)) * nx
                Wp[2] += (c * rng.uniform(0.9, 1.1)) * ny
        out.append((WL, WR, nx, ny))
    return out


@pytest.mark.parametrize('efix', [0.0, 0.1, 0.3])
@pytest.mark.parametrize('sonic', [False, True])
def test_roe_flux_matches_eigendecomposition(efix, sonic):
    worst = 0.0
    for WL, WR, nx, ny in _random_pairs(7 + int(sonic), 40, sonic):
        F = core.roe_flux(WL, WR, nx, ny, efix=efix)
        Ft, roe_prop = _roe_textbook(WL, WR, nx, ny, efix)
        assert roe_prop <= 1e-12                    # the averages are Roe's: A dq = dF
        scale = np.abs(_phys_flux_cons(_cons(WL), nx, ny)).max()
        worst = max(worst, np.abs(F - Ft).max() / scale)
    assert worst <= 1e-13, worst


def test_roe_entropy_fix_is_active_near_sonic_points():
    # the sonic cases above do exercise the fix: the flux changes with efix there
    changed = 0
    for WL, WR, nx, ny in _random_pairs(8, 40, True):
        d = np.abs(core.roe_flux(WL, WR, nx, ny, efix=0.3) - core.roe_flux(WL, WR, nx, ny, efix=0.0)).max()
        changed += d > 1e-8
    assert changed >= 20, changed


# ---- CFL step on curvilinear grids and with Sutherland viscosity ----------------------

def test_cfl_dt_curvilinear_box_equals_uniform_with_viscosity():
    prob, y = W.taylor_green(24, reynolds=40.0)
    xv, yv = W.perturbed_box_grid(24, 24, prob.lx, prob.ly, amp=0.0)
    pc = W.FlowProblem(**{**prob.__dict__, 'xv': xv, 'yv': yv})
    dt_u, dt_c = I.dt_from_cfl(prob, y, 2.0), I.dt_from_cfl(pc, y, 2.0)
    assert abs(dt_u - dt_c) <= 1e-13 * dt_u
    # the viscous part matters at this Re: dropping mu changes dt
    pe = W.FlowProblem(**{**prob.__dict__, 'kind': W.EULER})
    assert I.dt_from_cfl(pe, y, 2.0) > 1.02 * dt_u


def test_cfl_dt_uniform_viscous_closed_form():
    # dt = CFL / max[(|u| + c)/dx + (|v| + c)/dy + 2 nu_eff (1/dx^2 + 1/dy^2)],
    # nu_eff = max(4/3, gamma/Pr) mu / rho
    prob, y = W.taylor_green(20, reynolds=30.0)
    prob = W.FlowProblem(**{**prob.__dict__, 'ny': 20, 'ly': prob.ly * 0.5})
    rho = y[0]; u = y[1] / rho; v = y[2] / rho
    p = 0.4 * (y[3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(1.4 * p / rho)
    dx, dy = prob.lx / prob.nx, prob.ly / prob.ny
    nu = max(4 / 3, 1.4 / 0.72) * prob.mu / rho
    lam = (np.abs(u) + c) / dx + (np.abs(v) + c) / dy + 2 * nu * (1 / dx ** 2 + 1 / dy ** 2)
    assert np.isclose(I.dt_from_cfl(prob, y, 1.5), 1.5 / lam.max(), rtol=1e-13)


def test_cfl_dt_is_rotation_invariant():
    # rotating the grid and the velocity together leaves every |u.S|, |S| and Vol unchanged
    xv, yv = W.perturbed_box_grid(20, 16, 2.0, 1.6, amp=0.3, seed=5)
    prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=20, ny=16, xv=xv, yv=yv, mu=0.01,
                         sutherland_s=0.4, t_ref=0.9)
    y = W.random_smooth_state(prob, seed=6, amp=0.1)
    th = 0.7
    c, s = np.cos(th), np.sin(th)
    pr = W.FlowProblem(**{**prob.__dict__, 'xv': c * xv - s * yv, 'yv': s * xv + c * yv})
    yr = y.copy()
    yr[1], yr[2] = c * y[1] - s * y[2], s * y[1] + c * y[2]
    d0, d1 = I.dt_from_cfl(prob, y, 1.0), I.dt_from_cfl(pr, yr, 1.0)
    assert abs(d0 - d1) <= 1e-12 * d0


def test_cfl_dt_sutherland_uses_the_residuals_viscosity():
    # uniform temperature T: the Sutherland problem's dt equals the dt of a
    # constant-viscosity problem whose mu is the one the residual itself exhibits
    # at T (measured by the shear-flow pin above), and at T = T_ref it is mu_ref
    s, t_ref = 110.4 / 278.0, 0.8
    for t in (1.0, 2.5):
        prob, y, k, u = _shear_box(T=t * t_ref, mu=0.02, suth=s, t_ref=t_ref)
        mu_eff = _mu_effective(prob, y, k, u)[0].mean()
        pc = W.FlowProblem(**{**prob.__dict__, 'sutherland_s': 0.0, 'mu': mu_eff})
        d_s, d_c = I.dt_from_cfl(prob, y, 1.0), I.dt_from_cfl(pc, y, 1.0)
        assert abs(d_s - d_c) <= 1e-10 * d_c, (t, d_s, d_c)
        if t == 1.0:
            assert abs(mu_eff / 0.02 - 1) <= 1e-10


def test_compressive_stress_has_the_stokes_factor_four_thirds():
    # u = U sin(k x), v = 0: the viscous part of the residual (Navier-Stokes minus
    # Euler, the fluxes being additive) in the x-momentum equation is
    # d/dx (mu (2 u_x - 2/3 (u_x + v_y))) = 4/3 mu u_xx, discretely
    # 4/3 mu u_i (2 cos(k dx) - 2) / dx^2 (Stokes hypothesis, Eq. Nav_Stokes)
    n, mu0 = 32, 0.03
    prob = W.FlowProblem(kind=W.NAVIER_STOKES, nx=n, ny=4, lx=2.0, ly=0.25, mu=mu0)
    X, _ = W.cell_centres_uniform(n, 4, 2.0, 0.25)
    k = 2 * np.pi / 2.0
    u = 0.05 * np.sin(k * X)
    y = _state(np.ones_like(X), u, 0 * X, np.full_like(X, 1.0))
    pe = W.FlowProblem(**{**prob.__dict__, 'kind': W.EULER})
    dv = core.residual(prob, y) - core.residual(pe, y)
    dx = 2.0 / n
    ref = 4.0 / 3.0 * mu0 * u * (2 * np.cos(k * dx) - 2) / dx ** 2
    assert np.abs(dv[1] - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(dv[0]).max() == 0.0 and np.abs(dv[2]).max() <= 1e-13


@pytest.mark.parametrize('visc', [False, True])
def test_curvilinear_residual_is_rotation_equivariant(visc):
    # rotating a curvilinear grid and the velocity field by one angle rotates the
    # momentum residual and leaves the mass and energy residuals unchanged: pins
    # the face normals, lengths, volumes and the diamond (Green-Gauss) gradient
    # coefficients of a general quadrilateral grid
    xv, yv = W.perturbed_box_grid(20, 18, 2.0, 1.8, amp=0.35, seed=8)
    prob = W.FlowProblem(kind=W.NAVIER_STOKES if visc else W.EULER, nx=20, ny=18, xv=xv, yv=yv,
                         mu=0.02, sutherland_s=0.4 if visc else 0.0, t_ref=0.8)
    y = W.random_smooth_state(prob, seed=13, amp=0.1)
    th = 0.9
    c, s = np.cos(th), np.sin(th)
    pr = W.FlowProblem(**{**prob.__dict__, 'xv': c * xv - s * yv, 'yv': s * xv + c * yv})
    yr = y.copy()
    yr[1], yr[2] = c * y[1] - s * y[2], s * y[1] + c * y[2]
    f, fr = core.residual(prob, y), core.residual(pr, yr)
    scale = np.abs(f).max()
    assert np.abs(fr[0] - f[0]).max() <= 1e-11 * scale
    assert np.abs(fr[3] - f[3]).max() <= 1e-11 * scale
    assert np.abs(fr[1] - (c * f[1] - s * f[2])).max() <= 1e-11 * scale
    assert np.abs(fr[2] - (s * f[1] + c * f[2])).max() <= 1e-11 * scale
