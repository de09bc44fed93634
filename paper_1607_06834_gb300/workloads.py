"""Seeded synthetic inputs: problem descriptions, grids and initial states.

This module holds no arithmetic of the time-stepping method or of the
spatial residual; it only builds inputs (vertex coordinates, initial
conditions, closed-form exact solutions used as checks, and seeded draws).
Both the CUDA path and the CPU oracle take their inputs from here.

State layout everywhere: ``y[var, j, i]`` with var = (rho, rho*u, rho*v, E),
i the fastest index (structure of arrays, C order), float64.

The paper studies cylinder and airfoil flows whose grids are not published;
the problems here are synthetic stand-ins with the shapes and stiffness
sources of those workloads (Sec. 4.1-4.4): an isentropic vortex (smooth
Euler flow with an exact solution), a decaying Taylor-Green vortex
(acoustically stiff at low Mach number) and a viscous cylinder on a
stretched O-grid (wall-spacing stiffness), plus Lorenz-96 (appendix).
"""
from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import numpy as np

PERIODIC, WALL, FARFIELD = 0, 1, 2
EULER, NAVIER_STOKES, LORENZ96 = 0, 1, 2


@dataclass
class FlowProblem:
    """Problem description shared by the C-ABI binding and the oracle wrapper."""
    kind: int = EULER
    nx: int = 64
    ny: int = 64
    lx: float = 1.0
    ly: float = 1.0
    xv: Optional[np.ndarray] = None      # (ny+1, nx+1) vertex x, or None: uniform box
    yv: Optional[np.ndarray] = None
    bc: Tuple[int, int, int, int] = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    gamma: float = 1.4
    prandtl: float = 0.72
    mu: float = 0.0                      # viscosity at t_ref
    t_ref: float = 1.0
    sutherland_s: float = 0.0            # S / t_ref; <= 0 means constant mu
    q_inf: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 2.5)
    muscl_kappa: float = 1.0 / 3.0
    entropy_fix: float = 0.1
    lorenz_f: float = 8.0
    name: str = ''

    @property
    def curvilinear(self) -> bool:
        return self.xv is not None

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    @property
    def ndof(self) -> int:
        return self.nx if self.kind == LORENZ96 else 4 * self.nx * self.ny

    @property
    def shape(self):
        return (self.nx,) if self.kind == LORENZ96 else (4, self.ny, self.nx)


def _conservative(rho, u, v, p, gamma):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def cell_centres_uniform(nx, ny, lx, ly):
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    return np.meshgrid(x, y)  # X[j, i], Y[j, i]


# --- isentropic vortex ------------------------------------------------------

def vortex_state(X, Y, x0, y0, beta=5.0, gamma=1.4, mach=0.5, lx=10.0, ly=10.0):
    """Isentropic vortex of strength beta centred at (x0, y0) in a free stream of
    Mach number ``mach`` along the diagonal; rho_inf = p_inf = 1 (so T = p/rho = 1),
    nearest periodic image of the centre.  Point values at (X, Y)."""
    dx = X - x0
    dy = Y - y0
    dx = dx - lx * np.round(dx / lx)
    dy = dy - ly * np.round(dy / ly)
    r2 = dx * dx + dy * dy
    uinf = vinf = mach * np.sqrt(gamma) / np.sqrt(2.0)
    e = np.exp(0.5 * (1.0 - r2))
    u = uinf - beta / (2.0 * np.pi) * e * dy
    v = vinf + beta / (2.0 * np.pi) * e * dx
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _conservative(rho, u, v, p, gamma)


def isentropic_vortex(n=64, lx=10.0, centre=(5.0, 5.0), beta=5.0, gamma=1.4, mach=0.5):
    """Euler isentropic vortex on a periodic n x n uniform grid of [0, lx]^2."""
    uinf = mach * np.sqrt(gamma) / np.sqrt(2.0)
    qinf = tuple(float(v) for v in _conservative(np.array(1.0), np.array(uinf), np.array(uinf),
                                                  np.array(1.0), gamma))
    prob = FlowProblem(kind=EULER, nx=n, ny=n, lx=lx, ly=lx, gamma=gamma, q_inf=qinf,
                       name='isentropic-vortex-%dx%d' % (n, n))
    X, Y = cell_centres_uniform(n, n, lx, lx)
    y0 = vortex_state(X, Y, centre[0], centre[1], beta, gamma, mach, lx, lx)
    return prob, np.ascontiguousarray(y0)


def vortex_exact(prob, t, centre=(5.0, 5.0), beta=5.0, mach=0.5):
    """Exact solution of the vortex problem at time t: the initial vortex advected
    with the free stream (nearest periodic image)."""
    uinf = mach * np.sqrt(prob.gamma) / np.sqrt(2.0)
    X, Y = cell_centres_uniform(prob.nx, prob.ny, prob.lx, prob.ly)
    return vortex_state(X, Y, centre[0] + uinf * t, centre[1] + uinf * t, beta, prob.gamma, mach,
                        prob.lx, prob.ly)


# --- Taylor-Green vortex ----------------------------------------------------

def taylor_green(n=512, mach=0.1, reynolds=1600.0, gamma=1.4, prandtl=0.72):
    """Decaying 2-D Taylor-Green vortex on a periodic n x n grid of [0, 2 pi]^2,
    rho0 = U0 = 1, p0 = 1/(gamma M^2), mu = 1/Re."""
    L = 2.0 * np.pi
    X, Y = cell_centres_uniform(n, n, L, L)
    p0 = 1.0 / (gamma * mach * mach)
    u = np.sin(X) * np.cos(Y)
    v = -np.cos(X) * np.sin(Y)
    p = p0 + 0.25 * (np.cos(2.0 * X) + np.cos(2.0 * Y))
    rho = np.ones_like(X)
    prob = FlowProblem(kind=NAVIER_STOKES, nx=n, ny=n, lx=L, ly=L, gamma=gamma, prandtl=prandtl,
                       mu=1.0 / reynolds, q_inf=(1.0, 0.0, 0.0, p0 / (gamma - 1.0)),
                       name='taylor-green-%dx%d-Re%g-M%g' % (n, n, reynolds, mach))
    return prob, np.ascontiguousarray(_conservative(rho, u, v, p, gamma))


def kinetic_energy(y):
    """Domain-mean kinetic energy of a state (diagnostic)."""
    return float(np.mean(0.5 * (y[1] ** 2 + y[2] ** 2) / y[0]))


# --- viscous cylinder on a stretched O-grid ---------------------------------

def ogrid_ratio(n_radial, dr_wall, r_wall, r_outer):
    """Geometric stretching ratio such that n_radial cells starting at dr_wall
    reach from r_wall to r_outer (bisection)."""
    lo, hi = 1.0 + 1e-12, 2.0
    target = r_outer - r_wall
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        span = dr_wall * (mid ** n_radial - 1.0) / (mid - 1.0)
        if span > target:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def cylinder_ogrid(n_radial=256, n_theta=512, diameter=1.0, dr_wall=1e-4, r_outer=30.0,
                   mach=0.2, reynolds=100.0, gamma=1.4, prandtl=0.72,
                   sutherland_s=110.4 / 278.0, sutherland=True):
    """Viscous flow past a cylinder on a synthetic curvilinear O-grid.

    i runs clockwise around the cylinder (periodic), j runs outward from the
    no-slip adiabatic wall (j-low) to the far field (j-high), so the grid is
    right-handed.  Free stream rho = 1, p = 1/gamma (sound speed 1), velocity
    M along +x; Re on the diameter sets mu; Sutherland's law with S/T_inf.
    The state starts impulsively from the uniform free stream."""
    r_wall = 0.5 * diameter
    ratio = ogrid_ratio(n_radial, dr_wall, r_wall, r_outer)
    r = r_wall + dr_wall * (ratio ** np.arange(n_radial + 1) - 1.0) / (ratio - 1.0)
    r[-1] = r_outer
    theta = -2.0 * np.pi * np.arange(n_theta + 1) / n_theta
    R, TH = np.meshgrid(r, theta, indexing='ij')   # (ny+1, nx+1)
    xv = np.ascontiguousarray(R * np.cos(TH))
    yv = np.ascontiguousarray(R * np.sin(TH))
    xv[:, -1] = xv[:, 0]
    yv[:, -1] = yv[:, 0]
    rho_inf, p_inf, u_inf = 1.0, 1.0 / gamma, mach
    q_inf = (rho_inf, rho_inf * u_inf, 0.0, p_inf / (gamma - 1.0) + 0.5 * rho_inf * u_inf ** 2)
    mu = rho_inf * u_inf * diameter / reynolds
    prob = FlowProblem(kind=NAVIER_STOKES, nx=n_theta, ny=n_radial, xv=xv, yv=yv,
                       bc=(PERIODIC, PERIODIC, WALL, FARFIELD), gamma=gamma, prandtl=prandtl,
                       mu=mu, t_ref=p_inf / rho_inf, sutherland_s=sutherland_s if sutherland else 0.0,
                       q_inf=q_inf, name='cylinder-ogrid-%dx%d-Re%g-M%g' % (n_radial, n_theta, reynolds, mach))
    y0 = np.empty((4, n_radial, n_theta))
    for k in range(4):
        y0[k] = q_inf[k]
    return prob, y0, ratio


def perturbed_box_grid(nx, ny, lx, ly, amp=0.0, seed=0):
    """Vertices of an [0, lx] x [0, ly] box, optionally with a smooth periodic
    interior perturbation (a curvilinear test grid with periodic closure)."""
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    if amp:
        rng = np.random.default_rng(seed)
        ph = rng.uniform(0, 2 * np.pi, 2)
        X = X + amp * (lx / nx) * np.sin(2 * np.pi * X / lx + ph[0]) * np.sin(2 * np.pi * Y / ly)
        Y = Y + amp * (ly / ny) * np.sin(2 * np.pi * Y / ly + ph[1]) * np.sin(2 * np.pi * X / lx)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def random_smooth_state(prob, seed=0, amp=0.05):
    """A seeded smooth positive-density, positive-pressure state on any grid
    (for parity tests): free stream plus a few random low Fourier modes."""
    rng = np.random.default_rng(seed)
    J, I = np.meshgrid(np.arange(prob.ny), np.arange(prob.nx), indexing='ij')
    s = 2 * np.pi * I / prob.nx
    t = 2 * np.pi * J / prob.ny
    prims = []
    base = [1.0, 0.3, -0.2, 1.0 / prob.gamma]
    for k in range(4):
        fld = np.full(s.shape, base[k])
        for _ in range(3):
            a, b = rng.integers(1, 4, 2)
            ph = rng.uniform(0, 2 * np.pi, 2)
            fld = fld + amp * rng.normal() * np.sin(a * s + ph[0]) * np.cos(b * t + ph[1])
        prims.append(fld)
    rho, u, v, p = prims
    return np.ascontiguousarray(_conservative(rho, u, v, p, prob.gamma))


# --- Lorenz-96 (appendix) ---------------------------------------------------

def lorenz96(n=40, forcing=8.0, seed=0):
    """Lorenz-96 problem with n variables; initial state F + seeded N(0,1) noise."""
    rng = np.random.default_rng(seed)
    prob = FlowProblem(kind=LORENZ96, nx=n, ny=1, lorenz_f=forcing, name='lorenz96-%d' % n)
    return prob, forcing + rng.normal(size=n)


# --- batched instances --------------------------------------------------------

@dataclass
class Instance:
    problem: FlowProblem
    y0: np.ndarray
    cfl: float
    seed: int


def batched_instances(count=64, n_min=32, n_max=384):
    """Independent instances with per-instance seeds: type vortex/Taylor-Green
    (p = 1/2), square side ~ U{n_min..n_max}, vortex centre ~ U([0,10]^2),
    Taylor-Green Re ~ U[100, 5000], CFL ~ U[1, 5]."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(i)
        is_vortex = rng.random() < 0.5
        n = int(rng.integers(n_min, n_max + 1))
        cfl = float(rng.uniform(1.0, 5.0))
        if is_vortex:
            c = rng.uniform(0.0, 10.0, 2)
            prob, y0 = isentropic_vortex(n, centre=(float(c[0]), float(c[1])))
        else:
            re = float(rng.uniform(100.0, 5000.0))
            prob, y0 = taylor_green(n, reynolds=re)
        out.append(Instance(prob, y0, cfl, i))
    return out
