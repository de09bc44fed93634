"""Pins of the oracle integrators (Eq. ROK, Eq. RK, Eqs. Newton/SDIRK_Newton,
Arnoldi of Sec. 2.2.2) against closed forms, textbook identities, brute force
on tiny problems and the paper's observed orders."""
import json
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import coefficients as C
from oracle import core
from oracle import integrators as I
from paper_1607_06834_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), 'golden', 'paper_orders.json')))


class Linear:
    """y' = A y with exact Jacobian-vector products."""
    def __init__(self, A):
        self.A = A

    def f(self, y):
        return self.A @ y

    def jvp(self, y, v, f0, eps):
        return self.A @ v


class L96:
    """Lorenz-96 with either exact (analytic) or FD Jacobian-vector products."""
    def __init__(self, n=40, F=8.0, exact=True):
        self.prob, _ = W.lorenz96(n, F)
        self.exact = exact

    def f(self, u):
        return core.lorenz96_rhs(self.prob, u)

    def jvp(self, u, v, f0, eps):
        if not self.exact:
            return (self.f(u + eps * v) - f0) / eps
        return (np.roll(v, -1) - np.roll(v, 2)) * np.roll(u, 1) + (np.roll(u, -1) - np.roll(u, 2)) * np.roll(v, 1) - v


def _l96_start(T=0.3):
    from scipy.integrate import solve_ivp
    sys = L96()
    y0 = 8.0 * np.ones(40)
    y0[19] += 0.01
    y0 = solve_ivp(lambda t, u: sys.f(u), (0, 3), y0, rtol=1e-12, atol=1e-12, method='DOP853').y[:, -1]
    ref = solve_ivp(lambda t, u: sys.f(u), (0, T), y0, rtol=1e-13, atol=1e-13, method='DOP853').y[:, -1]
    return y0, ref


def _slopes(step, y0, ref, T, ns):
    errs = []
    for n in ns:
        y = y0.copy()
        for _ in range(n):
            y = step(y, T / n)
        errs.append(np.linalg.norm(y - ref))
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)], errs


# ---- coefficient tables ------------------------------------------------------

def _rok_conditions(al, gm, b, g):
    al, gm, b = np.array(al), np.array(gm), np.array(b)
    be = al + gm
    a = al.sum(1)
    bp = be.sum(1)
    s = len(b)
    c = {}
    c['1'] = b.sum() - 1
    c['2'] = b @ bp - (0.5 - g)
    c['3'] = b @ a ** 2 - 1 / 3
    c['4'] = b @ (be @ bp) - (1 / 6 - g + g * g)
    c['5'] = b @ a ** 3 - 1 / 4
    c['6'] = b @ (a * (al @ bp)) - (1 / 8 - g / 3)
    c['7a'] = b @ (al @ a ** 2) - 1 / 12
    c['7b'] = b @ (gm @ a ** 2) + g / 3
    c['8'] = b @ (be @ (be @ bp)) - (1 / 24 - g / 2 + 1.5 * g * g - g ** 3)
    return c


def test_rok4_order_conditions():
    c = _rok_conditions(C.ROK4_ALPHA, C.ROK4_GAMMA_OFFDIAG, C.ROK4_B, C.ROK4_GAMMA)
    for k, v in c.items():
        assert abs(v) <= 2e-15, (k, v)
    # alpha/b are the classical RK4 tableau (M = 0 limit)
    assert np.array_equal(np.array(C.ROK4_ALPHA), np.array(C.RK4_A))
    assert np.allclose(C.ROK4_B, C.RK4_B, rtol=0, atol=1e-17)


def test_rok4_stability_function_L_stable():
    # full-space (M = N) stability function R(z) = 1 + z b^T (I - z B)^{-1} 1,
    # B = alpha + Gamma (diag gamma): order 4 and R(inf) = 0
    B = np.array(C.ROK4_ALPHA) + np.array(C.ROK4_GAMMA_OFFDIAG) + C.ROK4_GAMMA * np.eye(4)
    b = np.array(C.ROK4_B)
    R = lambda z: 1 + z * b @ np.linalg.solve(np.eye(4) - z * B, np.ones(4))
    for z in (1e-2, -1e-2, 2e-2j):
        assert abs(R(z) - np.exp(z)) <= 3 * abs(z) ** 5
    assert abs(R(-1e12)) < 1e-9
    assert max(abs(R(1j * t)) for t in np.linspace(-50, 50, 2001)) <= 1 + 1e-12


def test_esdirk3_order_and_L_stability():
    A, b, c, g = np.array(C.ESDIRK3_A), np.array(C.ESDIRK3_B), np.array(C.ESDIRK3_C), C.ESDIRK3_GAMMA
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15
    assert abs(b @ A @ c - 1 / 6) < 1e-15
    assert np.allclose(A.sum(1), c, atol=1e-15)
    assert np.allclose(A[1:] @ c, 0.5 * c[1:] ** 2, atol=1e-15)   # stage order 2
    assert np.array_equal(A[-1], b)                                 # stiffly accurate
    assert np.allclose(np.diag(A)[1:], g) and A[0, 0] == 0.0
    assert abs(6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) < 1e-14
    R = lambda z: 1 + z * b @ np.linalg.solve(np.eye(4) - z * A, np.ones(4))
    # R(z) ~ c / z at infinity (L-stability): z R(z) settles to a constant
    assert abs(R(-1e6)) < 1e-5 and abs(1e4 * R(-1e4) - 1e6 * R(-1e6)) < 1e-2 * abs(1e6 * R(-1e6))
    assert max(abs(R(1j * t)) for t in np.linspace(-100, 100, 2001)) <= 1 + 1e-12


# ---- inner products ------------------------------------------------------------

def test_pairwise_sum_is_the_balanced_tree():
    import math
    x = np.array([1e16, 1.0, -1e16, 1.0, 3.0])
    # ((x0 + x1) + (x2 + x3)) + ((x4 + 0) + (0 + 0)), each addition rounded
    expect = ((1e16 + 1.0) + (-1e16 + 1.0)) + 3.0
    assert I.pairwise_sum(x) == expect
    rng = np.random.default_rng(5)
    for n in (1, 7, 1000, 4097):
        v = rng.normal(size=n) * 10.0 ** rng.uniform(-5, 5, size=n)
        exact = math.fsum(v)
        depth = max(1, int(np.ceil(np.log2(n))))
        bound = depth * 2.0 ** -53 / (1 - depth * 2.0 ** -53) * np.sum(np.abs(v))
        assert abs(I.pairwise_sum(v) - exact) <= bound
        ints = rng.integers(-1000, 1000, size=n).astype(float)
        assert I.pairwise_sum(ints) == float(ints.sum())
    a, b = rng.normal(size=300), rng.normal(size=300)
    assert abs(I.dot(a, b) - math.fsum(a * b)) <= 1e-13 * np.sum(np.abs(a * b))


# ---- Arnoldi -------------------------------------------------------------------

def test_arnoldi_relations_and_cgs2():
    prob, y = W.isentropic_vortex(16)
    sys = core.System(prob)
    F1 = sys.f(y)
    eps = I.fd_eps(np.linalg.norm(y))
    M = 10
    V, H, meff = I.arnoldi(sys, y, F1, M, eps)
    assert meff == M
    assert np.abs(V @ V.T - np.eye(M)).max() <= 1e-12 * M
    assert np.all(np.tril(H, -2) == 0) and np.all(np.diag(H, -1) > 0)
    Wm = np.stack([sys.jvp(y, V[j].reshape(y.shape), F1, eps).ravel() for j in range(M)])
    assert np.abs(V @ Wm.T - H).max() <= 1e-12 * np.abs(H).max()
    assert np.allclose(V[0], F1.ravel() / np.linalg.norm(F1), atol=1e-15)
    # classical Gram-Schmidt applied twice spans the same space with the same H
    Vc = np.zeros_like(V)
    Vc[0] = F1.ravel() / np.linalg.norm(F1)
    Hc = np.zeros((M, M))
    for j in range(M):
        w = sys.jvp(y, Vc[j].reshape(y.shape), F1, eps).ravel()
        h1 = Vc[:j + 1] @ w; w = w - Vc[:j + 1].T @ h1
        h2 = Vc[:j + 1] @ w; w = w - Vc[:j + 1].T @ h2
        Hc[:j + 1, j] = h1 + h2
        if j + 1 < M:
            Hc[j + 1, j] = np.linalg.norm(w)
            Vc[j + 1] = w / Hc[j + 1, j]
    assert np.abs(Vc.T @ Hc @ Vc - V.T @ H @ V).max() <= 1e-9 * np.abs(H).max()


def test_arnoldi_breakdown_free_stream():
    prob, y = W.isentropic_vortex(8)
    for k in range(4):
        y[k] = prob.q_inf[k]
    V, H, meff = I.arnoldi(core.System(prob), y, core.residual(prob, y), 6, 1e-7)
    assert meff == 0


# ---- ROK step ----------------------------------------------------------------

def test_rok_linear_full_krylov_is_R_of_hA():
    rng = np.random.default_rng(0)
    Q = np.linalg.qr(rng.normal(size=(12, 12)))[0]
    lam = -np.logspace(-1, 3, 12)
    A = Q @ np.diag(lam) @ Q.T
    y0 = rng.normal(size=12)
    h = 0.05
    y1 = I.rok_step(Linear(A), y0, h, 12)
    B = np.array(C.ROK4_ALPHA) + np.array(C.ROK4_GAMMA_OFFDIAG) + C.ROK4_GAMMA * np.eye(4)
    b = np.array(C.ROK4_B)
    Rz = np.array([1 + z * b @ np.linalg.solve(np.eye(4) - z * B, np.ones(4)) for z in h * lam])
    assert np.allclose(y1, Q @ (Rz * (Q.T @ y0)), rtol=1e-11, atol=1e-12)


def test_rok_M0_is_classical_rk4():
    prob, y = W.isentropic_vortex(16)
    sys = core.System(prob)
    h = I.dt_from_cfl(prob, y, 0.5)
    assert np.abs(I.rok_step(sys, y, h, 0) - I.rk_step(sys, y, h)).max() <= 1e-14 * np.abs(y).max()


@pytest.mark.parametrize('n', [4, 8])
def test_rok_equals_dense_w_method(n):
    # Eq. ROK is the W-method (I - h g A) k_i = h F_i + h A sum gamma_ij k_j with
    # A = V H V^T: solve that dense system directly and compare
    prob, y = W.taylor_green(n, reynolds=50.0)
    y = y + 0.02 * W.random_smooth_state(prob, seed=n)
    sys = core.System(prob)
    h = I.dt_from_cfl(prob, y, 3.0)
    info = {}
    M = 6
    y1 = I.rok_step(sys, y, h, M, info=info)
    V, H = info['V'], info['H']
    A = V.T @ H @ V
    N = y.size
    al, gm, b, g = np.array(C.ROK4_ALPHA), np.array(C.ROK4_GAMMA_OFFDIAG), np.array(C.ROK4_B), C.ROK4_GAMMA
    ks = []
    for i in range(4):
        Y = y.ravel() + sum(al[i, j] * ks[j] for j in range(i))
        rhs = h * sys.f(Y.reshape(y.shape)).ravel() + h * A @ sum((gm[i, j] * ks[j] for j in range(i)), np.zeros(N))
        ks.append(np.linalg.solve(np.eye(N) - h * g * A, rhs))
    yd = y.ravel() + sum(b[i] * ks[i] for i in range(4))
    assert np.abs(y1.ravel() - yd).max() <= 1e-12 * np.abs(y).max()


def test_rok_conserves_and_keeps_free_stream():
    prob, y = W.isentropic_vortex(16)
    sys = core.System(prob)
    h = I.dt_from_cfl(prob, y, 5.0)
    y1 = I.rok_step(sys, y, h, 8)
    for k in range(4):
        # each f sums to zero over the cells up to rounding; the FD quotient divides
        # that rounding by eps (~2^-22 here), so the basis vectors, and the step,
        # conserve to about u/eps relative
        assert abs(y1[k].sum() - y[k].sum()) <= 1e-9 * np.abs(y[k]).sum()
    yfs = np.empty_like(y)
    for k in range(4):
        yfs[k] = prob.q_inf[k]
    assert np.array_equal(I.rok_step(sys, yfs, h, 8), yfs)


def test_rok_order_lorenz96_matches_paper():
    y0, ref = _l96_start()
    target = GOLDEN['lorenz96']['theoretical']['ROK']
    observed_paper = GOLDEN['lorenz96']['observed']['ROK']
    sys = L96(exact=False)
    sl, errs = _slopes(lambda y, h: I.rok_step(sys, y, h, 4), y0, ref, 0.3, [16, 32, 64, 128])
    assert abs(sl[-1] - target) < 0.2, (sl, errs)
    assert sl[-1] >= observed_paper - 0.1


def test_rok_split_condition_is_necessary():
    # a table satisfying only the classical Rosenbrock conditions (7a/7b merged)
    # loses an order at M = 4 < N but keeps order 4 at M = N
    from scipy.optimize import least_squares
    g = C.ROK4_GAMMA
    al = np.zeros((4, 4))
    al[1, 0] = 0.4; al[2, 0] = 0.1; al[2, 1] = 0.5; al[3, 0] = 0.2; al[3, 1] = 0.3; al[3, 2] = 0.5
    c = al.sum(1)
    b = np.linalg.solve(np.vstack([c ** 0, c, c ** 2, c ** 3]), [1, 1 / 2, 1 / 3, 1 / 4])

    def res(x):
        gm = np.zeros((4, 4))
        gm[1, 0], gm[2, 0], gm[2, 1], gm[3, 1], gm[3, 2] = x
        gm[3, 0] = 0.3
        cc = _rok_conditions(al, gm, b, g)
        return [cc['2'], cc['4'], cc['6'], cc['7a'] + cc['7b'], cc['8']]
    sol = least_squares(res, np.full(5, -0.3), xtol=1e-15, ftol=1e-15, gtol=1e-15).x
    gm = np.zeros((4, 4))
    gm[1, 0], gm[2, 0], gm[2, 1], gm[3, 1], gm[3, 2] = sol
    gm[3, 0] = 0.3
    assert max(abs(v) for v in res(sol)) < 1e-12
    y0, ref = _l96_start()
    sys = L96(exact=True)
    step = lambda M: (lambda y, h: I.rok_step(sys, y, h, M, gamma=g, alpha=al, gamma_off=gm, b=b))
    sl4, _ = _slopes(step(4), y0, ref, 0.3, [64, 128, 256])
    slN, _ = _slopes(step(40), y0, ref, 0.3, [64, 128, 256])
    ours, _ = _slopes(lambda y, h: I.rok_step(sys, y, h, 4), y0, ref, 0.3, [64, 128, 256])
    assert sl4[-1] < 3.3 and slN[-1] > 3.8 and ours[-1] > 3.9, (sl4, slN, ours)


def test_rok_vortex_against_exact_solution():
    prob, y = W.isentropic_vortex(64)
    sys = core.System(prob)
    h = I.dt_from_cfl(prob, y, 5.0)
    yy = y.copy()
    for _ in range(10):
        yy = I.rok_step(sys, yy, h, 12)
    e_rok = I.l2_error(yy, W.vortex_exact(prob, 10 * h))
    # spatial error floor of this grid: the RK4 solution with a small step
    ys = y.copy()
    hs = h / 8
    for _ in range(80):
        ys = I.rk_step(sys, ys, hs)
    e_sp = I.l2_error(ys, W.vortex_exact(prob, 10 * h))
    assert e_rok < 2.0 * e_sp and e_sp < 5e-3, (e_rok, e_sp)


# ---- RK4, GMRES, ESDIRK ------------------------------------------------------

def test_rk4_exact_on_cubic_and_order():
    class Poly:
        def f(self, y):   # y = (t, x): x' = 4 t^3 is integrated exactly by RK4
            return np.array([1.0, 4.0 * y[0] ** 3])
    y = np.array([0.0, 0.0])
    for _ in range(7):
        y = I.rk_step(Poly(), y, 0.3)
    assert abs(y[1] - (2.1) ** 4) <= 1e-12 * 2.1 ** 4
    y0, ref = _l96_start()
    sl, _ = _slopes(lambda y, h: I.rk_step(L96(), y, h), y0, ref, 0.3, [32, 64, 128])
    assert abs(sl[-1] - GOLDEN['lorenz96']['observed']['ERK4']) < 0.15


def test_gmres_dense():
    rng = np.random.default_rng(3)
    A = np.eye(50) + 0.3 * rng.normal(size=(50, 50)) / np.sqrt(50)
    bvec = rng.normal(size=50)
    x, its, ok = I.gmres(lambda v: A @ v, bvec, m=30, tol=1e-10, max_restarts=5)
    assert ok and np.linalg.norm(A @ x - bvec) <= 1e-10 * np.linalg.norm(bvec)
    assert np.allclose(x, np.linalg.solve(A, bvec), rtol=1e-8, atol=1e-9)


def test_esdirk_linear_is_R_of_hA():
    rng = np.random.default_rng(1)
    Q = np.linalg.qr(rng.normal(size=(10, 10)))[0]
    lam = -np.logspace(-1, 2, 10)
    A = Q @ np.diag(lam) @ Q.T
    y0 = rng.normal(size=10)
    h = 0.1
    y1 = I.esdirk_step(Linear(A), y0, h, gmres_tol=1e-13, newton_tol=1e-14)
    Ab, b = np.array(C.ESDIRK3_A), np.array(C.ESDIRK3_B)
    Rz = np.array([1 + z * b @ np.linalg.solve(np.eye(4) - z * Ab, np.ones(4)) for z in h * lam])
    assert np.allclose(y1, Q @ (Rz * (Q.T @ y0)), rtol=1e-10, atol=1e-11)


def test_esdirk_order3_lorenz96():
    y0, ref = _l96_start()
    sys = L96(exact=True)
    sl, errs = _slopes(lambda y, h: I.esdirk_step(sys, y, h, gmres_tol=1e-12, newton_tol=1e-13),
                       y0, ref, 0.3, [32, 64, 128])
    assert abs(sl[-1] - 3.0) < 0.2, (sl, errs)


# ---- embedded estimates and adaptive steps -------------------------------------

def _trees(order):
    """All rooted trees with `order` nodes, as sorted tuples of child trees."""
    if order == 1:
        return [()]
    out = set()

    def parts(n, maxpart):
        if n == 0:
            yield []
            return
        for k in range(min(n, maxpart), 0, -1):
            for rest in parts(n - k, k):
                yield [k] + rest
    for p in parts(order - 1, order - 1):
        def combos(sizes):
            if not sizes:
                yield ()
                return
            for t in _trees(sizes[0]):
                for rest in combos(sizes[1:]):
                    yield (t,) + rest
        for ch in combos(p):
            out.add(tuple(sorted(ch)))
    return sorted(out)


def _butcher_condition(A, b, tree):
    """sum_i b_i Phi_i(tree) - 1/gamma(tree) in exact rationals."""
    from fractions import Fraction
    s = len(b)

    def phi(t):
        v = [Fraction(1)] * s
        for ch in t:
            pc = phi(ch)
            for i in range(s):
                v[i] *= sum(A[i][j] * pc[j] for j in range(s))
        return v

    def size(t):
        return 1 + sum(size(c) for c in t)

    def gam(t):
        g = size(t)
        for c in t:
            g *= gam(c)
        return g
    ph = phi(tree)
    return sum(b[i] * ph[i] for i in range(s)) - Fraction(1, gam(tree))


def test_dopri5_order_conditions_exact():
    # Butcher's conditions for every rooted tree: order 5 for b (17 trees), order 4
    # for bhat (8 trees), and the order-5 conditions are NOT all met by bhat
    from fractions import Fraction
    A = [[Fraction(x) for x in row] for row in C.DOPRI5_A_EXACT]
    b = [Fraction(x) for x in C.DOPRI5_B_EXACT]
    bh = [Fraction(x) for x in C.DOPRI5_BHAT_EXACT]
    counts = [len(_trees(p)) for p in range(1, 6)]
    assert counts == [1, 1, 2, 4, 9]
    for p in range(1, 6):
        for t in _trees(p):
            assert _butcher_condition(A, b, t) == 0, (p, t)
            if p <= 4:
                assert _butcher_condition(A, bh, t) == 0, (p, t)
    assert any(_butcher_condition(A, bh, t) != 0 for t in _trees(5))
    # the binary64 table is the rounding of the exact one; first same as last
    assert all(float(A[i][j]) == C.DOPRI5_A[i][j] for i in range(7) for j in range(7))
    assert [float(x) for x in b] == list(C.DOPRI5_A[6]) == list(C.DOPRI5_B)


def test_rok_embedded_weights_conditions():
    al = np.array(C.ROK4_ALPHA)
    gm = np.array(C.ROK4_GAMMA_OFFDIAG)
    bh = np.array(C.ROK4_BHAT)
    a = al.sum(axis=1)
    bp = (al + gm).sum(axis=1)
    assert abs(bh.sum() - 1.0) <= 1e-15
    assert abs(bh @ a - 0.5) <= 1e-15
    assert abs(bh @ bp - (0.5 - C.ROK4_GAMMA)) <= 1e-15
    assert bh[3] == 0.0 and np.abs(bh - np.array(C.ROK4_B)).max() > 0.1


def test_rok_embedded_estimate_is_third_order():
    # the estimate sum (b - bhat)_i k_i behaves like C h^3 (order-2 embedded
    # solution) on Lorenz-96 with M = 8 >= 3
    prob, y0 = W.lorenz96(40)
    sys_ = core.System(prob)
    hs = [0.02, 0.01, 0.005]
    es = [np.linalg.norm(I.rok_step_embedded(sys_, y0, h, 8)[1]) for h in hs]
    slopes = [np.log(es[k] / es[k + 1]) / np.log(2.0) for k in range(2)]
    assert all(2.8 < s < 3.3 for s in slopes), slopes


def test_dopri5_step_orders():
    # one step on Lorenz-96 against a fine RK4 reference: the local error falls
    # like h^6, the estimate like h^5
    prob, y0 = W.lorenz96(40)
    sys_ = core.System(prob)
    ref = {}
    for h in (0.02, 0.01):
        yr = y0.copy()
        for _ in range(64):
            yr = I.rk_step(sys_, yr, h / 64)
        ref[h] = yr
    err = {h: np.linalg.norm(I.dopri5_step(sys_, y0, h)[0] - ref[h]) for h in (0.02, 0.01)}
    est = {h: np.linalg.norm(I.dopri5_step(sys_, y0, h)[1]) for h in (0.02, 0.01)}
    assert 5.5 < np.log2(err[0.02] / err[0.01]) < 6.5, err
    assert 4.6 < np.log2(est[0.02] / est[0.01]) < 5.4, est


@pytest.mark.parametrize('method', ['rok', 'dopri5'])
def test_adaptive_integration_tolerance_proportionality(method):
    # tighter tolerances give proportionally smaller global errors and more steps
    prob, y0 = W.lorenz96(40)
    sys_ = core.System(prob)
    T = 0.5
    yr = y0.copy()
    for _ in range(2000):
        yr = I.rk_step(sys_, yr, T / 2000)
    errs, steps = [], []
    for tol in (1e-5, 1e-7, 1e-9):
        if method == 'rok':
            y, st = I.rok_integrate(sys_, y0, T, 0.01, 8, tol, tol)
        else:
            y, st = I.dopri5_integrate(sys_, y0, T, 0.01, tol, tol)
        assert abs(st['t'] - T) <= 1e-12 * T
        errs.append(np.linalg.norm(y - yr) / np.linalg.norm(yr))
        steps.append(st['accepted'])
    assert errs[0] > 10 * errs[1] and errs[1] > 10 * errs[2] and errs[2] < 1e-6, errs
    assert steps[0] < steps[1] < steps[2], steps


# ---- Rosenbrock (ROS4) and Rosenbrock-W (ROW) comparators, Eq. ROS --------------

def _ros_conditions(al, gm, b, g, order):
    """Order conditions of Rosenbrock methods (Hairer & Wanner IV.7, exact
    Jacobian) in the variables of Eq. ROS: beta = alpha + gamma (strictly lower),
    a_i = sum_j alpha_ij, beta'_i = sum_j beta_ij."""
    al, gm, b = np.array(al), np.array(gm), np.array(b)
    be = al + gm
    a, bp = al.sum(1), be.sum(1)
    c = {'1': b.sum() - 1, '2': b @ bp - (0.5 - g)}
    if order >= 3:
        c['3'] = b @ a ** 2 - 1 / 3
        c['4'] = b @ (be @ bp) - (1 / 6 - g + g * g)
    if order >= 4:
        c['5'] = b @ a ** 3 - 1 / 4
        c['6'] = b @ (a * (al @ bp)) - (1 / 8 - g / 3)
        c['7'] = b @ (be @ a ** 2) - (1 / 12 - g / 3)
        c['8'] = b @ (be @ (be @ bp)) - (1 / 24 - g / 2 + 1.5 * g * g - g ** 3)
    return c


def _ros_R(method):
    if method == 'ros4':
        al, gm, b, g = C.ROS4_ALPHA, C.ROS4_GAMMA_OFFDIAG, C.ROS4_B, C.ROS4_GAMMA
    else:
        al, gm, b, g = C.ROW_ALPHA, C.ROW_GAMMA_OFFDIAG, C.ROW_B, C.ROW_GAMMA
    B = np.array(al) + np.array(gm) + g * np.eye(4)
    bb = np.array(b)
    return lambda z: 1 + z * bb @ np.linalg.solve(np.eye(4) - z * B, np.ones(4))


def test_ros4_order_conditions_and_L_stability():
    c = _ros_conditions(C.ROS4_ALPHA, C.ROS4_GAMMA_OFFDIAG, C.ROS4_B, C.ROS4_GAMMA, 4)
    for k, v in c.items():
        assert abs(v) <= 1e-14, (k, v)
    R = _ros_R('ros4')
    for z in (1e-2, -1e-2, 2e-2j):
        assert abs(R(z) - np.exp(z)) <= 3 * abs(z) ** 5
    # L-stable: R(z) -> 0 like 1/z at infinity, |R| <= 1 on the imaginary axis
    assert abs(R(-1e3)) < 1e-2 and abs(R(-1e5)) < abs(R(-1e3)) / 50
    assert max(abs(R(1j * t)) for t in np.linspace(-200, 200, 4001)) <= 1 + 1e-12


def test_row_order3_conditions_embedded_pair_and_L_stability():
    c = _ros_conditions(C.ROW_ALPHA, C.ROW_GAMMA_OFFDIAG, C.ROW_B, C.ROW_GAMMA, 3)
    for k, v in c.items():
        assert abs(v) <= 1e-14, (k, v)
    ch = _ros_conditions(C.ROW_ALPHA, C.ROW_GAMMA_OFFDIAG, C.ROW_BHAT, C.ROW_GAMMA, 3)
    assert abs(ch['1']) <= 1e-14 and abs(ch['2']) <= 1e-14       # embedded weights: order 2
    assert abs(ch['3']) > 1e-3                                   # ... and not 3
    g = C.ROW_GAMMA
    assert abs(6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) < 1e-14
    R = _ros_R('row')
    for z in (1e-2, -1e-2, 2e-2j):
        assert abs(R(z) - np.exp(z)) <= 3 * abs(z) ** 4
    assert abs(R(-1e3)) < 1e-2 and abs(R(-1e5)) < abs(R(-1e3)) / 50
    assert max(abs(R(1j * t)) for t in np.linspace(-200, 200, 4001)) <= 1 + 1e-12


@pytest.mark.parametrize('method', ['ros4', 'row'])
def test_ros_linear_is_R_of_hA(method):
    # on y' = A y one step is y_1 = R(hA) y_0 (R of the tableau, textbook formula):
    # pins the stage structure, including the J term of the right-hand sides
    rng = np.random.default_rng(2)
    Q = np.linalg.qr(rng.normal(size=(10, 10)))[0]
    lam = -np.logspace(-1, 2, 10)
    A = Q @ np.diag(lam) @ Q.T
    y0 = rng.normal(size=10)
    h = 0.1
    y1 = I.ros_step(Linear(A), y0, h, method=method, gmres_tol=1e-14)
    R = _ros_R(method)
    Rz = np.array([R(z) for z in h * lam])
    assert np.allclose(y1, Q @ (Rz * (Q.T @ y0)), rtol=1e-10, atol=1e-11)


def test_ros4_order4_and_row_order3_lorenz96():
    y0, ref = _l96_start()
    sys = L96(exact=True)
    sl, errs = _slopes(lambda y, h: I.ros_step(sys, y, h, method='ros4', gmres_tol=1e-13), y0, ref, 0.3,
                       [16, 32, 64])
    assert abs(sl[-1] - 4.0) < 0.25, (sl, errs)
    sl, errs = _slopes(lambda y, h: I.ros_step(sys, y, h, method='row', gmres_tol=1e-13), y0, ref, 0.3,
                       [16, 32, 64])
    assert abs(sl[-1] - 3.0) < 0.25, (sl, errs)


class L96WrongJacobian(L96):
    """Lorenz-96 whose Jacobian-vector products use J + E, E a fixed matrix."""
    def __init__(self):
        super().__init__(exact=True)
        self.E = 0.5 * np.random.default_rng(5).normal(size=(40, 40)) / np.sqrt(40)

    def jvp(self, u, v, f0, eps):
        return super().jvp(u, v, f0, eps) + self.E @ v


def test_row_keeps_order3_with_a_wrong_jacobian_and_ros4_does_not():
    # the W-property (Sec. 2.2.1): ROW keeps order 3 for any matrix in place of
    # J; ROS4 drops to order 2 (its conditions assume the exact Jacobian)
    y0, ref = _l96_start()
    sys = L96WrongJacobian()
    sl, errs = _slopes(lambda y, h: I.ros_step(sys, y, h, method='row', gmres_tol=1e-13), y0, ref, 0.3,
                       [16, 32, 64])
    assert abs(sl[-1] - 3.0) < 0.25, (sl, errs)
    sl4, errs4 = _slopes(lambda y, h: I.ros_step(sys, y, h, method='ros4', gmres_tol=1e-13), y0, ref, 0.3,
                         [16, 32, 64])
    assert sl4[-1] < 2.5, (sl4, errs4)
