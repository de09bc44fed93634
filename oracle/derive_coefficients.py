"""Derive the method coefficient tables stored in ``oracle/coefficients.py``.

TEST INFRASTRUCTURE ONLY (writes the oracle's own table; the CUDA library
carries its own literal copy and never imports this file).

The paper defines the ROK step (Sec. 2.2.2, Eq. ROK) but prints no
coefficients, and the ESDIRK comparator has none either.  Both tables are
therefore solved here from their order conditions, in 40-digit arithmetic,
and rounded once to binary64.

ROK4 (4 stages, order 4 for Krylov dimension M >= 4)
----------------------------------------------------
Eq. ROK is algebraically a W-method (Sec. 2.2.1 form, h-scaled stages) with
the Jacobian replaced by A = V H V^T = P J P, P the orthogonal projector on
K_M(J, f(y_n)).  For M >= 4 every elementary differential of order <= 4 in
which A multiplies a chain J^k f (k <= 2) equals its exact-Jacobian twin,
because J^k f stays inside K_M.  The single exception at order 4 is
A f''(f, f) = P J P f''(f, f), so the classical Rosenbrock condition for the
tree [[tau, tau]] splits into an alpha-part (= 1/12) and a gamma-part
(= -gamma/3 off the diagonal).  The conditions are

  (1) sum b = 1                        (5) sum b_i a_i^3 = 1/4
  (2) sum b_i beta'_i = 1/2 - g        (6) sum b_i a_i alpha_ij beta'_j = 1/8 - g/3
  (3) sum b_i a_i^2 = 1/3              (7a) sum b_i alpha_ij a_j^2 = 1/12
  (4) sum b_i beta_ij beta'_j          (7b) sum b_i gamma_ij a_j^2 = -g/3
          = 1/6 - g + g^2              (8) sum b_i beta_ij beta_jk beta'_k
                                              = 1/24 - g/2 + 3g^2/2 - g^3

with beta = alpha + gamma (strictly lower), a_i = sum_j alpha_ij,
beta'_i = sum_j beta_ij.  Choices made here:
  * (alpha, b) = classical RK4, so (1), (3), (5), (7a) hold and the M = 0
    limit of the method is the classical RK4 step (Sec. 2.2.2 notes that
    M = 0 reduces ROK to an explicit Runge-Kutta method);
  * g = 0.5728160624821349, the root in the A-stability interval of
    g^4 - 4g^3 + 3g^2 - 2g/3 + 1/24 = 0, which makes the stability function
    of the full-space (M = N) method L-stable;
  * gamma_41 = 3/5 (the free parameter, near the minimum-norm member);
  * gamma_21, gamma_31, gamma_32, gamma_42, gamma_43 from (2), (4), (6),
    (7b), (8) by Newton's method.

ESDIRK3 (4 stages, explicit first stage, order 3, stage order 2,
stiffly accurate, L-stable)
-----------------------------------------------------------------
c = (0, 2g, 3/5, 1), a_21 = a_22 = g, a_ii = g, row 4 = b; stage order 2 on
stage 3 fixes a_32; b_2, b_3 from sum b c = 1/2 and sum b c^2 = 1/3 (order
3 then follows from stage order 2); g is the root in (0.4, 0.5) of the
condition R(inf) = 0, computed symbolically below.

Embedded ROK4 weights (error estimate for adaptive steps)
--------------------------------------------------------
bhat reuses the four stages: sum bhat = 1, sum bhat_i a_i = 1/2 and
sum bhat_i beta'_i = 1/2 - g (order 2 for every Krylov dimension: the first
holds the explicit part at M = 0, the second adds the gamma part inside the
Krylov space), and bhat_4 = 0.  The order-3 and R(inf) = 0 conditions cannot
be added: the main weights b satisfy all of them, so with four stages they
would force bhat = b.  y - yhat = sum (b_i - bhat_i) k_i is then an O(h^3)
local error estimate.

DOPRI5 (comparator with an embedded error estimate)
---------------------------------------------------
The Dormand-Prince 5(4) pair (Dormand & Prince, J. Comput. Appl. Math. 6,
1980), 7 stages, first-same-as-last, written here as exact rationals; the
order conditions it satisfies are checked in the oracle's tests.

ROS4 and ROW (Rosenbrock comparators, Sec. 2.2, Eq. ROS)
---------------------------------------------------------
The paper's ROS4 is a 4-stage, order-4, L-stable Rosenbrock method and its
ROW a 4-stage, order-3, L-stable Rosenbrock-W method (table of methods,
Sec. 3.1); it cites Hairer & Wanner IV.7 for the former and Rang &
Angermann (BIT 45, 2005) for W-methods.  Tables used here:
  * ROS4: the L-stable method of Hairer & Wanner (Solving ODEs II, Sec. IV.7,
    g = 0.57282), whose coefficients are published for the implementation
    form (1/(h g) I - J) u_i = f(y + sum a_ij u_j) + sum (c_ij / h) u_j,
    y_1 = y_0 + sum m_j u_j.  Eq. ROS is recovered exactly (rational
    arithmetic on the published decimals): Gamma = (diag(1/g) - C)^{-1},
    alpha = A Gamma, b = m Gamma (the paper's stages are h-free: k = u / h
    combinations, so alpha and gamma carry over unchanged).
  * ROW: ROS34PW2 of Rang & Angermann, published in the form of Eq. ROS
    (g = 0.435866521508459, the root of 6x^3 - 18x^2 + 9x - 1 in (0.4, 0.5)),
    with its embedded order-2 weights.
The oracle's tests check the order conditions (8 for ROS4, the classical
order-3 set for ROW), L-stability, and the orders reached on Lorenz-96,
for ROW also with a wrong Jacobian (the W-property).

Run ``python oracle/derive_coefficients.py`` to regenerate the table file.
"""
import os

import mpmath as mp
import sympy as sp

mp.mp.dps = 40


def rok4():
    g = [r for r in mp.polyroots([1, -4, 3, mp.mpf(-2) / 3, mp.mpf(1) / 24],
                                 maxsteps=200, extraprec=200)
         if mp.mpf('0.39') < r < mp.mpf('1.28')][0]
    al = {(2, 1): mp.mpf(1) / 2, (3, 1): mp.mpf(0), (3, 2): mp.mpf(1) / 2,
          (4, 1): mp.mpf(0), (4, 2): mp.mpf(0), (4, 3): mp.mpf(1)}
    b = {1: mp.mpf(1) / 6, 2: mp.mpf(1) / 3, 3: mp.mpf(1) / 3, 4: mp.mpf(1) / 6}
    g41 = mp.mpf(3) / 5

    def conds(g21, g31, g32, g42, g43):
        gm = {(2, 1): g21, (3, 1): g31, (3, 2): g32, (4, 1): g41, (4, 2): g42, (4, 3): g43}
        A = lambda i, j: al.get((i, j), mp.mpf(0))
        G = lambda i, j: gm.get((i, j), mp.mpf(0))
        B = lambda i, j: A(i, j) + G(i, j)
        a = lambda i: sum(A(i, j) for j in range(1, i))
        bp = lambda i: sum(B(i, j) for j in range(1, i))
        I = range(1, 5)
        c2 = sum(b[i] * bp(i) for i in I) - (mp.mpf(1) / 2 - g)
        c4 = sum(b[i] * B(i, j) * bp(j) for i in I for j in range(1, i)) - (mp.mpf(1) / 6 - g + g ** 2)
        c6 = sum(b[i] * a(i) * A(i, j) * bp(j) for i in I for j in range(1, i)) - (mp.mpf(1) / 8 - g / 3)
        c7b = sum(b[i] * G(i, j) * a(j) ** 2 for i in I for j in range(1, i)) + g / 3
        c8 = sum(b[i] * B(i, j) * B(j, k) * bp(k) for i in I for j in range(1, i) for k in range(1, j)) \
            - (mp.mpf(1) / 24 - g / 2 + 3 * g ** 2 / 2 - g ** 3)
        return [c2, c4, c6, c7b, c8]

    x0 = [mp.mpf('0.02506863'), mp.mpf('0.24774743'), mp.mpf('-1.40591387'),
          mp.mpf('-0.02036991'), mp.mpf('-1.75033085')]
    sol = mp.findroot(conds, x0, tol=mp.mpf(10) ** -35, maxsteps=100)
    g21, g31, g32, g42, g43 = [sol[k] for k in range(5)]
    gm = {(2, 1): g21, (3, 1): g31, (3, 2): g32, (4, 1): g41, (4, 2): g42, (4, 3): g43}
    alpha = [[al.get((i, j), mp.mpf(0)) for j in range(1, 5)] for i in range(1, 5)]
    gamma = [[gm.get((i, j), mp.mpf(0)) for j in range(1, 5)] for i in range(1, 5)]
    # embedded weights: sum bhat = 1, sum bhat a = 1/2, sum bhat beta' = 1/2 - g, bhat_4 = 0
    a = [sum(alpha[i][j] for j in range(4)) for i in range(4)]
    bp = [sum(alpha[i][j] + gamma[i][j] for j in range(4)) for i in range(4)]
    Mx = mp.matrix([[1, 1, 1, 1], a, bp, [0, 0, 0, 1]])
    rhs = mp.matrix([1, mp.mpf(1) / 2, mp.mpf(1) / 2 - g, 0])
    bhat = mp.lu_solve(Mx, rhs)
    return dict(gamma=g, alpha=alpha, gamma_offdiag=gamma, b=[b[i] for i in range(1, 5)],
                bhat=[mp.chop(bhat[k], tol=mp.mpf(10) ** -30) for k in range(4)])


def esdirk3():
    x = sp.symbols('x', positive=True)
    c3 = sp.Rational(3, 5)
    a32 = (c3 ** 2 / 2 - x * c3) / (2 * x)
    a31 = c3 - x - a32
    b2, b3 = sp.symbols('b2 b3')
    solb = sp.solve([b2 * 2 * x + b3 * c3 + x - sp.Rational(1, 2),
                     b2 * 4 * x ** 2 + b3 * c3 ** 2 + x - sp.Rational(1, 3)], [b2, b3])
    B2, B3 = sp.simplify(solb[b2]), sp.simplify(solb[b3])
    B1 = 1 - B2 - B3 - x
    A = sp.Matrix([[0, 0, 0, 0], [x, x, 0, 0], [a31, a32, x, 0], [B1, B2, B3, x]])
    z = sp.symbols('z')
    R = 1 + z * (sp.Matrix([[B1, B2, B3, x]]) * (sp.eye(4) - z * A).LUsolve(sp.ones(4, 1)))[0]
    Rinf = sp.simplify(sp.limit(sp.simplify(R), z, sp.oo))
    num = sp.numer(sp.together(Rinf))
    poly = sp.Poly(sp.expand(num), x)
    roots = [r for r in sp.Poly(poly).nroots(n=40) if r.is_real and 0.4 < r < 0.5]
    g = mp.mpf(str(roots[0]))
    subs = {x: sp.Float(str(roots[0]), 40)}
    Ar = [[mp.mpf(str(sp.N(A[i, j].subs(subs), 40))) for j in range(4)] for i in range(4)]
    return dict(gamma=g, A=Ar, b=Ar[3], c=[sum(Ar[i]) for i in range(4)], rinf_poly=str(poly.as_expr()))


def dopri5():
    F = sp.Rational
    A = [[0, 0, 0, 0, 0, 0, 0],
         [F(1, 5), 0, 0, 0, 0, 0, 0],
         [F(3, 40), F(9, 40), 0, 0, 0, 0, 0],
         [F(44, 45), F(-56, 15), F(32, 9), 0, 0, 0, 0],
         [F(19372, 6561), F(-25360, 2187), F(64448, 6561), F(-212, 729), 0, 0, 0],
         [F(9017, 3168), F(-355, 33), F(46732, 5247), F(49, 176), F(-5103, 18656), 0, 0],
         [F(35, 384), 0, F(500, 1113), F(125, 192), F(-2187, 6784), F(11, 84), 0]]
    b = [F(35, 384), 0, F(500, 1113), F(125, 192), F(-2187, 6784), F(11, 84), 0]
    bhat = [F(5179, 57600), 0, F(7571, 16695), F(393, 640), F(-92097, 339200), F(187, 2100), F(1, 40)]
    return dict(A=A, b=b, bhat=bhat, c=[sum(r) for r in A])


def ros4():
    F = sp.Rational
    g = F('0.57282')
    A = sp.zeros(4, 4)
    C = sp.zeros(4, 4)
    A[1, 0] = F('2.000000000000000')
    A[2, 0] = F('1.867943637803922')
    A[2, 1] = F('0.2344449711399156')
    A[3, 0], A[3, 1], A[3, 2] = A[2, 0], A[2, 1], 0
    C[1, 0] = F('-7.137615036412310')
    C[2, 0] = F('2.580708087951457')
    C[2, 1] = F('0.6515950076447975')
    C[3, 0] = F('-2.137148994382534')
    C[3, 1] = F('-0.3214669691237626')
    C[3, 2] = F('-0.6949742501781779')
    m = sp.Matrix([[F('2.255570073418735'), F('0.2870493262186792'), F('0.4353179431840180'),
                    F('1.093502252409163')]])
    Gam = (sp.eye(4) / g - C).inv()
    alpha = A * Gam
    b = m * Gam
    off = [[Gam[i, j] if j < i else 0 for j in range(4)] for i in range(4)]
    return dict(gamma=g, alpha=[[alpha[i, j] for j in range(4)] for i in range(4)], gamma_offdiag=off,
                b=[b[0, j] for j in range(4)])


def row():
    F = sp.Rational
    g = F('0.43586652150845900')
    al = [[0, 0, 0, 0],
          [F('0.87173304301691801'), 0, 0, 0],
          [F('0.84457060015369423'), F('-0.11299064236484185'), 0, 0],
          [0, 0, 1, 0]]
    ga = [[0, 0, 0, 0],
          [F('-0.87173304301691801'), 0, 0, 0],
          [F('-0.90338057013044082'), F('0.054180672388095326'), 0, 0],
          [F('0.24212380706095346'), F('-1.2232505839045147'), F('0.54526025533510214'), 0]]
    b = [F('0.24212380706095346'), F('-1.2232505839045147'), F('1.5452602553351020'), F('0.43586652150845900')]
    bhat = [F('0.37810903145819369'), F('-0.096042292212423178'), F('0.5'), F('0.21793326075422950')]
    return dict(gamma=g, alpha=al, gamma_offdiag=ga, b=b, bhat=bhat)


def fmt(v):
    return repr(float(v))


def main():
    r = rok4()
    e = esdirk3()
    d = dopri5()
    ro = ros4()
    rw = row()
    lines = [
        '"""Method coefficient tables of the oracle (binary64).',
        '',
        'TEST INFRASTRUCTURE ONLY.  Written by oracle/derive_coefficients.py; the',
        'derivation and the order conditions are stated in that file.',
        '"""',
        '',
        '# ROK4: Eq. ROK with s = 4; alpha and b are the classical RK4 tableau.',
        'ROK4_GAMMA = ' + fmt(r['gamma']),
        'ROK4_ALPHA = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']' for row in r['alpha']) + ']',
        'ROK4_GAMMA_OFFDIAG = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']'
                                           for row in r['gamma_offdiag']) + ']',
        'ROK4_B = [' + ', '.join(fmt(v) for v in r['b']) + ']',
        '# embedded weights (order 2, bhat_4 = 0): error estimate sum (b - bhat)_i k_i',
        'ROK4_BHAT = [' + ', '.join(fmt(v) for v in r['bhat']) + ']',
        '',
        '# classical RK4 (Sec. 2.1, Eq. RK with a, b below)',
        'RK4_A = [[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]',
        'RK4_B = [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]',
        '',
        '# ESDIRK3: explicit first stage, diagonal gamma, stiffly accurate (b = last row)',
        '# R(inf) = 0 numerator polynomial in gamma: ' + e['rinf_poly'],
        'ESDIRK3_GAMMA = ' + fmt(e['gamma']),
        'ESDIRK3_A = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']' for row in e['A']) + ']',
        'ESDIRK3_B = [' + ', '.join(fmt(v) for v in e['b']) + ']',
        'ESDIRK3_C = [' + ', '.join(fmt(v) for v in e['c']) + ']',
        '',
        '# DOPRI5: Dormand-Prince 5(4), first same as last (row 7 of A = b)',
        'DOPRI5_A = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']' for row in d['A']) + ']',
        'DOPRI5_B = [' + ', '.join(fmt(v) for v in d['b']) + ']',
        'DOPRI5_BHAT = [' + ', '.join(fmt(v) for v in d['bhat']) + ']',
        'DOPRI5_C = [' + ', '.join(fmt(v) for v in d['c']) + ']',
        '# exact rationals of the same table (order-condition checks)',
        'DOPRI5_A_EXACT = ' + repr([[str(v) for v in row] for row in d['A']]),
        'DOPRI5_B_EXACT = ' + repr([str(v) for v in d['b']]),
        'DOPRI5_BHAT_EXACT = ' + repr([str(v) for v in d['bhat']]),
        '',
        '# ROS4: L-stable Rosenbrock method of order 4 (Hairer & Wanner), Eq. ROS form',
        'ROS4_GAMMA = ' + fmt(ro['gamma']),
        'ROS4_ALPHA = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']' for row in ro['alpha']) + ']',
        'ROS4_GAMMA_OFFDIAG = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']'
                                           for row in ro['gamma_offdiag']) + ']',
        'ROS4_B = [' + ', '.join(fmt(v) for v in ro['b']) + ']',
        '',
        '# ROW: ROS34PW2 (Rang & Angermann), Rosenbrock-W method of order 3, Eq. ROS form',
        'ROW_GAMMA = ' + fmt(rw['gamma']),
        'ROW_ALPHA = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']' for row in rw['alpha']) + ']',
        'ROW_GAMMA_OFFDIAG = [' + ', '.join('[' + ', '.join(fmt(v) for v in row) + ']'
                                          for row in rw['gamma_offdiag']) + ']',
        'ROW_B = [' + ', '.join(fmt(v) for v in rw['b']) + ']',
        'ROW_BHAT = [' + ', '.join(fmt(v) for v in rw['bhat']) + ']',
        '',
    ]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'coefficients.py')
    with open(out, 'w') as fh:
        fh.write('\n'.join(lines))
    print('\n'.join(lines))


if __name__ == '__main__':
    main()
