"""FP64 NumPy oracle of the time integrators: Arnoldi (modified Gram-Schmidt),
the ROK step, classical RK4, ESDIRK3 with Newton-GMRES, the finite-difference
epsilon, the CFL time step and the L2 error metric.

TEST INFRASTRUCTURE ONLY.  Each function follows the paper's equations in
their printed order.  Every inner product of the ROK step is the pairwise sum of
the rounded entrywise products (``dot``) and the small dense systems are solved
by a plain LU, so that the floating-point result of a step is fully specified.
Readings of silent points are stated where they are used.

The integrators see the problem only through a ``System``: ``sys.f(y)`` and
``sys.jvp(y, v, f0, eps)`` (``core.System`` wraps the C residual).
"""
import math

import numpy as np

from . import coefficients as C
from . import core

MACH_EPS = 2.0 ** -52


def pairwise_sum(x, dtype=np.float64):
    """Sum of the entries of x by pairwise summation (Higham): a balanced binary
    tree over the index range, x zero-padded to a power-of-two length, each level
    adding entry 2i and entry 2i+1, every addition rounded in `dtype`.  This fixes
    one rounding of the sum."""
    x = np.ravel(np.asarray(x, dtype=dtype))
    n = 1
    while n < x.size:
        n *= 2
    buf = np.zeros(n, dtype=dtype)
    buf[:x.size] = x
    while buf.size > 1:
        buf = buf[0::2] + buf[1::2]
    return buf[0]


def _cx(*xs):
    """True when any argument is complex: the integrators then run on the
    analytic continuation (complex-step derivatives), every comparison and
    every rounding-to-a-power-of-two on real parts; products are not
    conjugated, so inner products and norms stay analytic."""
    return any(np.iscomplexobj(x) for x in xs)


def dot(a, b, dtype=np.float64):
    """Inner product: the entrywise products rounded in `dtype`, summed pairwise."""
    if _cx(a, b):
        dtype = np.complex128
    a = np.ravel(np.asarray(a, dtype=dtype))
    b = np.ravel(np.asarray(b, dtype=dtype))
    r = pairwise_sum(a * b, dtype)
    if dtype == np.complex128:
        return complex(r)
    return float(r) if dtype == np.float64 else r


def norm(a, dtype=np.float64):
    if _cx(a):
        return complex(np.sqrt(dot(a, a)))
    if dtype == np.float64:
        return math.sqrt(dot(a, a))
    return np.sqrt(dot(a, a, dtype))


def fd_eps(ynorm, vnorm=1.0):
    """Finite-difference increment for Eq. matvecFD.

    The paper asks for the optimum trade-off between truncation and
    round-off (citing Knoll & Keyes) without a formula.  Reading:
    eps = sqrt(u (1 + ||y||)) / ||v||, u = 2^-52, rounded to the nearest
    power of two (log-scale rounding), which keeps it within sqrt(2) of the
    Knoll-Keyes value and makes eps*v and the division by eps exact."""
    x = math.sqrt(MACH_EPS * (1.0 + ynorm)) / vnorm
    m, e = math.frexp(x)           # x = m 2^e, 0.5 <= m < 1
    if m < math.sqrt(0.5):
        e -= 1
    return math.ldexp(1.0, e)


def arnoldi(sys, y, F1, M, eps, breakdown_tol=None, basis=np.float64):
    """Modified-Gram-Schmidt Arnoldi (Sec. 2.2.2): V (M_eff x N, rows orthonormal)
    and H = V^T J V (M_eff x M_eff, upper Hessenberg) of K_M(J, f(y_n)), with the
    Jacobian applied by Eq. matvecFD.  Returns (V, H, M_eff).

    Readings: beta = ||F1|| = 0 gives M_eff = 0; the basis is cut at column j
    when h_{j+1,j} <= tol * ||J v_j|| (a scale-consistent test; tol 1e-12 in
    binary64, 1e-5 in binary32); h_{j+1,j} > 0 makes V unique; normalisation
    multiplies by 1/h.

    basis = np.float32 is the mixed-precision form: the basis is stored and the
    Gram-Schmidt arithmetic (inner products, updates, norms) is done in binary32;
    each JVP result (a binary64 difference quotient at y + eps v) is rounded to
    binary32 before orthogonalisation; H is kept in binary64."""
    if breakdown_tol is None:
        breakdown_tol = 1e-12 if basis == np.float64 else 1e-5
    T = np.complex128 if _cx(y, F1) else basis
    N = F1.size
    V = np.zeros((M, N), dtype=T)
    H = np.zeros((M, M), dtype=np.complex128 if T == np.complex128 else np.float64)
    w = np.asarray(F1, dtype=T).ravel()
    beta = norm(w, T)
    if M == 0 or not np.real(beta) > 0.0:
        return V[:0], H[:0, :0], 0
    V[0] = w * (T(1.0) / beta)
    y_flat = y.ravel()
    shape = y.shape
    f0 = F1
    meff = M
    for j in range(M):
        vj = V[j].astype(np.complex128 if T == np.complex128 else np.float64).reshape(shape)
        w = np.asarray(sys.jvp(y_flat.reshape(shape), vj, f0, eps), dtype=T).ravel()
        wnorm0 = norm(w, T)
        for i in range(j + 1):
            hij = dot(V[i], w, T)
            H[i, j] = hij if T == np.complex128 else float(hij)
            w = w - T(hij) * V[i]
        if j + 1 < M:
            hn = norm(w, T)
            if not np.real(hn) > breakdown_tol * np.real(wnorm0):
                meff = j + 1
                break
            H[j + 1, j] = hn if T == np.complex128 else float(hn)
            V[j + 1] = w * (T(1.0) / hn)
    return V[:meff], H[:meff, :meff], meff


def lu_factor(A):
    """LU factorisation with partial pivoting (first largest |pivot|), row
    interchanges applied to the whole rows; returns (LU, piv) with the unit
    lower factor below the diagonal.  Plain loops."""
    A = np.array(A, dtype=np.complex128 if _cx(A) else np.float64)
    m = A.shape[0]
    piv = np.zeros(m, dtype=int)
    for k in range(m):
        p = k + int(np.argmax(np.abs(np.real(A[k:, k]))))
        piv[k] = p
        if p != k:
            A[[k, p]] = A[[p, k]]
        d = A[k, k]
        for i in range(k + 1, m):
            l = A[i, k] / d
            A[i, k] = l
            for j in range(k + 1, m):
                A[i, j] = A[i, j] - l * A[k, j]
    return A, piv


def lu_solve(LU, piv, b):
    """Solve with the factors of lu_factor: interchanges, unit-lower forward and
    upper backward substitution, plain loops."""
    x = [complex(v) if _cx(LU, b) else float(v) for v in b]
    m = len(x)
    for k in range(m):
        p = int(piv[k])
        if p != k:
            x[k], x[p] = x[p], x[k]
    for i in range(m):
        t = x[i]
        for j in range(i):
            t = t - LU[i, j] * x[j]
        x[i] = t
    for i in range(m - 1, -1, -1):
        t = x[i]
        for j in range(i + 1, m):
            t = t - LU[i, j] * x[j]
        x[i] = t / LU[i, i]
    return np.array(x)


def rok_step(sys, y, h, M, gamma=None, alpha=None, gamma_off=None, b=None, info=None, basis=np.float64,
             stages=None):
    """One step of the Rosenbrock-Krylov method, Eq. ROK (Sec. 2.2.2):

        F_i      = f(y_n + sum_{j<i} alpha_ij k_j)
        phi_i    = V^T F_i
        lambda_i = (I - h g H)^{-1} (h phi_i + h H sum_{j<i} gamma_ij lambda_j)
        k_i      = V lambda_i + h (F_i - V phi_i)
        y_{n+1}  = y_n + sum_i b_i k_i

    with V, H from Arnoldi on K_M(J_n, f(y_n)).  The M x M system is solved by
    LU with partial pivoting (lu_factor/lu_solve); k_i is evaluated as
    V (lambda_i - h phi_i) + h F_i, the same vector grouped once; sums over the
    basis run in basis order.  With basis = np.float32 only the basis storage and
    Gram-Schmidt are binary32 (see arnoldi); phi, the stage solves and the stage
    vectors read the basis exactly as binary64 and compute in binary64.
    `stages` (a list, optional) receives the stage vectors k_i."""
    g = C.ROK4_GAMMA if gamma is None else gamma
    al = np.array(C.ROK4_ALPHA if alpha is None else alpha)
    gm = np.array(C.ROK4_GAMMA_OFFDIAG if gamma_off is None else gamma_off)
    bb = np.array(C.ROK4_B if b is None else b)
    s = len(bb)
    shape = y.shape
    yf = y.ravel()
    F1 = np.asarray(sys.f(y))
    eps = fd_eps(float(np.real(norm(yf))))   # a constant of the step (real part)
    V, H, meff = arnoldi(sys, y, F1, M, eps, basis=basis)
    cx = _cx(y, F1)
    V = V.astype(np.complex128 if cx else np.float64)
    LU, piv = lu_factor(np.eye(meff) - (h * g) * H)
    ks, lams = [], []
    for i in range(s):
        if i == 0:
            F = F1.ravel()
        else:
            Y = yf.copy()
            for j in range(i):
                if al[i, j] != 0.0:
                    Y = Y + al[i, j] * ks[j]
            F = np.asarray(sys.f(Y.reshape(shape))).ravel()
        phi = np.array([dot(V[m], F) for m in range(meff)])
        acc = np.zeros(meff, dtype=V.dtype)
        for j in range(i):
            acc = acc + gm[i, j] * lams[j]
        rhs = np.zeros(meff, dtype=V.dtype)
        for r in range(meff):
            t = 0.0
            for c in range(meff):
                t = t + H[r, c] * acc[c]
            rhs[r] = h * phi[r] + h * t
        lam = lu_solve(LU, piv, rhs) if meff > 0 else np.zeros(0, dtype=V.dtype)
        cvec = lam - h * phi
        k = np.zeros_like(yf)
        for m in range(meff):
            k = k + cvec[m] * V[m]
        k = k + h * F
        ks.append(k)
        lams.append(lam)
    ynew = yf.copy()
    for i in range(s):
        ynew = ynew + bb[i] * ks[i]
    if info is not None:
        info.update(m_eff=meff, eps=eps, H=H, V=V)
    if stages is not None:
        stages.extend(ks)
    return ynew.reshape(shape)


# ---- embedded error estimates and adaptive steps ----------------------------------

def wrms(e, y, ynew, atol, rtol):
    """Weighted RMS norm of an error estimate (Hairer, Norsett & Wanner, Solving
    ODEs I, Sec. II.4): sqrt(sum_i (e_i / sc_i)^2 / N), sc_i = atol + rtol
    max(|y_i|, |ynew_i|), the sum pairwise."""
    e, y, ynew = np.ravel(e), np.ravel(y), np.ravel(ynew)
    sc = atol + rtol * np.maximum(np.abs(y), np.abs(ynew))
    r = e / sc
    return math.sqrt(pairwise_sum(r * r) / r.size)


def rok_step_embedded(sys, y, h, M):
    """ROK4 step (Eq. ROK) and its error estimate y_{n+1} - yhat =
    sum_i (b_i - bhat_i) k_i, bhat the embedded order-2 weights."""
    ks = []
    ynew = rok_step(sys, y, h, M, stages=ks)
    d = [C.ROK4_B[i] - C.ROK4_BHAT[i] for i in range(4)]
    e = np.zeros(y.size)
    for q in range(4):
        e = e + d[q] * ks[q]
    return ynew, e.reshape(y.shape)


def dopri5_step(sys, y, h, k1=None):
    """One Dormand-Prince 5(4) step: k_i = f(y + sum_j (h a_ij) k_j), y_{n+1} = the
    7th stage state y + sum_j (h b_j) k_j, error estimate sum_j (h (b_j - bhat_j)) k_j;
    k_7 = f(y_{n+1}) is returned for the next step (first same as last)."""
    A, b, bh = C.DOPRI5_A, C.DOPRI5_B, C.DOPRI5_BHAT
    ks = [np.asarray(sys.f(y)) if k1 is None else k1]
    Y = y
    for i in range(1, 7):
        Y = y.copy()
        for j in range(i):
            if A[i][j] != 0.0:
                Y = Y + (h * A[i][j]) * ks[j]
        ks.append(np.asarray(sys.f(Y)))
    e = np.zeros_like(y)
    for j in range(7):
        d = b[j] - bh[j]
        if d != 0.0:
            e = e + (h * d) * ks[j]
    return Y, e, ks[6]


def integrate_adaptive(try_step, y0, T, h0, q, atol, rtol, safety=0.9, facmin=0.2, facmax=5.0,
                       max_steps=100000):
    """Adaptive step-size control (Hairer, Norsett & Wanner I, Sec. II.4).
    try_step(y, h) -> (ynew, e); a step is accepted when err = wrms(e) <= 1;
    the next step is h min(facmax, max(facmin, safety err^(-1/(q+1)))), q the
    order of the embedded solution, never larger than h right after a
    rejection; a non-finite err rejects with facmin.  The last step ends at T.
    Returns (y, dict(accepted, rejected, t, h))."""
    t, h, y = 0.0, h0, y0
    acc = rej = 0
    after_reject = False
    while T - t > 1e-12 * T and acc + rej < max_steps:
        if t + h > T:
            h = T - t
        ynew, e = try_step(y, h)
        err = wrms(e, y, ynew, atol, rtol)
        if not math.isfinite(err):
            fac = facmin
        elif err == 0.0:
            fac = facmax
        else:
            fac = min(facmax, max(facmin, safety * err ** (-1.0 / (q + 1))))
        if math.isfinite(err) and err <= 1.0:
            t = t + h
            y = ynew
            acc += 1
            if after_reject:
                fac = min(fac, 1.0)
            after_reject = False
        else:
            rej += 1
            after_reject = True
            fac = min(fac, 1.0)
        h = h * fac
    return y, dict(accepted=acc, rejected=rej, t=t, h=h)


def rok_integrate(sys, y0, T, h0, M, atol, rtol, **kw):
    """Adaptive ROK4 with the embedded order-2 estimate (exponent 1/3)."""
    return integrate_adaptive(lambda y, h: rok_step_embedded(sys, y, h, M), y0, T, h0, 2, atol, rtol, **kw)


def dopri5_integrate(sys, y0, T, h0, atol, rtol, **kw):
    """Adaptive DOPRI5 (embedded order 4, exponent 1/5).  First same as last:
    the k_7 of a step is f(y_{n+1}), reused as k_1 when y_{n+1} is accepted; after
    a rejection the k_1 of the retried step is reused."""
    known = []   # (state, f(state)) of the last attempt's start and result

    def try_step(y, h):
        k1 = next((k for a, k in known if a is y), None)
        if k1 is None:
            k1 = np.asarray(sys.f(y))
        ynew, e, k7 = dopri5_step(sys, y, h, k1)
        known[:] = [(y, k1), (ynew, k7)]
        return ynew, e

    return integrate_adaptive(try_step, y0, T, h0, 4, atol, rtol, **kw)


def rk_step(sys, y, h, A=None, b=None):
    """Explicit Runge-Kutta step, Eq. RK (Sec. 2.1): k_i = f(y_n + h sum_j a_ij k_j),
    y_{n+1} = y_n + h sum_j b_j k_j; classical RK4 by default."""
    A = np.array(C.RK4_A if A is None else A)
    b = np.array(C.RK4_B if b is None else b)
    ks = []
    for i in range(len(b)):
        acc = np.zeros_like(y)
        for j in range(i):
            if A[i, j] != 0.0:
                acc = acc + A[i, j] * ks[j]
        ks.append(np.asarray(sys.f(y + h * acc)))
    acc = np.zeros_like(y)
    for j in range(len(b)):
        acc = acc + b[j] * ks[j]
    return y + h * acc


def gmres(matvec, rhs, m=30, tol=1e-6, max_restarts=5):
    """Restarted GMRES(m), no preconditioner, x0 = 0, modified Gram-Schmidt
    Arnoldi, least-squares on the (j+2) x (j+1) Hessenberg each iteration.
    Stops when ||rhs - A x|| <= tol ||rhs||.  Returns (x, iterations, converged)."""
    n = rhs.size
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(rhs))
    if bnorm == 0.0:
        return x, 0, True
    its = 0
    for _cycle in range(max_restarts + 1):
        r = rhs - matvec(x) if its else rhs.copy()
        beta = float(np.linalg.norm(r))
        if beta <= tol * bnorm:
            return x, its, True
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        yls = None
        for j in range(m):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(V[i], w))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            its += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            yls = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = float(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ yls))
            if res <= tol * bnorm or H[j + 1, j] == 0.0:
                x = x + V[:j + 1].T @ yls
                return x, its, True
            V[j + 1] = w / H[j + 1, j]
        x = x + V[:m].T @ yls
    r = rhs - matvec(x)
    return x, its, float(np.linalg.norm(r)) <= tol * bnorm


def esdirk_step(sys, y, h, gmres_m=30, gmres_tol=1e-6, gmres_restarts=5, newton_tol=1e-10,
                newton_max=10, info=None):
    """ESDIRK3 step (Sec. 2.1, Eqs. RK, Newton, SDIRK_Newton, Newton_Jac_Matrix):
    k_1 = f(y_n); for i >= 2 solve k_i = f(xi_i + h g k_i), xi_i = y_n + h sum_{j<i} a_ij k_j,
    by Newton with the matrix I - h g J_n (J_n at y_n, applied by Eq. matvecFD) and
    GMRES for each Newton correction; y_{n+1} = y_n + h sum b_j k_j.

    Readings: predictor k_i^0 = k_{i-1}; Newton stops when
    h g ||dk|| <= newton_tol ||xi_i + h g k_i|| or after newton_max iterations."""
    A = np.array(C.ESDIRK3_A)
    b = np.array(C.ESDIRK3_B)
    g = C.ESDIRK3_GAMMA
    shape = y.shape
    yf = y.ravel()
    F0 = np.asarray(sys.f(y)).ravel()
    eps = fd_eps(float(np.linalg.norm(yf)))

    def jv(v):
        return np.asarray(sys.jvp(y, v.reshape(shape), F0.reshape(shape), eps)).ravel()

    def op(v):
        return v - (h * g) * jv(v)

    ks = [F0]
    newton_its, gmres_its, ok = 0, 0, True
    for i in range(1, len(b)):
        xi = yf.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                xi = xi + (h * A[i, j]) * ks[j]
        k = ks[-1].copy()
        conv = False
        for _it in range(newton_max):
            Yst = xi + (h * g) * k
            G = k - np.asarray(sys.f(Yst.reshape(shape))).ravel()
            dk, its, _c = gmres(op, -G, gmres_m, gmres_tol, gmres_restarts)
            gmres_its += its
            newton_its += 1
            k = k + dk
            if (h * g) * float(np.linalg.norm(dk)) <= newton_tol * float(np.linalg.norm(xi + (h * g) * k)):
                conv = True
                break
        ok = ok and conv
        ks.append(k)
    ynew = yf.copy()
    acc = np.zeros_like(yf)
    for j in range(len(b)):
        acc = acc + b[j] * ks[j]
    ynew = ynew + h * acc
    if info is not None:
        info.update(newton_iters=newton_its, gmres_iters=gmres_its, converged=ok, eps=eps)
    return ynew.reshape(shape)


def ros_step(sys, y, h, method='ros4', gmres_m=30, gmres_tol=1e-6, gmres_restarts=5, info=None):
    """Rosenbrock step, Sec. 2.2, Eq. ROS (method 'ros4') or Rosenbrock-W step
    of the same form (method 'row'):
        Y_i = y_n + h sum_{j<i} alpha_ij k_j,
        (I - h g J_n) k_i = f(Y_i) + h J_n sum_{j<i} gamma_ij k_j   (Eq. ROS_stage_eq),
        y_{n+1} = y_n + h sum_j b_j k_j,
    J_n at y_n applied by Eq. matvecFD (eps from ||y_n||), every stage system
    solved by GMRES(m) from x0 = 0 (the matrix-free setting of the paper's
    experiments).  Reading: the J_n term of the right-hand side is one more
    Jacobian-vector product per stage (skipped when all gamma_ij of the stage
    vanish)."""
    if method == 'ros4':
        al, ga, b, g = np.array(C.ROS4_ALPHA), np.array(C.ROS4_GAMMA_OFFDIAG), np.array(C.ROS4_B), C.ROS4_GAMMA
    elif method == 'row':
        al, ga, b, g = np.array(C.ROW_ALPHA), np.array(C.ROW_GAMMA_OFFDIAG), np.array(C.ROW_B), C.ROW_GAMMA
    else:
        raise ValueError(method)
    shape = y.shape
    yf = y.ravel()
    F0 = np.asarray(sys.f(y)).ravel()
    eps = fd_eps(float(np.linalg.norm(yf)))

    def jv(v):
        return np.asarray(sys.jvp(y, v.reshape(shape), F0.reshape(shape), eps)).ravel()

    def op(v):
        return v - (h * g) * jv(v)

    ks = []
    gmres_its, ok = 0, True
    for i in range(len(b)):
        if i == 0:
            rhs = F0.copy()
        else:
            Yi = yf.copy()
            for j in range(i):
                if al[i, j] != 0.0:
                    Yi = Yi + (h * al[i, j]) * ks[j]
            rhs = np.asarray(sys.f(Yi.reshape(shape))).ravel()
            u = np.zeros_like(yf)
            any_g = False
            for j in range(i):
                if ga[i, j] != 0.0:
                    u = u + ga[i, j] * ks[j]
                    any_g = True
            if any_g:
                rhs = rhs + h * jv(u)
        k, its, conv = gmres(op, rhs, gmres_m, gmres_tol, gmres_restarts)
        gmres_its += its
        ok = ok and conv
        ks.append(k)
    acc = np.zeros_like(yf)
    for j in range(len(b)):
        acc = acc + b[j] * ks[j]
    ynew = yf + h * acc
    if info is not None:
        info.update(gmres_iters=gmres_its, converged=ok, eps=eps)
    return ynew.reshape(shape)


def dt_from_cfl(prob, y, cfl):
    """Time step from a CFL number (the paper does not define one).  Reading:
    dt = CFL / max_cells [ (|u.S_i| + c|S_i|)/Vol + (|u.S_j| + c|S_j|)/Vol
                           + 2 nu_eff (|S_i|^2 + |S_j|^2)/Vol^2 ],
    S_i, S_j the mean face-area vectors of the cell's i and j faces,
    nu_eff = max(4/3, gamma/Pr) mu / rho (zero for Euler)."""
    if prob.kind == 2:
        return cfl / (np.max(np.abs(y)) + 1.0)
    g = prob.gamma
    rho = y[0]
    u = y[1] / rho
    v = y[2] / rho
    p = (g - 1.0) * (y[3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(g * p / rho)
    if prob.xv is None:
        dx, dy = prob.lx / prob.nx, prob.ly / prob.ny
        six, siy = np.full(rho.shape, dy), np.zeros(rho.shape)
        sjx, sjy = np.zeros(rho.shape), np.full(rho.shape, dx)
        vol = np.full(rho.shape, dx * dy)
    else:
        xv, yv = prob.xv, prob.yv
        # i-face area vectors (e_y, -e_x) at i and i+1, averaged
        exi = xv[1:, :] - xv[:-1, :]
        eyi = yv[1:, :] - yv[:-1, :]
        six = 0.5 * (eyi[:, :-1] + eyi[:, 1:])
        siy = 0.5 * (-exi[:, :-1] - exi[:, 1:])
        exj = xv[:, 1:] - xv[:, :-1]
        eyj = yv[:, 1:] - yv[:, :-1]
        sjx = 0.5 * (-eyj[:-1, :] - eyj[1:, :])
        sjy = 0.5 * (exj[:-1, :] + exj[1:, :])
        vol = core.cell_volumes(prob)
    si2 = six * six + siy * siy
    sj2 = sjx * sjx + sjy * sjy
    lam = (np.abs(u * six + v * siy) + c * np.sqrt(si2)) / vol + (np.abs(u * sjx + v * sjy) + c * np.sqrt(sj2)) / vol
    if prob.kind == 1 and prob.mu > 0.0:
        T = p / rho
        if prob.sutherland_s > 0.0:
            t = T / prob.t_ref
            mu = prob.mu * t ** 1.5 * (1.0 + prob.sutherland_s) / (t + prob.sutherland_s)
        else:
            mu = prob.mu
        nu = max(4.0 / 3.0, g / prob.prandtl) * mu / rho
        lam = lam + 2.0 * nu * (si2 + sj2) / (vol * vol)
    return float(cfl / np.max(lam))


def l2_error(y, yref, relative=True):
    """Error metric of Sec. 4.1: ||y_N - y_ref||_2 over the full state vector
    (relative to ||y_ref||_2 when ``relative``)."""
    e = float(np.linalg.norm((y - yref).ravel()))
    return e / float(np.linalg.norm(yref.ravel())) if relative else e
