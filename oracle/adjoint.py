"""Discrete adjoints for gradients of a final-time functional: the transposed
Jacobian of the residual, the viscosity derivative of the residual, and the
reverse of one ROK4 step (Sec. 2.2.2, Eq. ROK) with finite-difference
Jacobian-vector products (Eq. matvecFD).

TEST INFRASTRUCTURE ONLY.  Plain NumPy, binary64, written out step by step.

residual_vjp: u^T J(y) from exact Jacobian columns, each the complex-step
derivative Im f(y + i h e) / h of the C residual.  Columns are taken in groups:
the residual of a cell depends only on cells within two cells along each grid
direction (MUSCL) and the diagonal neighbours (viscous diamond), so cells
whose indices agree modulo p >= 5 in both directions never share a residual
row; one complex evaluation per (class, variable) gives all their columns at
once, and every row knows which class member it belongs to.

rok_step_vjp: the step is recomputed with every intermediate kept, then each
statement is reversed in the opposite order.  The increment eps of the
finite-difference quotient is a constant of the step (it is chosen from
||y_n|| and rounded to a power of two, a step function of y_n).
"""
import numpy as np

from . import coefficients as C
from . import core
from . import integrators as I


def _period(n, periodic):
    """Smallest class period >= 5 that tiles a periodic direction exactly."""
    if not periodic:
        return 5
    for p in range(5, n + 1):
        if n % p == 0:
            return p
    return n


def residual_vjp(prob, y, u):
    """J(y)^T u for the residual f of `prob` (shape prob.shape)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    if prob.kind == 2:
        # Lorenz-96: f_i = (y_{i+1} - y_{i-2}) y_{i-1} - y_i + F
        r = np.roll
        return (r(u, 1) * r(y, 2) - r(u, -2) * r(y, -1) + r(u, -1) * (r(y, -2) - r(y, 1)) - u)
    nx, ny = prob.nx, prob.ny
    per_x = prob.bc[0] == 0
    per_y = prob.bc[2] == 0
    px, py = _period(nx, per_x), _period(ny, per_y)
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    out = np.zeros((4, ny, nx))
    for ci in range(px):
        # the class member at or after i - 2 (the only one a row can depend on)
        ai = ii + (ci - ii + 2) % px - 2
        ai = ai % nx if per_x else np.clip(ai, 0, nx - 1)
        for cj in range(py):
            aj = jj + (cj - jj + 2) % py - 2
            aj = aj % ny if per_y else np.clip(aj, 0, ny - 1)
            members = ((ii % px) == ci) & ((jj % py) == cj)
            if not members.any():
                continue
            AI = np.broadcast_to(ai, (ny, nx))
            AJ = np.broadcast_to(aj, (ny, nx))
            for q in range(4):
                e = np.zeros((4, ny, nx))
                e[q][members] = 1.0
                D = core.jvp_exact(prob, y, e)          # D[:, r] = d f_r / d y_{q, member(r)}
                contrib = np.sum(D * u, axis=0)         # per row cell r
                np.add.at(out[q], (AJ, AI), contrib)
    return out


def residual_dmu(prob, y):
    """d f / d mu, mu the constant viscosity or, under Sutherland's law
    (Sec. 3.2), the viscosity at t_ref: every cell's viscosity is mu times a
    function of its temperature, the viscous flux is linear in the face
    viscosity and the heat flux goes through k = mu_face gamma / ((gamma - 1) Pr),
    so f is affine in mu and the derivative is f(y; mu = 1) - f(y; mu = 0)."""
    if prob.kind != 1:
        return np.zeros(prob.shape)
    p1 = type(prob)(**{**prob.__dict__, 'mu': 1.0})
    p0 = type(prob)(**{**prob.__dict__, 'mu': 0.0})
    return core.residual(p1, y) - core.residual(p0, y)


def _forward(prob, y, h, M):
    """The FD-JVP ROK4 step of integrators.rok_step, every intermediate kept."""
    g, al, gm, bb = C.ROK4_GAMMA, np.array(C.ROK4_ALPHA), np.array(C.ROK4_GAMMA_OFFDIAG), np.array(C.ROK4_B)
    s = len(bb)
    shape = y.shape
    yf = y.ravel()
    sys_ = core.System(prob)
    F1 = np.asarray(sys_.f(y)).ravel()
    eps = I.fd_eps(I.norm(yf))
    N = yf.size
    V = np.zeros((M, N))
    H = np.zeros((M, M))
    Wfin = np.zeros((M, N))     # w of column j after its Gram-Schmidt passes
    meff = 0
    beta = I.norm(F1)
    if M > 0 and beta > 0.0:
        V[0] = F1 * (1.0 / beta)
        meff = M
        for j in range(M):
            w = core.jvp_fd(prob, y, V[j].reshape(shape), F1.reshape(shape), eps).ravel()
            wnorm0 = I.norm(w)
            for i in range(j + 1):
                hij = I.dot(V[i], w)
                H[i, j] = hij
                w = w - hij * V[i]
            Wfin[j] = w
            if j + 1 < M:
                hn = I.norm(w)
                if not hn > 1e-12 * wnorm0:
                    meff = j + 1
                    break
                H[j + 1, j] = hn
                V[j + 1] = w * (1.0 / hn)
    V, H, Wfin = V[:meff], H[:meff, :meff], Wfin[:meff]
    L = np.eye(meff) - (h * g) * H
    LU, piv = I.lu_factor(L)
    ks, lams, phis, accs, Fs, Ys = [], [], [], [], [], []
    for i in range(s):
        if i == 0:
            Y, F = yf, F1
        else:
            Y = yf.copy()
            for j in range(i):
                if al[i, j] != 0.0:
                    Y = Y + al[i, j] * ks[j]
            F = np.asarray(sys_.f(Y.reshape(shape))).ravel()
        phi = np.array([I.dot(V[m], F) for m in range(meff)])
        acc = np.zeros(meff)
        for j in range(i):
            acc = acc + gm[i, j] * lams[j]
        rhs = h * phi + h * (H @ acc) if meff else np.zeros(0)
        lam = I.lu_solve(LU, piv, rhs) if meff else np.zeros(0)
        k = V.T @ (lam - h * phi) + h * F if meff else h * F
        ks.append(k)
        lams.append(lam)
        phis.append(phi)
        accs.append(acc)
        Fs.append(F)
        Ys.append(Y)
    ynew = yf.copy()
    for i in range(s):
        ynew = ynew + bb[i] * ks[i]
    return dict(eps=eps, F1=F1, V=V, H=H, Wfin=Wfin, meff=meff, beta=beta, L=L, ks=ks, lams=lams, phis=phis,
                accs=accs, Fs=Fs, Ys=Ys, ynew=ynew.reshape(shape))


def rok_step_vjp(prob, y, h, M, ybar):
    """Reverse of one FD-JVP ROK4 step: given ybar = dJ/dy_{n+1}, returns
    (dJ/dy_n, dJ/dmu) (mu: the constant viscosity; 0 for Euler), the step
    recomputed from y_n.  eps is held constant."""
    g, al, gm, bb = C.ROK4_GAMMA, np.array(C.ROK4_ALPHA), np.array(C.ROK4_GAMMA_OFFDIAG), np.array(C.ROK4_B)
    s = len(bb)
    shape = y.shape
    fw = _forward(prob, y, h, M)
    eps, V, H, m = fw['eps'], fw['V'], fw['H'], fw['meff']
    yb = np.asarray(ybar, dtype=np.float64).ravel().copy()
    yfl = y.ravel()
    kb = [bb[i] * yb for i in range(s)]          # y_{n+1} = y_n + sum b_i k_i
    Vb = np.zeros_like(V)
    Hb = np.zeros_like(H)
    lamb = [np.zeros(m) for _ in range(s)]
    F1b = np.zeros_like(yb)
    mub = 0.0
    visc = prob.kind == 1
    for i in range(s - 1, -1, -1):
        lam, phi, acc, F = fw['lams'][i], fw['phis'][i], fw['accs'][i], fw['Fs'][i]
        Fb = h * kb[i]                            # k_i = V^T c_i + h F_i, c_i = lam_i - h phi_i
        phib = np.zeros(m)
        if m:
            c = lam - h * phi
            cb = V @ kb[i]
            Vb += np.outer(c, kb[i])
            lamb[i] = lamb[i] + cb
            phib = phib - h * cb
            # lam_i = L^{-1} rhs_i, L = I - h g H
            rhsb = np.linalg.solve(fw['L'].T, lamb[i])
            Hb += (h * g) * np.outer(rhsb, lam)
            # rhs_i = h phi_i + h H acc_i
            phib = phib + h * rhsb
            Hb += h * np.outer(rhsb, acc)
            accb = h * (H.T @ rhsb)
            for j in range(i):
                lamb[j] = lamb[j] + gm[i, j] * accb
            # phi_i = V F_i
            Vb += np.outer(phib, F)
            Fb = Fb + V.T @ phib
        if i == 0:
            F1b = F1b + Fb
        else:
            Y = fw['Ys'][i].reshape(shape)
            Yb = residual_vjp(prob, Y, Fb.reshape(shape)).ravel()
            if visc:
                mub += float(np.sum(Fb * residual_dmu(prob, Y).ravel()))
            yb = yb + Yb
            for j in range(i):
                if al[i, j] != 0.0:
                    kb[j] = kb[j] + al[i, j] * Yb
    # Arnoldi, columns in reverse
    for j in range(m - 1, -1, -1):
        wb = np.zeros_like(yb)
        if j + 1 < m:                             # v_{j+1} = w / hn, hn = ||w||
            v, hn = V[j + 1], H[j + 1, j]
            wb = Vb[j + 1] / hn - (np.dot(v, Vb[j + 1]) / hn) * v + Hb[j + 1, j] * v
        wcur = fw['Wfin'][j]
        for i in range(j, -1, -1):                # w <- w - h_ij v_i, h_ij = <v_i, w>
            hij = H[i, j]
            wprev = wcur + hij * V[i]
            hb = Hb[i, j] - np.dot(V[i], wb)
            Vb[i] = Vb[i] - hij * wb + hb * wprev
            wb = wb + hb * V[i]
            wcur = wprev
        # w_0 = (f(y + eps v_j) - F1) / eps
        Ypert = (yfl + eps * V[j]).reshape(shape)
        gvec = residual_vjp(prob, Ypert, wb.reshape(shape)).ravel()
        if visc:
            mub += float(np.sum(wb * residual_dmu(prob, Ypert).ravel())) / eps
        Vb[j] = Vb[j] + gvec
        yb = yb + gvec / eps
        F1b = F1b - wb / eps
    if m:                                          # v_1 = F1 / beta, beta = ||F1||
        v, beta = V[0], fw['beta']
        F1b = F1b + Vb[0] / beta - (np.dot(v, Vb[0]) / beta) * v
    yb = yb + residual_vjp(prob, y, F1b.reshape(shape)).ravel()
    if visc:
        mub += float(np.sum(F1b * residual_dmu(prob, y).ravel()))
    return yb.reshape(shape), mub
