/*
 * FP64 CPU oracle for the semi-discrete compressible Euler / Navier-Stokes
 * right-hand side f(y) of the IVP y' = f(y) (Sec. 2, Eq. ode) and for the
 * finite-difference Jacobian-vector product (Sec. 2.3, Eq. matvecFD).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table
 * or constant generator with the CUDA path.
 *
 * What it computes (Sec. 3.2, Eq. Nav_Stokes, and the setting of Sec. 4.2):
 *   - cell-centred finite volume on a structured grid (uniform box, or
 *     curvilinear quadrilaterals given by vertex coordinates);
 *   - second-order MUSCL reconstruction of the primitive variables
 *     (rho, u, v, p), kappa-scheme, with NO limiter (Sec. 4.2: no flux
 *     limiter is employed);
 *   - Roe's approximate Riemann solver for the inviscid face flux;
 *   - central viscous flux: stress tensor with the Stokes hypothesis and
 *     Fourier heat flux (Eq. Nav_Stokes, tau_ij and q_i), face gradients
 *     by Green-Gauss on the face "diamond" (two cell centres, two vertices);
 *   - optional Sutherland viscosity (Sec. 4.2 uses Sutherland's law);
 *   - boundary conditions by two layers of ghost cells: periodic,
 *     no-slip adiabatic wall (mirror), far-field (free-stream ghosts).
 *
 * Readings of places where the paper is silent (each one listed in the
 * design notes): ideal gas with R = 1 so T = p/rho; Pr and gamma are
 * parameters; kappa and the entropy-fix coefficient are parameters; the
 * Harten entropy fix acts on the two acoustic waves with
 * delta = efix * (|q_n| + c) of the Roe-averaged state; the
 * energy equation is the standard one (the printed energy line multiplies
 * div q by k and the stress work by mu a second time, which is read as a
 * typesetting slip).
 *
 * Every expression below is written out in one fixed evaluation order and
 * must be compiled with -ffp-contract=off so that no multiply-add is fused:
 * the residual is then a deterministic function of its input bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Scalar of every state-dependent quantity.  The file is compiled twice: with
 * real_t = double (the residual and the FD-JVP), and with ORACLE_COMPLEX,
 * real_t = double complex, for the complex-step derivative
 * J v = Im f(y + i h v) / h (Squire & Trapp 1998), which is exact to rounding
 * (no difference of nearly equal numbers).  |x| continues analytically as
 * x sign(Re x) and every branch compares real parts. */
#ifdef ORACLE_COMPLEX
#include <complex.h>
typedef double complex real_t;
#define RSQRT(x) csqrt(x)
#define RABS(x) (creal(x) < 0.0 ? -(x) : (x))
#define RLT(a, b) (creal(a) < creal(b))
#else
typedef double real_t;
#define RSQRT(x) sqrt(x)
#define RABS(x) fabs(x)
#define RLT(a, b) ((a) < (b))
#endif

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_FARFIELD = 2 };

typedef struct {
    int nx, ny;          /* cells; i (x / first grid index) runs fastest  */
    int curvilinear;     /* 0: uniform box of spacing dx, dy             */
    int viscous;         /* 0: Euler, 1: Navier-Stokes                   */
    int bc[4];           /* i-low, i-high, j-low, j-high                 */
    double dx, dy;       /* uniform spacing when curvilinear == 0        */
    const double *xv;    /* (ny+1)*(nx+1) vertex x, index j*(nx+1)+i      */
    const double *yv;    /* (ny+1)*(nx+1) vertex y                        */
    double gamma, prandtl;
    double mu_ref;       /* viscosity at t_ref (constant mu if suth_s<=0) */
    double t_ref;        /* reference temperature for Sutherland's law   */
    double suth_s;       /* Sutherland constant S / t_ref; <= 0: const mu */
    double q_inf[4];     /* free stream, conservative                    */
    double kappa;        /* MUSCL kappa                                  */
    double efix;         /* Harten entropy-fix coefficient               */
} oracle_problem;

/* primitive state of one (possibly ghost) cell */
typedef struct { real_t r, u, v, p, T, mu; } prim;

#define NG 2

/* Every loop marked with this macro writes each entry from its own inputs
 * only (grid rows, faces or vector entries are independent).  The CPU
 * baseline build (-fopenmp) runs such loops over threads; the test build
 * ignores the pragma.  Either way every entry is the same sequence of
 * operations, so both builds give the same bits. */
#define ROWS_IN_PARALLEL _Pragma("omp parallel for schedule(static)")

static real_t sutherland(const oracle_problem *P, real_t T)
{
    if (P->suth_s <= 0.0) return P->mu_ref;
    real_t t = T * (1.0 / P->t_ref);
    return P->mu_ref * (t * RSQRT(t)) * ((1.0 + P->suth_s) / (t + P->suth_s));
}

static prim to_prim(const oracle_problem *P, real_t rho, real_t mx, real_t my, real_t E)
{
    prim w;
    real_t rinv = 1.0 / rho;
    w.r = rho;
    w.u = mx * rinv;
    w.v = my * rinv;
    w.p = (P->gamma - 1.0) * (E - 0.5 * (mx * w.u + my * w.v));
    w.T = w.p * rinv;
    w.mu = P->viscous ? sutherland(P, w.T) : 0.0;
    return w;
}

static prim mirror(prim w) { w.u = -w.u; w.v = -w.v; return w; }

/* extended-array index, ghosts included: i in [-2, nx+1], j in [-2, ny+1] */
#define EX(i, j) (((j) + NG) * (nx + 2 * NG) + ((i) + NG))

static void fill_prims(const oracle_problem *P, const real_t *q, prim *W)
{
    const int nx = P->nx, ny = P->ny;
    const size_t nc = (size_t)nx * ny;
    prim inf = to_prim(P, P->q_inf[0], P->q_inf[1], P->q_inf[2], P->q_inf[3]);
    ROWS_IN_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            W[EX(i, j)] = to_prim(P, q[c], q[nc + c], q[2 * nc + c], q[3 * nc + c]);
        }
    /* j ghosts for interior columns */
    for (int g = 1; g <= NG; ++g)
        for (int i = 0; i < nx; ++i) {
            switch (P->bc[2]) {
            case BC_PERIODIC: W[EX(i, -g)] = W[EX(i, ny - g)]; break;
            case BC_WALL:     W[EX(i, -g)] = mirror(W[EX(i, g - 1)]); break;
            default:          W[EX(i, -g)] = inf; break;
            }
            switch (P->bc[3]) {
            case BC_PERIODIC: W[EX(i, ny - 1 + g)] = W[EX(i, g - 1)]; break;
            case BC_WALL:     W[EX(i, ny - 1 + g)] = mirror(W[EX(i, ny - g)]); break;
            default:          W[EX(i, ny - 1 + g)] = inf; break;
            }
        }
    /* i ghosts for every row, ghost rows included */
    for (int j = -NG; j < ny + NG; ++j)
        for (int g = 1; g <= NG; ++g) {
            switch (P->bc[0]) {
            case BC_PERIODIC: W[EX(-g, j)] = W[EX(nx - g, j)]; break;
            case BC_WALL:     W[EX(-g, j)] = mirror(W[EX(g - 1, j)]); break;
            default:          W[EX(-g, j)] = inf; break;
            }
            switch (P->bc[1]) {
            case BC_PERIODIC: W[EX(nx - 1 + g, j)] = W[EX(g - 1, j)]; break;
            case BC_WALL:     W[EX(nx - 1 + g, j)] = mirror(W[EX(nx - g, j)]); break;
            default:          W[EX(nx - 1 + g, j)] = inf; break;
            }
        }
}

/* kappa-MUSCL, no limiter, on one primitive variable.  m2, m1 | p1, p2 are
 * the four cells along the grid line, the face sits between m1 and p1. */
static void muscl(real_t m2, real_t m1, real_t p1, real_t p2, double c_lo, double c_hi,
                  real_t *wl, real_t *wr)
{
    real_t dl = m1 - m2, dc = p1 - m1, dr = p2 - p1;
    *wl = (m1 + c_lo * dl) + c_hi * dc;
    *wr = (p1 - c_lo * dr) - c_hi * dc;
}

static real_t harten(real_t lam, real_t delta)
{
    real_t a = RABS(lam);
    if (RLT(a, delta)) a = (a * a + delta * delta) / (2.0 * delta);
    return a;
}

/* Roe flux through a face of unit normal (nx, ny), primitive L/R states
 * WL = (rho, u, v, p).  Result F = 1/2 (F(L) + F(R)) - 1/2 sum |lam| a r. */
static void roe(const real_t *WL, const real_t *WR, double nx, double ny,
                real_t gm1, double inv_gm1, double efix, real_t *F)
{
    real_t rL = WL[0], uL = WL[1], vL = WL[2], pL = WL[3];
    real_t rR = WR[0], uR = WR[1], vR = WR[2], pR = WR[3];
    real_t qnL = uL * nx + vL * ny;
    real_t qnR = uR * nx + vR * ny;
    /* rho H = E + p on each side */
    real_t eL = (pL * inv_gm1 + rL * (0.5 * (uL * uL + vL * vL))) + pL;
    real_t eR = (pR * inv_gm1 + rR * (0.5 * (uR * uR + vR * vR))) + pR;

    /* Roe averages with weights RSQRT(rho): wl = sL/(sL+sR) = rL sR / (sL sR (sL+sR)),
     * H~ = (sL HL + sR HR)/(sL+sR) = (eL sR + eR sL) / (sL sR (sL+sR)) */
    real_t sL = RSQRT(rL), sR = RSQRT(rR);
    real_t rt = sL * sR;
    real_t den = 1.0 / (rt * (sL + sR));
    real_t wl = (rL * sR) * den, wr = (rR * sL) * den;
    real_t ut = wl * uL + wr * uR;
    real_t vt = wl * vL + wr * vR;
    real_t Ht = (eL * sR + eR * sL) * den;
    real_t kt = 0.5 * (ut * ut + vt * vt);
    real_t ct2 = gm1 * (Ht - kt);
    real_t ct = RSQRT(ct2);
    real_t qnt = ut * nx + vt * ny;

    real_t drho = rR - rL, dp = pR - pL, du = uR - uL, dv = vR - vL, dqn = qnR - qnL;
    real_t inv_c2 = 1.0 / ct2;
    real_t rcdq = rt * ct * dqn;
    real_t a1 = 0.5 * (dp - rcdq) * inv_c2;
    real_t a2 = drho - dp * inv_c2;
    real_t a3 = 0.5 * (dp + rcdq) * inv_c2;

    /* Harten's entropy fix on the two acoustic (genuinely nonlinear) waves */
    real_t delta = efix * (RABS(qnt) + ct);
    real_t l1 = harten(qnt - ct, delta);
    real_t l2 = RABS(qnt);
    real_t l3 = harten(qnt + ct, delta);

    /* sum_k |lam_k| a_k r_k with the eigenvectors r_1,3 = (1, u -+ c n, H -+ c q_n),
     * r_2 = (1, u, k), shear r_s = (0, du - dq_n n, u.du - q_n dq_n), grouped by
     * the wave sums sA = A1 + A3 and dA = A3 - A1 */
    real_t A1 = l1 * a1, A2 = l2 * a2, A3 = l3 * a3, As = l2 * rt;
    real_t sA = A1 + A3, dA = A3 - A1;
    real_t D0 = sA + A2;
    real_t D1 = (ut * D0 + (ct * nx) * dA) + As * (du - dqn * nx);
    real_t D2 = (vt * D0 + (ct * ny) * dA) + As * (dv - dqn * ny);
    real_t D3 = ((Ht * sA + kt * A2) + (ct * qnt) * dA) + As * ((ut * du + vt * dv) - qnt * dqn);

    real_t mL = rL * qnL, mR = rR * qnR;
    real_t FL1 = mL * uL + pL * nx, FR1 = mR * uR + pR * nx;
    real_t FL2 = mL * vL + pL * ny, FR2 = mR * vR + pR * ny;
    F[0] = 0.5 * ((mL + mR) - D0);
    F[1] = 0.5 * ((FL1 + FR1) - D1);
    F[2] = 0.5 * ((FL2 + FR2) - D2);
    F[3] = 0.5 * ((qnL * eL + qnR * eR) - D3);
}

/* viscous face flux (tau . n, u . tau . n - q . n) for unit normal n;
 * g = (ux, uy, vx, vy, Tx, Ty) are face gradients. */
static void viscous(const real_t *g, real_t mu_f, real_t u_f, real_t v_f, double nx, double ny,
                    real_t kfac, double c23, real_t *Fv)
{
    real_t ux = g[0], uy = g[1], vx = g[2], vy = g[3], Tx = g[4], Ty = g[5];
    real_t div = ux + vy;
    real_t txx = mu_f * (2.0 * ux - c23 * div);
    real_t tyy = mu_f * (2.0 * vy - c23 * div);
    real_t txy = mu_f * (uy + vx);
    real_t tnx = txx * nx + txy * ny;
    real_t tny = txy * nx + tyy * ny;
    real_t kf = mu_f * kfac;
    real_t dTn = Tx * nx + Ty * ny;
    Fv[0] = 0.0;
    Fv[1] = tnx;
    Fv[2] = tny;
    Fv[3] = (u_f * tnx + v_f * tny) + kf * dTn;
}

static real_t pget(const prim *w, int k)
{
    switch (k) { case 0: return w->r; case 1: return w->u; case 2: return w->v; default: return w->p; }
}

/* 2x2 vertex average of the four cells around vertex (i, j) */
static void vertex_vals(const oracle_problem *P, const prim *W, int i, int j, real_t *uvT)
{
    const int nx = P->nx;
    const prim *a = &W[EX(i - 1, j - 1)], *b = &W[EX(i, j - 1)], *c = &W[EX(i - 1, j)], *d = &W[EX(i, j)];
    uvT[0] = 0.25 * (((a->u + b->u) + c->u) + d->u);
    uvT[1] = 0.25 * (((a->v + b->v) + c->v) + d->v);
    uvT[2] = 0.25 * (((a->T + b->T) + c->T) + d->T);
}

/* ---- curvilinear geometry ------------------------------------------------ */
typedef struct {
    double *cx, *cy;       /* cell centres, ghost layer 1 included, (nx+2)*(ny+2) */
    double *inv_vol;       /* nx*ny */
    /* i-faces: (nx+1)*ny, j-faces: nx*(ny+1): unit normal, length, diamond coefficients */
    double *in_x, *in_y, *il, *ic[4];
    double *jn_x, *jn_y, *jl, *jc[4];
} geom;

#define VX(i, j) xv[(size_t)(j) * (nx + 1) + (i)]
#define VY(i, j) yv[(size_t)(j) * (nx + 1) + (i)]
#define CI(i, j) (((j) + 1) * (nx + 2) + ((i) + 1))

/* vertex coordinates extended by one layer: periodic sides wrap with the
 * period offset, other sides extrapolate linearly along the grid line */
static void vert_ext(const oracle_problem *P, int i, int j, double *x, double *y)
{
    const int nx = P->nx, ny = P->ny;
    const double *xv = P->xv, *yv = P->yv;
    double ox = 0.0, oy = 0.0;
    if (i < 0 || i > nx) {
        if (P->bc[0] == BC_PERIODIC) {
            int jj = j < 0 ? 0 : (j > ny ? ny : j);
            double px = VX(nx, jj) - VX(0, jj), py = VY(nx, jj) - VY(0, jj);
            if (i < 0) { i += nx; ox -= px; oy -= py; } else { i -= nx; ox += px; oy += py; }
        } else {
            double ax, ay, bx, by;
            int i0 = i < 0 ? 0 : nx, i1 = i < 0 ? 1 : nx - 1;
            vert_ext(P, i0, j, &ax, &ay);
            vert_ext(P, i1, j, &bx, &by);
            *x = 2.0 * ax - bx; *y = 2.0 * ay - by;
            return;
        }
    }
    if (j < 0 || j > ny) {
        if (P->bc[2] == BC_PERIODIC) {
            double px = VX(i, ny) - VX(i, 0), py = VY(i, ny) - VY(i, 0);
            if (j < 0) { j += ny; ox -= px; oy -= py; } else { j -= ny; ox += px; oy += py; }
        } else {
            int j0 = j < 0 ? 0 : ny, j1 = j < 0 ? 1 : ny - 1;
            *x = (2.0 * VX(i, j0) - VX(i, j1)) + ox;
            *y = (2.0 * VY(i, j0) - VY(i, j1)) + oy;
            return;
        }
    }
    *x = VX(i, j) + ox;
    *y = VY(i, j) + oy;
}

static void diamond(double p0x, double p0y, double p1x, double p1y, double p2x, double p2y,
                    double p3x, double p3y, double *c)
{
    /* quadrilateral P0 (cell L), P1 (vertex), P2 (cell R), P3 (vertex), counter-clockwise;
     * Green-Gauss with trapezoidal edges: grad = [dC*c0 + dV*c1, dC*c2 + dV*c3],
     * dC = phi(P2) - phi(P0), dV = phi(P3) - phi(P1). */
    double d1x = p2x - p0x, d1y = p2y - p0y, d2x = p3x - p1x, d2y = p3y - p1y;
    double inv2a = 1.0 / (d1x * d2y - d1y * d2x);
    c[0] = d2y * inv2a;
    c[1] = -d1y * inv2a;
    c[2] = -d2x * inv2a;
    c[3] = d1x * inv2a;
}

static void build_geom(const oracle_problem *P, geom *G)
{
    const int nx = P->nx, ny = P->ny;
    size_t nce = (size_t)(nx + 2) * (ny + 2), nfi = (size_t)(nx + 1) * ny, nfj = (size_t)nx * (ny + 1);
    G->cx = malloc(nce * sizeof(double)); G->cy = malloc(nce * sizeof(double));
    G->inv_vol = malloc((size_t)nx * ny * sizeof(double));
    G->in_x = malloc(nfi * sizeof(double)); G->in_y = malloc(nfi * sizeof(double)); G->il = malloc(nfi * sizeof(double));
    G->jn_x = malloc(nfj * sizeof(double)); G->jn_y = malloc(nfj * sizeof(double)); G->jl = malloc(nfj * sizeof(double));
    for (int k = 0; k < 4; ++k) { G->ic[k] = malloc(nfi * sizeof(double)); G->jc[k] = malloc(nfj * sizeof(double)); }

    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            double x0, y0, x1, y1, x2, y2, x3, y3;
            vert_ext(P, i, j, &x0, &y0); vert_ext(P, i + 1, j, &x1, &y1);
            vert_ext(P, i + 1, j + 1, &x2, &y2); vert_ext(P, i, j + 1, &x3, &y3);
            G->cx[CI(i, j)] = 0.25 * (((x0 + x1) + x2) + x3);
            G->cy[CI(i, j)] = 0.25 * (((y0 + y1) + y2) + y3);
            if (i >= 0 && i < nx && j >= 0 && j < ny) {
                /* quadrilateral area from its diagonals */
                double area = 0.5 * ((x2 - x0) * (y3 - y1) - (y2 - y0) * (x3 - x1));
                G->inv_vol[(size_t)j * nx + i] = 1.0 / area;
            }
        }
    const double *xv = P->xv, *yv = P->yv;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t f = (size_t)j * (nx + 1) + i;
            double ex = VX(i, j + 1) - VX(i, j), ey = VY(i, j + 1) - VY(i, j);
            double len = sqrt(ex * ex + ey * ey);
            G->il[f] = len; G->in_x[f] = ey / len; G->in_y[f] = -ex / len;
            double c[4];
            diamond(G->cx[CI(i - 1, j)], G->cy[CI(i - 1, j)], VX(i, j), VY(i, j),
                    G->cx[CI(i, j)], G->cy[CI(i, j)], VX(i, j + 1), VY(i, j + 1), c);
            for (int k = 0; k < 4; ++k) G->ic[k][f] = c[k];
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t f = (size_t)j * nx + i;
            double ex = VX(i + 1, j) - VX(i, j), ey = VY(i + 1, j) - VY(i, j);
            double len = sqrt(ex * ex + ey * ey);
            G->jl[f] = len; G->jn_x[f] = -ey / len; G->jn_y[f] = ex / len;
            double c[4];
            diamond(G->cx[CI(i, j - 1)], G->cy[CI(i, j - 1)], VX(i + 1, j), VY(i + 1, j),
                    G->cx[CI(i, j)], G->cy[CI(i, j)], VX(i, j), VY(i, j), c);
            for (int k = 0; k < 4; ++k) G->jc[k][f] = c[k];
        }
}

static void free_geom(geom *G)
{
    free(G->cx); free(G->cy); free(G->inv_vol);
    free(G->in_x); free(G->in_y); free(G->il); free(G->jn_x); free(G->jn_y); free(G->jl);
    for (int k = 0; k < 4; ++k) { free(G->ic[k]); free(G->jc[k]); }
}

/* one face: MUSCL states, Roe flux, viscous flux; total (F_inv - F_visc) */
static void face_flux(const oracle_problem *P, const prim *m2, const prim *m1, const prim *p1,
                      const prim *p2, double nx_, double ny_, const real_t *grad, real_t *F)
{
    const double gm1 = P->gamma - 1.0, inv_gm1 = 1.0 / gm1;
    const double c_lo = 0.25 * (1.0 - P->kappa), c_hi = 0.25 * (1.0 + P->kappa);
    real_t WL[4], WR[4];
    for (int k = 0; k < 4; ++k)
        muscl(pget(m2, k), pget(m1, k), pget(p1, k), pget(p2, k), c_lo, c_hi, &WL[k], &WR[k]);
    roe(WL, WR, nx_, ny_, gm1, inv_gm1, P->efix, F);
    if (P->viscous) {
        const double kfac = P->gamma / (gm1 * P->prandtl), c23 = 2.0 / 3.0;
        real_t Fv[4];
        real_t mu_f = 0.5 * (m1->mu + p1->mu);
        real_t u_f = 0.5 * (m1->u + p1->u), v_f = 0.5 * (m1->v + p1->v);
        viscous(grad, mu_f, u_f, v_f, nx_, ny_, kfac, c23, Fv);
        for (int k = 0; k < 4; ++k) F[k] = F[k] - Fv[k];
    }
}

static int residual_impl(const oracle_problem *P, const real_t *q, real_t *f)
{
    const int nx = P->nx, ny = P->ny;
    if (nx < 1 || ny < 1) return 0;
    const size_t nc = (size_t)nx * ny;
    prim *W = malloc((size_t)(nx + 2 * NG) * (ny + 2 * NG) * sizeof(prim));
    real_t *FX = malloc((size_t)4 * (nx + 1) * ny * sizeof(real_t));
    real_t *FY = malloc((size_t)4 * nx * (ny + 1) * sizeof(real_t));
    if (!W || !FX || !FY) { free(W); free(FX); free(FY); return -1; }
    fill_prims(P, q, W);
    const size_t nfi = (size_t)(nx + 1) * ny, nfj = (size_t)nx * (ny + 1);
    geom G;
    if (P->curvilinear) build_geom(P, &G);

    const double rdx = 1.0 / P->dx, rdy = 1.0 / P->dy;
    const double q_rdx = 0.25 * rdx, q_rdy = 0.25 * rdy;

    /* i-faces: between cells (i-1, j) and (i, j) */
    ROWS_IN_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t fidx = (size_t)j * (nx + 1) + i;
            const prim *L = &W[EX(i - 1, j)], *R = &W[EX(i, j)];
            real_t g[6] = {0, 0, 0, 0, 0, 0};
            double nx_ = 1.0, ny_ = 0.0;
            if (P->curvilinear) { nx_ = G.in_x[fidx]; ny_ = G.in_y[fidx]; }
            if (P->viscous) {
                if (!P->curvilinear) {
                    const prim *ln = &W[EX(i - 1, j + 1)], *rn = &W[EX(i, j + 1)];
                    const prim *ls = &W[EX(i - 1, j - 1)], *rs = &W[EX(i, j - 1)];
                    g[0] = (R->u - L->u) * rdx;
                    g[1] = ((ln->u + rn->u) - (ls->u + rs->u)) * q_rdy;
                    g[2] = (R->v - L->v) * rdx;
                    g[3] = ((ln->v + rn->v) - (ls->v + rs->v)) * q_rdy;
                    g[4] = (R->T - L->T) * rdx;
                    g[5] = ((ln->T + rn->T) - (ls->T + rs->T)) * q_rdy;
                } else {
                    real_t a[3], b[3];
                    vertex_vals(P, W, i, j, a);      /* P1 */
                    vertex_vals(P, W, i, j + 1, b);  /* P3 */
                    real_t dC[3] = {R->u - L->u, R->v - L->v, R->T - L->T};
                    for (int k = 0; k < 3; ++k) {
                        real_t dV = b[k] - a[k];
                        g[2 * k] = dC[k] * G.ic[0][fidx] + dV * G.ic[1][fidx];
                        g[2 * k + 1] = dC[k] * G.ic[2][fidx] + dV * G.ic[3][fidx];
                    }
                }
            }
            real_t F[4];
            face_flux(P, &W[EX(i - 2, j)], L, R, &W[EX(i + 1, j)], nx_, ny_, g, F);
            if (P->curvilinear) for (int k = 0; k < 4; ++k) F[k] = F[k] * G.il[fidx];
            for (int k = 0; k < 4; ++k) FX[k * nfi + fidx] = F[k];
        }
    /* j-faces: between cells (i, j-1) and (i, j) */
    ROWS_IN_PARALLEL
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t fidx = (size_t)j * nx + i;
            const prim *B = &W[EX(i, j - 1)], *T = &W[EX(i, j)];
            real_t g[6] = {0, 0, 0, 0, 0, 0};
            double nx_ = 0.0, ny_ = 1.0;
            if (P->curvilinear) { nx_ = G.jn_x[fidx]; ny_ = G.jn_y[fidx]; }
            if (P->viscous) {
                if (!P->curvilinear) {
                    const prim *eb = &W[EX(i + 1, j - 1)], *et = &W[EX(i + 1, j)];
                    const prim *wb = &W[EX(i - 1, j - 1)], *wt = &W[EX(i - 1, j)];
                    g[0] = ((eb->u + et->u) - (wb->u + wt->u)) * q_rdx;
                    g[1] = (T->u - B->u) * rdy;
                    g[2] = ((eb->v + et->v) - (wb->v + wt->v)) * q_rdx;
                    g[3] = (T->v - B->v) * rdy;
                    g[4] = ((eb->T + et->T) - (wb->T + wt->T)) * q_rdx;
                    g[5] = (T->T - B->T) * rdy;
                } else {
                    real_t a[3], b[3];
                    vertex_vals(P, W, i + 1, j, a);  /* P1 */
                    vertex_vals(P, W, i, j, b);      /* P3 */
                    real_t dC[3] = {T->u - B->u, T->v - B->v, T->T - B->T};
                    for (int k = 0; k < 3; ++k) {
                        real_t dV = b[k] - a[k];
                        g[2 * k] = dC[k] * G.jc[0][fidx] + dV * G.jc[1][fidx];
                        g[2 * k + 1] = dC[k] * G.jc[2][fidx] + dV * G.jc[3][fidx];
                    }
                }
            }
            real_t F[4];
            face_flux(P, &W[EX(i, j - 2)], B, T, &W[EX(i, j + 1)], nx_, ny_, g, F);
            if (P->curvilinear) for (int k = 0; k < 4; ++k) F[k] = F[k] * G.jl[fidx];
            for (int k = 0; k < 4; ++k) FY[k * nfj + fidx] = F[k];
        }
    /* cell balance, faces summed west/east then south/north */
    ROWS_IN_PARALLEL
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            size_t fw = (size_t)j * (nx + 1) + i, fs = (size_t)j * nx + i, fn = (size_t)(j + 1) * nx + i;
            for (int k = 0; k < 4; ++k) {
                real_t dX = FX[k * nfi + fw + 1] - FX[k * nfi + fw];
                real_t dY = FY[k * nfj + fn] - FY[k * nfj + fs];
                if (P->curvilinear)
                    f[k * nc + c] = -((dX + dY) * G.inv_vol[c]);
                else
                    f[k * nc + c] = -(dX * rdx + dY * rdy);
            }
        }
    if (P->curvilinear) free_geom(&G);
    free(W); free(FX); free(FY);
    return 0;
}

#ifndef ORACLE_COMPLEX
int oracle_residual(const oracle_problem *P, const double *q, double *f) { return residual_impl(P, q, f); }

/* Sum over cells of Vol * f (discrete conservation check); volumes as used above */
int oracle_cell_volumes(const oracle_problem *P, double *vol)
{
    const int nx = P->nx, ny = P->ny;
    if (!P->curvilinear) {
        for (size_t c = 0; c < (size_t)nx * ny; ++c) vol[c] = P->dx * P->dy;
        return 0;
    }
    geom G;
    build_geom(P, &G);
    for (size_t c = 0; c < (size_t)nx * ny; ++c) vol[c] = 1.0 / G.inv_vol[c];
    free_geom(&G);
    return 0;
}

/* Finite-difference Jacobian-vector product, Eq. matvecFD:
 *   w = (f(y + eps v) - f(y)) / eps, with f0 = f(y) supplied. */
int oracle_jvp_fd(const oracle_problem *P, const double *y, const double *v, const double *f0,
                  double eps, double *w)
{
    const size_t n = (size_t)4 * P->nx * P->ny;
    double *yp = malloc(n * sizeof(double));
    if (!yp) return -1;
    ROWS_IN_PARALLEL
    for (size_t k = 0; k < n; ++k) yp[k] = y[k] + eps * v[k];
    int rc = oracle_residual(P, yp, w);
    ROWS_IN_PARALLEL
    for (size_t k = 0; k < n; ++k) w[k] = (w[k] - f0[k]) / eps;
    free(yp);
    return rc;
}

/* Roe flux of Eq. (Sec. 3.2 setting) for one face, exported for the pin tests:
 * primitive states WL, WR = (rho, u, v, p), unit normal (nx, ny). */
void oracle_roe_flux(const double *WL, const double *WR, double nx, double ny, double gamma,
                     double efix, double *F)
{
    double gm1 = gamma - 1.0;
    roe(WL, WR, nx, ny, gm1, 1.0 / gm1, efix, F);
}
#else
/* Exact Jacobian-vector product by the complex step: Im f(y + i h v) / h. */
int oracle_jvp_cs(const oracle_problem *P, const double *y, const double *v, double h, double *jv)
{
    const size_t n = (size_t)4 * P->nx * P->ny;
    real_t *q = malloc(n * sizeof(real_t));
    real_t *f = malloc(n * sizeof(real_t));
    if (!q || !f) { free(q); free(f); return -1; }
    for (size_t k = 0; k < n; ++k) q[k] = y[k] + I * (h * v[k]);
    int rc = residual_impl(P, q, f);
    for (size_t k = 0; k < n; ++k) jv[k] = cimag(f[k]) / h;
    free(q);
    free(f);
    return rc;
}

/* f at a complex state, real and imaginary parts in separate arrays (the
 * complex-step derivative of integrators built on f). */
int oracle_residual_cx(const oracle_problem *P, const double *q_re, const double *q_im, double *f_re, double *f_im)
{
    const size_t n = (size_t)4 * P->nx * P->ny;
    real_t *q = malloc(n * sizeof(real_t));
    real_t *f = malloc(n * sizeof(real_t));
    if (!q || !f) { free(q); free(f); return -1; }
    for (size_t k = 0; k < n; ++k) q[k] = q_re[k] + I * q_im[k];
    int rc = residual_impl(P, q, f);
    for (size_t k = 0; k < n; ++k) {
        f_re[k] = creal(f[k]);
        f_im[k] = cimag(f[k]);
    }
    free(q);
    free(f);
    return rc;
}
#endif
