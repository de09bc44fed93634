// Reverse mode (vector-Jacobian products) of the residual and of one ROK4 step
// with finite-difference Jacobian-vector products (Sec. 2.2.2, Eq. ROK;
// Sec. 2.3, Eq. matvecFD), for gradients of a final-time functional with
// respect to the state and the viscosity (the constant one, or the reference
// viscosity of Sutherland's law).  Uniform periodic grids (below) and
// curvilinear grids (their own two passes, further down) take hand-written
// reverse sweeps; Lorenz-96 takes a compressed Jacobian of exact JVPs.
//
// Residual VJP, uniform periodic grids: f_c = -(F_{c+1/2} - F_{c-1/2}) / dx
// - (G_{c+1/2} - G_{c-1/2}) / dy, so a face flux's adjoint is
// Fbar = (ubar_R - ubar_L) / dx.  Pass 0 computes every cell's primitives once.
// Pass 1 (one thread per face) takes Fbar back through the face flux: one
// evaluation of the Roe flux keeps its intermediates and a hand-written reverse
// sweep gives (dF/dW_L)^T Fbar and (dF/dW_R)^T Fbar for the reconstructed
// left/right primitive states; the central viscous flux is reversed by hand
// too.  Each face stores the adjoints of
// its MUSCL states and of its viscous inputs.  Pass 2 (one thread per cell)
// gathers, in a fixed order, the contributions of the faces whose stencils
// contain the cell (MUSCL reaches two cells along the normal, the viscous
// gradients one cell across) and maps primitive adjoints to conserved ones.
// No atomics: the result is deterministic.
//
// ROK step reverse: the step is recomputed from y_n (its stage vectors, basis,
// Hessenberg matrix and stage solutions stay in the context), or its internals
// are copied back from a tape that a recording step wrote, then every
// statement is reversed in the opposite order; eps is a constant of the step.
// The reverse Gram-Schmidt passes of one Arnoldi column run as one cooperative
// launch where the device allows it (pass by pass otherwise).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "coefficients.h"
#include "context.h"

#define ROK_NS adj
#define ROK_STENCIL_DEVICE_ONLY
#define ROK_LINALG_DEVICE_ONLY
#include "linalg_impl.cuh"
#include "stencil_impl.cuh"

using namespace rok;
using namespace rok::adj;

namespace rok_host {
rok_status enqueue_step_body(rok_ctx *c, double *y, int M);
rok_status launch_stencil(rok_ctx *c, const StencilIO &io);
StencilIO plain_io(rok_ctx *c, const double *y, double *out);
}  // namespace rok_host

// ---- device state of the reverse step ------------------------------------------
struct AdjState {
    double Hb[(kMaxKrylov + 1) * kMaxKrylov];   // adjoint of H (row-major, stride kMaxKrylov)
    double lamb[4][kMaxKrylov];                 // adjoint of lambda_i
    double phib[4][kMaxKrylov];                 // adjoint of phi_i
    double mub;                                 // adjoint of the viscosity
    double scratch[2 * kMaxKrylov];
};

struct AdjWork {
    size_t N = 0;
    int M = 0, P = 0;
    double *Vb = nullptr;      // M x N adjoint of the basis
    double *kb[4] = {};        // adjoints of the stage vectors
    double *yb = nullptr, *Fb = nullptr, *F1b = nullptr, *F1acc = nullptr;
    double *wb = nullptr, *wcur = nullptr, *wlast = nullptr, *Yt = nullptr, *y1 = nullptr;
    double *pA = nullptr, *pB = nullptr, *pM = nullptr;
    double *faces = nullptr;   // 16 x (nx ny) per direction
    double *prims = nullptr;   // rho, u, v, p, T of every cell (5 x nx ny)
    double *mupart = nullptr;  // CTA partials of the viscosity adjoint
    // compressed-Jacobian products (Lorenz-96, curvilinear grids below 2 x 2):
    // class direction, its JVP, g = J^T u, reduction partials (2P: dot2 writes both sets)
    double *cseed = nullptr, *cD = nullptr, *cg = nullptr, *cpart = nullptr;
    // curvilinear reverse sweep: 17 values per face, CTA partials of the viscosity adjoint
    double *cfaces = nullptr, *cmupart = nullptr;
    int nmu = 0;
    int rev_ctas = -1;         // CTAs of the cooperative reverse-MGS launch (0: pass by pass)
    AdjState *as = nullptr;
    StepState *h_st = nullptr;
    double *h_mub = nullptr;
};

namespace {

#define CU(x)                                      \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return ROK_ERR_CUDA; \
    } while (0)

constexpr int AT = 256;
// Threads per CTA of the face pass: it needs about 140-160 registers a thread,
// so only one 256-thread CTA fits an SM and 256^2 faces take two waves with
// half the SMs idle in the second; 64-thread CTAs, 7 per SM (at most 144
// registers), take one wave and split the faces over the SMs to within a
// seventh of an SM's share.
constexpr int FT = 64;
// MUSCL left/right adjoints (8) + viscous input adjoints (7) + the adjoint of
// each neighbour's Sutherland viscosity (1; Sutherland's law only)
constexpr int kFaceVals = 16;

// primitives (rho, u, v, p) and T = p / rho of the conservative state (rho, mx, my, E)
__device__ __forceinline__ void prim_of(const StencilConsts &C, double rho, double mx, double my, double E, double *P,
                                        double &T)
{
    const double rinv = 1.0 / rho;
    const double u = mx * rinv, v = my * rinv;
    const double p = C.gm1 * (E - 0.5 * (mx * u + my * v));
    P[0] = rho;
    P[1] = u;
    P[2] = v;
    P[3] = p;
    T = p * rinv;
}

// Pass 0: the primitives of every cell, once (the face pass reads each cell's
// from four faces and the viscous terms from four more).  The state is y, or
// y + (*scale) dir formed on load (the perturbed state y + eps v_j of a JVP in
// reverse; eps is a power of two, so the sum rounds as a separate pass would).
__global__ void __launch_bounds__(AT) prim_kernel(const StencilConsts C, const double *__restrict__ y,
                                                  const double *__restrict__ dir, const double *scale,
                                                  double *__restrict__ pr)
{
    const size_t nc = (size_t)C.nx * C.ny;
    const size_t t = (size_t)blockIdx.x * AT + threadIdx.x;
    if (t >= nc) return;
    double q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = y[k * nc + t];
    if (dir) {
        const double a = *scale;
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = q[k] + a * dir[k * nc + t];
    }
    double P[4], T;
    prim_of(C, q[0], q[1], q[2], q[3], P, T);
#pragma unroll
    for (int k = 0; k < 4; ++k) pr[k * nc + t] = P[k];
    pr[4 * nc + t] = T;
}

// Sutherland's law (Sec. 3.2) written mu(T) = mu_ref g(T) with
// g = t^{3/2} (1 + S) / (t + S), t = T / T_ref; also dg/dT = g (t + 3 S) / (2 T (t + S)).
__device__ __forceinline__ double suth_g(const StencilConsts &C, double T, double &dgdT)
{
    const double t = T * C.inv_tref, S = C.suth_s;
    const double r = 1.0 / (t + S);
    const double g = (t * sqrt(t)) * ((1.0 + S) * r);
    dgdT = (0.5 * g) * ((t + 3.0 * S) * r) / T;
    return g;
}

__device__ __forceinline__ void prim_load(const double *__restrict__ pr, size_t nc, size_t c, double *P, double &T)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) P[k] = pr[k * nc + c];
    T = pr[4 * nc + c];
}

// Reverse of the Roe flux of roe_x (DIR 0) / roe_y (DIR 1): Lb = (dF/dL)^T Fb,
// Rb = (dF/dR)^T Fb for the left and right primitive states (rho, u, v, p),
// one forward sweep that keeps the intermediates and one reverse sweep
// (about three flux evaluations, against eight dual-number evaluations for
// the Jacobian columns).  N is the normal and T the tangential velocity
// component; |x| and Harten's switch differentiate as the dual numbers do
// (sign +1 at 0, the branch taken by the value).
template <int DIR>
__device__ __forceinline__ void roe_vjp(const double *L, const double *R, const StencilConsts &C, const double *Fb,
                                        double *Lb, double *Rb)
{
    constexpr int N = 1 + DIR, T = 2 - DIR;
    const double rL = L[0], nL = L[N], tL = L[T], pL = L[3];
    const double rR = R[0], nR = R[N], tR = R[T], pR = R[3];
    // forward (the order of roe_avg and roe_x / roe_y)
    const double kinL = 0.5 * (L[1] * L[1] + L[2] * L[2]), kinR = 0.5 * (R[1] * R[1] + R[2] * R[2]);
    const double eL = (pL * C.inv_gm1 + rL * kinL) + pL, eR = (pR * C.inv_gm1 + rR * kinR) + pR;
    // square roots from reciprocal square roots (the reverse needs 1/sqrt as well;
    // an FP64 square root or division costs about twenty FP64 instructions)
    const double qL = rsqrt(rL), qR = rsqrt(rR);
    const double sL = rL * qL, sR = rR * qR;
    const double rt = sL * sR;
    const double Y = rt * (sL + sR), den = 1.0 / Y;
    const double rLsR = rL * sR, rRsL = rR * sL;
    const double wl = rLsR * den, wr = rRsL * den;
    const double nt = wl * nL + wr * nR, tt = wl * tL + wr * tR;
    const double X = eL * sR + eR * sL, Ht = X * den;
    const double kt = 0.5 * (nt * nt + tt * tt);
    const double ct2 = C.gm1 * (Ht - kt);
    const double rc = rsqrt(ct2);
    const double ct = ct2 * rc, inv_c2 = rc * rc;
    const double drho = rR - rL, dp = pR - pL, dn = nR - nL, dt = tR - tL;
    const double rtct = rt * ct, rcdq = rtct * dn;
    const double q1 = 0.5 * (dp - rcdq), q3 = 0.5 * (dp + rcdq);
    const double a1 = q1 * inv_c2, a2 = drho - dp * inv_c2, a3 = q3 * inv_c2;
    const double snt = nt < 0.0 ? -1.0 : 1.0, l2 = snt * nt;
    const double delta = C.efix * (l2 + ct);
    const double lam1 = nt - ct, lam3 = nt + ct;
    const double s1 = lam1 < 0.0 ? -1.0 : 1.0, s3 = lam3 < 0.0 ? -1.0 : 1.0;
    const double m1 = s1 * lam1, m3 = s3 * lam3;   // |lambda|
    const bool h1 = m1 < delta, h3 = m3 < delta;
    const double l1 = h1 ? (m1 * m1 + delta * delta) / (2.0 * delta) : m1;
    const double l3 = h3 ? (m3 * m3 + delta * delta) / (2.0 * delta) : m3;
    const double A1 = l1 * a1, A2 = l2 * a2, A3 = l3 * a3, As = l2 * rt;
    const double sA = A1 + A3, dA = A3 - A1, D0 = sA + A2;
    const double mL = rL * nL, mR = rR * nR;
    // reverse
    const double F0b = Fb[0], Fnb = Fb[N], Ftb = Fb[T], F3b = Fb[3];
    double mLb = 0.5 * F0b, mRb = 0.5 * F0b, D0b = -0.5 * F0b;
    mLb += 0.5 * Fnb * nL;
    mRb += 0.5 * Fnb * nR;
    double nLb = 0.5 * Fnb * mL, nRb = 0.5 * Fnb * mR, pLb = 0.5 * Fnb, pRb = 0.5 * Fnb;
    const double Dnb = -0.5 * Fnb;
    mLb += 0.5 * Ftb * tL;
    mRb += 0.5 * Ftb * tR;
    double tLb = 0.5 * Ftb * mL, tRb = 0.5 * Ftb * mR;
    const double Dtb = -0.5 * Ftb;
    nLb += 0.5 * F3b * eL;
    nRb += 0.5 * F3b * eR;
    double eLb = 0.5 * F3b * nL, eRb = 0.5 * F3b * nR;
    const double D3b = -0.5 * F3b;
    double rLb = mLb * nL, rRb = mRb * nR;
    nLb += mLb * rL;
    nRb += mRb * rR;
    // D3 = Ht sA + kt A2 + ct nt dA + As tt dt
    double Htb = D3b * sA, sAb = D3b * Ht, ktb = D3b * A2, A2b = D3b * kt;
    double ctb = D3b * nt * dA, ntb = D3b * ct * dA, dAb = D3b * ct * nt;
    double Asb = D3b * tt * dt, ttb = D3b * As * dt, dtb = D3b * As * tt;
    // Dt = tt D0 + As dt;  Dn = nt D0 + ct dA
    ttb += Dtb * D0;
    D0b += Dtb * tt;
    Asb += Dtb * dt;
    dtb += Dtb * As;
    ntb += Dnb * D0;
    D0b += Dnb * nt;
    ctb += Dnb * dA;
    dAb += Dnb * ct;
    // D0 = sA + A2;  sA = A1 + A3;  dA = A3 - A1
    sAb += D0b;
    A2b += D0b;
    const double A1b = sAb - dAb, A3b = sAb + dAb;
    // A1 = l1 a1, A2 = l2 a2, A3 = l3 a3, As = l2 rt
    const double l1b = A1b * a1, l3b = A3b * a3;
    const double a1b = A1b * l1, a2b = A2b * l2, a3b = A3b * l3;
    double l2b = A2b * a2 + Asb * rt;
    double rtb = Asb * l2;
    // Harten's switch on the acoustic speeds
    double deltab = 0.0, m1b, m3b;
    if (h1) {
        m1b = l1b * m1 / delta;
        deltab += l1b * (delta * delta - m1 * m1) / (2.0 * delta * delta);
    } else {
        m1b = l1b;
    }
    if (h3) {
        m3b = l3b * m3 / delta;
        deltab += l3b * (delta * delta - m3 * m3) / (2.0 * delta * delta);
    } else {
        m3b = l3b;
    }
    const double lam1b = s1 * m1b, lam3b = s3 * m3b;
    ntb += lam1b + lam3b;
    ctb += lam3b - lam1b;
    // delta = efix (l2 + ct), l2 = |nt|
    l2b += C.efix * deltab;
    ctb += C.efix * deltab;
    ntb += snt * l2b;
    // a1 = q1 / c^2, a3 = q3 / c^2, a2 = drho - dp / c^2
    const double q1b = a1b * inv_c2, q3b = a3b * inv_c2;
    double inv_c2b = a1b * q1 + a3b * q3 - a2b * dp;
    const double drhob = a2b;
    double dpb = 0.5 * q1b + 0.5 * q3b - a2b * inv_c2;
    const double rcdqb = 0.5 * (q3b - q1b);
    const double rtctb = rcdqb * dn;
    double dnb = rcdqb * rtct;
    rtb += rtctb * ct;
    ctb += rtctb * rt;
    // differences
    rRb += drhob;
    rLb -= drhob;
    pRb += dpb;
    pLb -= dpb;
    nRb += dnb;
    nLb -= dnb;
    tRb += dtb;
    tLb -= dtb;
    // ct = sqrt(ct2), inv_c2 = 1 / ct2, ct2 = gm1 (Ht - kt)
    const double ct2b = (ctb * 0.5) * rc - inv_c2b * inv_c2 * inv_c2;
    Htb += C.gm1 * ct2b;
    ktb -= C.gm1 * ct2b;
    // kt = (nt^2 + tt^2) / 2
    ntb += ktb * nt;
    ttb += ktb * tt;
    // Ht = X den, X = eL sR + eR sL
    const double Xb = Htb * den;
    double denb = Htb * X;
    eLb += Xb * sR;
    eRb += Xb * sL;
    double sRb = Xb * eL, sLb = Xb * eR;
    // nt = wl nL + wr nR, tt = wl tL + wr tR
    const double wlb = ntb * nL + ttb * tL, wrb = ntb * nR + ttb * tR;
    nLb += ntb * wl;
    nRb += ntb * wr;
    tLb += ttb * wl;
    tRb += ttb * wr;
    // wl = (rL sR) den, wr = (rR sL) den
    denb += wlb * rLsR + wrb * rRsL;
    rLb += wlb * den * sR;
    sRb += wlb * den * rL;
    rRb += wrb * den * sL;
    sLb += wrb * den * rR;
    // den = 1 / Y, Y = rt (sL + sR)
    const double Yb = -denb * den * den;
    rtb += Yb * (sL + sR);
    sLb += Yb * rt;
    sRb += Yb * rt;
    // rt = sL sR, s = sqrt(rho)
    sLb += rtb * sR;
    sRb += rtb * sL;
    rLb += (sLb * 0.5) * qL;
    rRb += (sRb * 0.5) * qR;
    // e = p / (gamma - 1) + rho kin + p, kin = (u^2 + v^2) / 2
    pLb += eLb * (C.inv_gm1 + 1.0);
    pRb += eRb * (C.inv_gm1 + 1.0);
    rLb += eLb * kinL;
    rRb += eRb * kinR;
    const double kinLb = eLb * rL, kinRb = eRb * rR;
    nLb += kinLb * nL;
    tLb += kinLb * tL;
    nRb += kinRb * nR;
    tRb += kinRb * tR;
    Lb[0] = rLb;
    Lb[N] = nLb;
    Lb[T] = tLb;
    Lb[3] = pLb;
    Rb[0] = rRb;
    Rb[N] = nRb;
    Rb[T] = tRb;
    Rb[3] = pRb;
}

// Pass 1: face D (0: x-faces, face i of row j between cells (i-1, j) and (i, j);
// 1: y-faces, face j of column i between (i, j-1) and (i, j)).  Stores
// fa[q * nc + face] for q < 15 (q = 15 too with Sutherland's law) and one
// partial of ubar . df/dmu per CTA (mu: the viscosity at T_ref with Sutherland's law).
template <bool VISC, bool SUTH, int D>
__global__ void __launch_bounds__(FT, 7) vjp_face_kernel(const StencilConsts C, const double *__restrict__ pr,
                                                      const double *__restrict__ ub, double *__restrict__ fa,
                                                      double *__restrict__ mupart)
{
    static_assert(FT == 64, "the CTA sum below adds two warp sums");
    __shared__ double sh[2];
    const int nx = C.nx, ny = C.ny;
    const size_t nc = (size_t)nx * ny;
    const size_t t = (size_t)blockIdx.x * FT + threadIdx.x;
    double mu_c = 0.0;
    if (t < nc) {
        const int i = (int)(t % nx), j = (int)(t / nx);
        auto cell = [&](int s) -> size_t {   // s-th cell along the normal, s = 0 is the face's upper cell
            return D == 0 ? (size_t)j * nx + wrapi(i + s, nx) : (size_t)wrapi(j + s, ny) * nx + i;
        };
        const size_t cm2 = cell(-2), cm1 = cell(-1), cp1 = cell(0), cp2 = cell(1);
        double Pm2[4], Pm1[4], Pp1[4], Pp2[4], Tm2, Tm1, Tp1, Tp2;
        prim_load(pr, nc, cm2, Pm2, Tm2);
        prim_load(pr, nc, cm1, Pm1, Tm1);
        prim_load(pr, nc, cp1, Pp1, Tp1);
        prim_load(pr, nc, cp2, Pp2, Tp2);
        double WL[4], WR[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) muscl(Pm2[k], Pm1[k], Pp1[k], Pp2[k], C.c_lo, C.c_hi, WL[k], WR[k]);
        const double rd = D == 0 ? C.rdx : C.rdy;
        double Fb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) Fb[k] = rd * (ub[k * nc + cp1] - ub[k * nc + cm1]);
        // Roe flux: (dF/dWL)^T Fb and (dF/dWR)^T Fb by one reverse sweep
        {
            double Lb[4], Rb[4];
            roe_vjp<D>(WL, WR, C, Fb, Lb, Rb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fa[q * nc + t] = Lb[q];
                fa[(q + 4) * nc + t] = Rb[q];
            }
        }
        if (VISC) {
            // normal cells a = cm1, b = cp1; tangential neighbours across the face
            auto cross = [&](size_t c0, int s) -> size_t {
                const int ci = (int)(c0 % nx), cj = (int)(c0 / nx);
                return D == 0 ? (size_t)wrapi(cj + s, ny) * nx + ci : (size_t)cj * nx + wrapi(ci + s, nx);
            };
            auto uv = [&](size_t c0, int comp) -> double { return pr[(1 + comp) * nc + c0]; };
            const double q_rt = D == 0 ? C.q_rdy : C.q_rdx;
            // normal and tangential derivatives of u and v, normal derivative of T
            const double un = (Pp1[1] - Pm1[1]) * rd, vn = (Pp1[2] - Pm1[2]) * rd, Tn = (Tp1 - Tm1) * rd;
            const double ut = ((uv(cross(cm1, 1), 0) + uv(cross(cp1, 1), 0)) -
                               (uv(cross(cm1, -1), 0) + uv(cross(cp1, -1), 0))) * q_rt;
            const double vt = ((uv(cross(cm1, 1), 1) + uv(cross(cp1, 1), 1)) -
                               (uv(cross(cm1, -1), 1) + uv(cross(cp1, -1), 1))) * q_rt;
            const double uf = 0.5 * (Pm1[1] + Pp1[1]), vf = 0.5 * (Pm1[2] + Pp1[2]);
            // face viscosity mu_f: mu, or with Sutherland's law the mean of the two
            // cells' mu(T) = mu_ref gf (gf = 1 for a constant viscosity)
            double gf = 1.0;
            if (SUTH) {
                double dg_m, dg_p;
                gf = 0.5 * (suth_g(C, Tm1, dg_m) + suth_g(C, Tp1, dg_p));
            }
            const double mu = SUTH ? C.mu * gf : C.mu, kf = mu * C.kfac;
            // x-face: ux = un, uy = ut, vx = vn, vy = vt; y-face: uy = un, ux = ut, vy = vn, vx = vt
            const double ux = D == 0 ? un : ut, uy = D == 0 ? ut : un, vx = D == 0 ? vn : vt, vy = D == 0 ? vt : vn;
            const double div = ux + vy;
            const double txx1 = 2.0 * ux - C.c23 * div, tyy1 = 2.0 * vy - C.c23 * div, txy1 = uy + vx;
            // flux terms removed by the viscous flux: x-face (txx, txy), y-face (txy, tyy)
            const double s1 = D == 0 ? txx1 : txy1, s2 = D == 0 ? txy1 : tyy1;
            // reverse of F1 -= mu s1, F2 -= mu s2, F3 -= (uf mu s1 + vf mu s2 + kf Tn)
            const double s1b = -mu * (Fb[1] + uf * Fb[3]);     // adjoint of mu s1 ... times mu
            const double s2b = -mu * (Fb[2] + vf * Fb[3]);
            const double ufb = -mu * s1 * Fb[3], vfb = -mu * s2 * Fb[3], Tnb = -kf * Fb[3];
            double uxb = 0.0, uyb = 0.0, vxb = 0.0, vyb = 0.0;
            if (D == 0) {   // s1 = 2 ux - c23 (ux + vy), s2 = uy + vx
                uxb = (2.0 - C.c23) * s1b;
                vyb = -C.c23 * s1b;
                uyb = s2b;
                vxb = s2b;
            } else {        // s1 = uy + vx, s2 = 2 vy - c23 (ux + vy)
                uyb = s1b;
                vxb = s1b;
                vyb = (2.0 - C.c23) * s2b;
                uxb = -C.c23 * s2b;
            }
            fa[8 * nc + t] = D == 0 ? uxb : uyb;    // normal derivative of u
            fa[9 * nc + t] = D == 0 ? uyb : uxb;    // tangential derivative of u
            fa[10 * nc + t] = D == 0 ? vxb : vyb;   // normal derivative of v
            fa[11 * nc + t] = D == 0 ? vyb : vxb;   // tangential derivative of v
            fa[12 * nc + t] = Tnb;
            fa[13 * nc + t] = ufb;
            fa[14 * nc + t] = vfb;
            // adjoint of mu_f; each neighbour's mu(T) enters mu_f with weight 1/2
            const double mufb = -((Fb[1] * s1 + Fb[2] * s2) + Fb[3] * ((uf * s1 + vf * s2) + C.kfac * Tn));
            if (SUTH) fa[15 * nc + t] = 0.5 * mufb;
            mu_c = SUTH ? mufb * gf : mufb;   // d mu_f / d mu_ref = gf
        }
    }
    const double s = lane_tree(mu_c);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) mupart[blockIdx.x] = sh[0] + sh[1];
}

struct VjpOut {
    double *out1;            // out1 += s1 (* s1dev) g   (nullable)
    double s1;
    const double *s1dev;
    double *out2;            // out2 += s2 (* s2dev) g   (nullable)
    double s2;
    const double *s2dev;
};

// Pass 2: g = J^T ubar at each cell from the face adjoints
template <bool VISC, bool SUTH>
__global__ void __launch_bounds__(AT) vjp_cell_kernel(const StencilConsts C, const double *__restrict__ pr,
                                                      const double *__restrict__ fx, const double *__restrict__ fy,
                                                      const VjpOut o)
{
    const int nx = C.nx, ny = C.ny;
    const size_t nc = (size_t)nx * ny;
    const size_t t = (size_t)blockIdx.x * AT + threadIdx.x;
    if (t >= nc) return;
    const int i = (int)(t % nx), j = (int)(t / nx);
    auto xf = [&](int fi, int fj) -> size_t { return (size_t)wrapi(fj, ny) * nx + wrapi(fi, nx); };
    const double a1 = (1.0 + C.c_lo) - C.c_hi;
    double Pb[4] = {0.0, 0.0, 0.0, 0.0}, Tb = 0.0;
    // MUSCL: the cell is m2 of face +2, m1 of face +1, p1 of face 0, p2 of face -1
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double *xl = fx + (size_t)k * nc, *xr = fx + (size_t)(k + 4) * nc;
        const double *yl = fy + (size_t)k * nc, *yr = fy + (size_t)(k + 4) * nc;
        double s = -C.c_lo * xl[xf(i + 2, j)];
        s = s + (a1 * xl[xf(i + 1, j)] + C.c_hi * xr[xf(i + 1, j)]);
        s = s + (C.c_hi * xl[xf(i, j)] + a1 * xr[xf(i, j)]);
        s = s - C.c_lo * xr[xf(i - 1, j)];
        s = s - C.c_lo * yl[xf(i, j + 2)];
        s = s + (a1 * yl[xf(i, j + 1)] + C.c_hi * yr[xf(i, j + 1)]);
        s = s + (C.c_hi * yl[xf(i, j)] + a1 * yr[xf(i, j)]);
        s = s - C.c_lo * yr[xf(i, j - 1)];
        Pb[k] = s;
    }
    if (VISC) {
        auto F = [&](const double *f, int q, size_t idx) { return f[(size_t)q * nc + idx]; };
        // x-faces: upper cell of face i, lower cell of face i + 1 (row j)
        {
            const size_t up = xf(i, j), lo = xf(i + 1, j);
            Pb[1] += (F(fx, 8, up) - F(fx, 8, lo)) * C.rdx + 0.5 * (F(fx, 13, up) + F(fx, 13, lo));
            Pb[2] += (F(fx, 10, up) - F(fx, 10, lo)) * C.rdx + 0.5 * (F(fx, 14, up) + F(fx, 14, lo));
            Tb += (F(fx, 12, up) - F(fx, 12, lo)) * C.rdx;
            // tangential: faces i, i+1 of row j-1 (+) and of row j+1 (-)
            const size_t a = xf(i, j - 1), b = xf(i + 1, j - 1), c2 = xf(i, j + 1), d = xf(i + 1, j + 1);
            Pb[1] += ((F(fx, 9, a) + F(fx, 9, b)) - (F(fx, 9, c2) + F(fx, 9, d))) * C.q_rdy;
            Pb[2] += ((F(fx, 11, a) + F(fx, 11, b)) - (F(fx, 11, c2) + F(fx, 11, d))) * C.q_rdy;
        }
        // y-faces: upper cell of face j, lower cell of face j + 1 (column i)
        {
            const size_t up = xf(i, j), lo = xf(i, j + 1);
            Pb[1] += (F(fy, 8, up) - F(fy, 8, lo)) * C.rdy + 0.5 * (F(fy, 13, up) + F(fy, 13, lo));
            Pb[2] += (F(fy, 10, up) - F(fy, 10, lo)) * C.rdy + 0.5 * (F(fy, 14, up) + F(fy, 14, lo));
            Tb += (F(fy, 12, up) - F(fy, 12, lo)) * C.rdy;
            const size_t a = xf(i - 1, j), b = xf(i - 1, j + 1), c2 = xf(i + 1, j), d = xf(i + 1, j + 1);
            Pb[1] += ((F(fy, 9, a) + F(fy, 9, b)) - (F(fy, 9, c2) + F(fy, 9, d))) * C.q_rdx;
            Pb[2] += ((F(fy, 11, a) + F(fy, 11, b)) - (F(fy, 11, c2) + F(fy, 11, d))) * C.q_rdx;
        }
    }
    double P[4], T;
    prim_load(pr, nc, t, P, T);
    if (SUTH) {
        // the cell's mu(T) enters the viscosity of the four faces around it
        const double mub = (fx[15 * nc + xf(i, j)] + fx[15 * nc + xf(i + 1, j)]) +
                           (fy[15 * nc + xf(i, j)] + fy[15 * nc + xf(i, j + 1)]);
        double dg;
        suth_g(C, T, dg);
        Tb += mub * (C.mu * dg);
    }
    const double rho = P[0], u = P[1], v = P[2];
    const double rinv = 1.0 / rho;
    // T = p / rho
    Pb[3] += Tb * rinv;
    Pb[0] -= Tb * T * rinv;
    // rho = q0, u = q1 / rho, v = q2 / rho, p = (gamma - 1) (q3 - (q1^2 + q2^2) / (2 q0))
    double qb[4];
    qb[0] = (Pb[0] - (u * Pb[1] + v * Pb[2]) * rinv) + C.gm1 * 0.5 * (u * u + v * v) * Pb[3];
    qb[1] = Pb[1] * rinv - C.gm1 * u * Pb[3];
    qb[2] = Pb[2] * rinv - C.gm1 * v * Pb[3];
    qb[3] = C.gm1 * Pb[3];
    const double s1 = o.s1dev ? o.s1 * *o.s1dev : o.s1;
    const double s2 = o.s2dev ? o.s2 * *o.s2dev : o.s2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t e = (size_t)k * nc + t;
        if (o.out1) o.out1[e] = o.out1[e] + s1 * qb[k];
        if (o.out2) o.out2[e] = o.out2[e] + s2 * qb[k];
    }
}

// dst += factor (* fdev) tree(part[0..n)), one CTA
__global__ void tree_add_kernel(const double *part, int n, double factor, const double *fdev, double *dst)
{
    __shared__ double sh[10];
    const double s = tree_partials(part, n, sh);
    if (threadIdx.x == 0) *dst = *dst + (fdev ? factor * *fdev : factor) * s;
}

// out = c0 x0 + (c1 * c1dev) x1   (x0 nullable)
__global__ void __launch_bounds__(AT) lin2_kernel(double *out, const double *x0, double c0, const double *x1,
                                                  double c1, const double *c1dev, size_t n)
{
    const double a = c1dev ? c1 * *c1dev : c1;
    for (size_t e = (size_t)blockIdx.x * AT + threadIdx.x; e < n; e += (size_t)gridDim.x * AT)
        out[e] = (x0 ? c0 * x0[e] : 0.0) + a * x1[e];
}

// Fbar = h kbar + sum_m phib[m] V_m
__global__ void __launch_bounds__(AT) fbar_kernel(double *out, const double *kb, double h, const double *V, size_t ldv,
                                                  size_t n, const double *phib, const StepState *st)
{
    __shared__ double c[kMaxKrylov];
    const int m = st->meff;
    for (int q = threadIdx.x; q < m; q += AT) c[q] = phib[q];
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * AT + threadIdx.x; e < n; e += (size_t)gridDim.x * AT) {
        double a = h * kb[e];
        for (int q = 0; q < m; ++q) a = a + c[q] * V[(size_t)q * ldv + e];
        out[e] = a;
    }
}

// Vbar_m = sum_i (cvec_i[m] kbar_i + phib_i[m] F_i), m < meff
__global__ void __launch_bounds__(AT) assemble_vb_kernel(double *Vb, size_t ldv, size_t n, const double *k0,
                                                         const double *k1, const double *k2, const double *k3,
                                                         const double *F0, const double *F1, const double *F2,
                                                         const double *F3, const StepState *st, const AdjState *as)
{
    const int m = st->meff;
    for (size_t e = (size_t)blockIdx.x * AT + threadIdx.x; e < n; e += (size_t)gridDim.x * AT) {
        const double kk[4] = {k0[e], k1[e], k2[e], k3[e]};
        const double ff[4] = {F0[e], F1[e], F2[e], F3[e]};
        for (int q = 0; q < m; ++q) {
            double a = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) a = a + (st->cvec[i][q] * kk[i] + as->phib[i][q] * ff[i]);
            Vb[(size_t)q * ldv + e] = a;
        }
    }
}

struct GamRowA {
    double g[4];
};

// Reverse of stage i's small system (one CTA):
//   cbar = V^T kbar_i (tree of the CTA partials pc[m * P + b]);
//   lambda_i = L^{-1} rhs_i, L = I - h g H (LU with row interchanges from the step);
//   rhs_i = h phi_i + h H acc_i, acc_i = sum_{j<i} gamma_ij lambda_j.
__global__ void __launch_bounds__(AT) stage_rev_kernel(int stage, GamRowA gr, const double *pc, int P,
                                                       const StepState *st, AdjState *as)
{
    const int m = st->meff;
    const double h = st->h, hg = st->hg;
    const int tid = threadIdx.x;
    __shared__ double cb[kMaxKrylov], z[kMaxKrylov], acc[kMaxKrylov], lam[kMaxKrylov];
    __shared__ double A[kMaxKrylov * kMaxKrylov];
    for (int q = tid >> 5; q < m; q += blockDim.x >> 5) {
        const double v = warp_tree_partials(pc + (size_t)q * P, P);
        if ((tid & 31) == 0) cb[q] = v;
    }
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
        const int r = idx / m, q = idx % m;
        A[r * kMaxKrylov + q] = st->LU[r * kMaxKrylov + q];
    }
    for (int q = tid; q < m; q += blockDim.x) {
        double a = 0.0;
        for (int jj = 0; jj < stage; ++jj) a = a + gr.g[jj] * st->lam[jj][q];
        acc[q] = a;
        lam[q] = st->lam[stage][q];
    }
    __syncthreads();
    double *lamb = as->lamb[stage];
    double *phib = as->phib[stage];
    for (int q = tid; q < m; q += blockDim.x) {
        const double l = lamb[q] + cb[q];
        lamb[q] = l;
        z[q] = l;
        phib[q] = -h * cb[q];
    }
    __syncthreads();
    // z = L^{-T} lamb: U^T s = lamb, L^T t = s, then the interchanges in reverse
    // order; one warp, column by column (lane l holds rows l and l + 32)
    if (tid < 32) {
        const int r0 = tid, r1 = tid + 32;
        double s0 = r0 < m ? z[r0] : 0.0, s1 = r1 < m ? z[r1] : 0.0;
        for (int k = 0; k < m; ++k) {   // U^T: row r needs z_k for k < r, ascending k
            if (r0 == k) s0 = s0 / A[k * kMaxKrylov + k];
            if (r1 == k) s1 = s1 / A[k * kMaxKrylov + k];
            const double zk = __shfl_sync(0xffffffffu, k < 32 ? s0 : s1, k & 31);
            if (r0 > k && r0 < m) s0 = s0 - A[k * kMaxKrylov + r0] * zk;
            if (r1 > k && r1 < m) s1 = s1 - A[k * kMaxKrylov + r1] * zk;
        }
        for (int k = m - 1; k > 0; --k) {   // L^T (unit): row r needs z_k for k > r
            const double zk = __shfl_sync(0xffffffffu, k < 32 ? s0 : s1, k & 31);
            if (r0 < k) s0 = s0 - A[k * kMaxKrylov + r0] * zk;
            if (r1 < k) s1 = s1 - A[k * kMaxKrylov + r1] * zk;
        }
        if (r0 < m) z[r0] = s0;
        if (r1 < m) z[r1] = s1;
        __syncwarp();
        if (tid == 0)
            for (int k = m - 1; k >= 0; --k) {
                const int p = st->piv[k];
                if (p != k) { double tmp = z[k]; z[k] = z[p]; z[p] = tmp; }
            }
    }
    __syncthreads();
    // H_bar += h g z lambda_i^T + h z acc_i^T ; phi_bar += h z ; acc_bar = h H^T z
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
        const int r = idx / m, q = idx % m;
        as->Hb[r * kMaxKrylov + q] += hg * z[r] * lam[q] + h * z[r] * acc[q];
    }
    for (int q = tid; q < m; q += blockDim.x) {
        phib[q] += h * z[q];
        double a = 0.0;
        for (int r = 0; r < m; ++r) a = a + st->H[r * kMaxKrylov + q] * z[r];
        const double accb = h * a;
        for (int jj = 0; jj < stage; ++jj) as->lamb[jj][q] += gr.g[jj] * accb;
    }
}

// Reverse of v = w / hn, hn = ||w|| (or of v_1 = F1 / beta):
//   out = (base ? base : 0) + vb / hn + (extra - <v, vb> / hn) v, <v, vb> = tree(pin);
// wout (nullable) = hn v, the orthogonalised w that the pass before needs
__global__ void __launch_bounds__(AT) normrev_kernel(double *out, const double *base, const double *vb,
                                                     const double *v, size_t n, const double *pin, int P,
                                                     const double *hn_ptr, const double *extra_ptr, double *wout)
{
    __shared__ double sh[10];
    const double d = tree_partials(pin, P, sh);
    const double hn = *hn_ptr;
    // one division per thread; the entries are scaled by the reciprocal (an
    // FP64 division costs about twenty FP64 instructions on this part)
    const double rh = 1.0 / hn;
    const double cv = (extra_ptr ? *extra_ptr : 0.0) - d * rh;
    for (size_t e = (size_t)blockIdx.x * AT + threadIdx.x; e < n; e += (size_t)gridDim.x * AT) {
        const double ve = v[e];
        out[e] = (base ? base[e] : 0.0) + vb[e] * rh + cv * ve;
        if (wout) wout[e] = hn * ve;   // w = h v (the normalised column scaled back)
    }
}

// Reverse of one modified-Gram-Schmidt pass of column j: w_{i+1} = w_i - h_ij v_i,
// h_ij = <v_i, w_i>, given wbar = adjoint of w_{i+1} and wcur = w_{i+1}:
//   hb = Hbar_ij - <v_i, wbar>;  w_i = wcur + h_ij v_i;
//   Vbar_i += -h_ij wbar + hb w_i;  wbar += hb v_i;  wcur = w_i;
// then the partials of <v_{i-1}, wbar> for the next pass (CTA chunks of 2048).
__global__ void __launch_bounds__(RT) mgsrev_kernel(double *__restrict__ wb, double *__restrict__ wcur,
                                                    double *__restrict__ Vbi, const double *__restrict__ vi,
                                                    const double *__restrict__ vprev, size_t n,
                                                    const double *__restrict__ pin, int P, const double *hij_ptr,
                                                    const double *hbij_ptr, double *__restrict__ pout)
{
    __shared__ double sh[10];
    const size_t e0 = lane_e0();
    double w[EPL], c[EPL], v[EPL], g[EPL], x[EPL];
    load8(wb, e0, n, w);
    load8(wcur, e0, n, c);
    load8(vi, e0, n, v);
    load8(Vbi, e0, n, g);
    const double d = tree_partials(pin, P, sh);
    const double hij = *hij_ptr;
    const double hb = *hbij_ptr - d;
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        const double wi = c[k] + hij * v[k];
        g[k] = (g[k] - hij * w[k]) + hb * wi;
        w[k] = w[k] + hb * v[k];
        c[k] = wi;
    }
    store8(wb, e0, n, w);
    store8(wcur, e0, n, c);
    store8(Vbi, e0, n, g);
    if (vprev) {
        load8(vprev, e0, n, x);
        const double s = chunk_sumv(lane_dot(x, w), sh);   // <v_{i-1}, wbar>
        if (threadIdx.x == 0) pout[blockIdx.x] = s;
    }
}

// The j+1 reverse passes of mgsrev_kernel for Arnoldi column j in one
// cooperative launch (the mirror of arnoldi_column_kernel: the adjoint wbar and
// w stay in registers, v_i is carried from one pass to the next, bounded waits
// on per-pass arrival counters).  On entry wb holds the adjoint of w_{j+1}, wcur =
// w_{j+1} and partA the chunk partials of <v_j, wbar> (dot2, as on the
// pass-by-pass path); on exit wb holds the adjoint of w_0 = J v_j (wcur is not
// updated).  cnt[0 .. j) are the arrival counters of the passes' partials
// (zero on entry).  The same arithmetic as the pass-by-pass kernels.  NC:
// chunks per CTA (1 when the grid covers every chunk once, which keeps the
// state of one chunk in registers without spilling, else 2).
template <int NC>
__global__ void __launch_bounds__(RT, 2) mgsrev_column_kernel(double *__restrict__ wb, const double *__restrict__ wcur,
                                                              double *__restrict__ Vb, const double *__restrict__ V,
                                                              size_t ldv, size_t n, int j, int P, double *partA,
                                                              double *partB, unsigned *cnt, StepState *st,
                                                              const AdjState *as)
{
    static_assert(NC == 1 || NC == 2, "one or two chunks per CTA");
    __shared__ double sh[16];
    const unsigned G = gridDim.x;
    double b[NC][EPL], w[NC][EPL], v[NC][EPL];
    size_t e0[NC];
    bool have[NC];
    double x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int blk = blockIdx.x + c * G;
        have[c] = blk < P;
        e0[c] = ((size_t)blk * RT + threadIdx.x) * EPL;
        if (have[c]) {
            load8(wb, e0[c], n, b[c]);
            load8(wcur, e0[c], n, w[c]);
            load8(V + (size_t)j * ldv, e0[c], n, v[c]);
        }
    }
    double sa, sb;
    double *pin = partA, *pout = partB;
    for (int i = j; i >= 0; --i) {
        // the partials of pass i + 1 (counter j - i - 1; those of pass j come
        // from the preceding launch)
        if (i < j && !gen_wait(cnt + (j - i - 1), G, &st->status)) return;
        const double d = tree_partials(pin, P, sh);
        const double hij = st->H[i * kMaxKrylov + j];
        const double hb = as->Hb[i * kMaxKrylov + j] - d;
        double *vbi = Vb + (size_t)i * ldv;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            x[c] = 0.0;
            if (!have[c]) continue;
            double g[EPL];
            load8(vbi, e0[c], n, g);
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const double wi = w[c][k] + hij * v[c][k];
                g[k] = (g[k] - hij * b[c][k]) + hb * wi;
                b[c][k] = b[c][k] + hb * v[c][k];
                w[c][k] = wi;
            }
            store8(vbi, e0[c], n, g);
            if (i > 0) {
                load8(V + (size_t)(i - 1) * ldv, e0[c], n, v[c]);
                if (i >= 2) prefetch_l2(V + (size_t)(i - 2) * ldv, e0[c], n);
                x[c] = lane_dot(v[c], b[c]);   // <v_{i-1}, wbar>
            }
        }
        if (i == 0) break;
        if (NC == 2 && have[NC - 1]) {
            chunk_sum2v(x[0], x[NC - 1], sh, sa, sb);
        } else {
            sa = chunk_sumv(x[0], sh);
        }
        if (threadIdx.x == 0) pout[blockIdx.x] = sa;
        if (NC == 2 && threadIdx.x == 8 && have[NC - 1]) pout[blockIdx.x + G] = sb;
        gen_arrive(cnt + (j - i));
        double *t = pin;
        pin = pout;
        pout = t;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (have[c]) store8(wb, e0[c], n, b[c]);
}

// ---- residual VJP by a compressed Jacobian (Lorenz-96, tiny curvilinear grids) ----
//
// The residual of a cell depends only on cells at most two away along each
// grid direction: MUSCL reaches two cells along a face normal, the viscous
// gradients one cell across (the diamond's vertex values), the wall ghosts
// mirror cells within two of the wall, and Lorenz-96 reads u_{i-2} .. u_{i+1}.
// Cells whose indices agree modulo (px, py), both periods >= 5 (or the whole
// periodic extent), therefore never enter the same residual row.  One exact
// (dual-number) JVP along the direction that is 1 in variable q at every cell
// of such a class gives, in each row within two cells of a class member, the
// derivative of that row with respect to that member alone (the column
// grouping of Curtis, Powell and Reid).  g = J^T u at the member is the sum
// over those rows of D_r . u_r.  4 px py exact JVPs per product (px for
// Lorenz-96), each g entry written once with a fixed summation order.

// class period along a direction of n cells
int class_period(int n, bool periodic)
{
    if (!periodic) return 5;
    for (int p = 5; p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

// e = 1 in variable q at the cells i = ci (mod px), j = cj (mod py), else 0
__global__ void __launch_bounds__(AT) seed_kernel(double *__restrict__ e, int nx, int ny, int ncomp, int q, int ci,
                                                  int cj, int px, int py)
{
    const size_t nc = (size_t)nx * ny, n = nc * (size_t)ncomp;
    for (size_t t = (size_t)blockIdx.x * AT + threadIdx.x; t < n; t += (size_t)gridDim.x * AT) {
        const size_t cell = t % nc;
        const int k = (int)(t / nc), i = (int)(cell % nx), j = (int)(cell / nx);
        e[t] = (k == q && i % px == ci && j % py == cj) ? 1.0 : 0.0;
    }
}

// the rows along one direction that a member at index m reaches: m - 2 .. m + 2
// (wrapped when periodic, clipped otherwise), or all n rows of a periodic
// direction shorter than 5 (each row once)
__device__ __forceinline__ int row_of(int m, int o, int n, bool periodic, bool all)
{
    if (all) return o;
    int r = m + o;
    if (periodic) return ((r % n) + n) % n;
    return (r < 0 || r >= n) ? -1 : r;
}

// g[q][c] = sum over the rows r that member c of class (ci, cj) reaches of
// sum_k D[k][r] u[k][r]
__global__ void __launch_bounds__(AT) gather_kernel(double *__restrict__ g, const double *__restrict__ D,
                                                    const double *__restrict__ u, int nx, int ny, int ncomp, int q,
                                                    int ci, int cj, int px, int py, int perx, int pery)
{
    const size_t nc = (size_t)nx * ny;
    const int mx = (nx - ci + px - 1) / px, my = (ny - cj + py - 1) / py;
    const bool allx = perx && nx < 5, ally = pery && ny < 5;
    const int ox0 = allx ? 0 : -2, ox1 = allx ? nx - 1 : 2;
    const int oy0 = ally ? 0 : -2, oy1 = ally ? ny - 1 : 2;
    for (long long t = (long long)blockIdx.x * AT + threadIdx.x; t < (long long)mx * my;
         t += (long long)gridDim.x * AT) {
        const int i = ci + (int)(t % mx) * px, j = cj + (int)(t / mx) * py;
        double sum = 0.0;
        for (int oy = oy0; oy <= oy1; ++oy) {
            const int rj = row_of(j, oy, ny, pery != 0, ally);
            if (rj < 0) continue;
            for (int ox = ox0; ox <= ox1; ++ox) {
                const int ri = row_of(i, ox, nx, perx != 0, allx);
                if (ri < 0) continue;
                const size_t r = (size_t)rj * nx + ri;
                for (int k = 0; k < ncomp; ++k) sum += D[(size_t)k * nc + r] * u[(size_t)k * nc + r];
            }
        }
        g[(size_t)q * nc + (size_t)j * nx + i] = sum;
    }
}

// out1 += s1 (* s1dev) g, out2 += s2 (* s2dev) g
__global__ void __launch_bounds__(AT) vjp_apply_kernel(const VjpOut o, const double *__restrict__ g, size_t n)
{
    const double s1 = o.s1dev ? o.s1 * *o.s1dev : o.s1;
    const double s2 = o.s2dev ? o.s2 * *o.s2dev : o.s2;
    for (size_t e = (size_t)blockIdx.x * AT + threadIdx.x; e < n; e += (size_t)gridDim.x * AT) {
        if (o.out1) o.out1[e] = o.out1[e] + s1 * g[e];
        if (o.out2) o.out2[e] = o.out2[e] + s2 * g[e];
    }
}

// the curvilinear residual launch with other constants (the viscosity derivative)
rok_status curv_stencil_with(rok_ctx *c, const StencilConsts &Cx, const StencilIO &io)
{
    const cudaError_t e = c->strict ? strict::launch_curv(Cx, c->G, io, c->stream)
                                    : fast::launch_curv(Cx, c->G, io, c->stream);
    c->launches++;
    return e == cudaSuccess ? ROK_OK : ROK_ERR_CUDA;
}

// the constants with the viscosity (at T_ref under Sutherland's law) set to mu
StencilConsts with_mu(const StencilConsts &C0, double mu)
{
    StencilConsts C = C0;
    C.mu = mu;
    double g = 1.0;
    if (C.sutherland) {
        const double t = C.prim_inf[4] * C.inv_tref;
        g = (t * sqrt(t)) * ((1.0 + C.suth_s) / (t + C.suth_s));
    }
    C.prim_inf[5] = mu * g;
    set_fast_consts(C);
    return C;
}

rok_status vjp_colored(rok_ctx *c, AdjWork *A, const double *ystate, const double *ub, const VjpOut &o,
                       double *dst_mu, double mu_factor, const double *mu_dev, const double *dir,
                       const double *dir_scale)
{
    const StencilConsts &C = c->C;
    const bool lor = c->kind == ROK_LORENZ96;
    const int nx = C.nx, ny = lor ? 1 : C.ny, ncomp = lor ? 1 : 4;
    const bool perx = lor || C.bc[0] == ROK_BC_PERIODIC, pery = lor || C.bc[2] == ROK_BC_PERIODIC;
    const int px = class_period(nx, perx), py = class_period(ny, pery);
    const size_t N = c->N;
    const int eg = c->egrid;
    cudaStream_t s = c->stream;
    rok_status r;
    StencilIO io = rok_host::plain_io(c, ystate, A->cD);
    if (dir) {   // the state y + (*dir_scale) dir, formed in the stencil's load stage
        io.add[0] = dir;
        io.coef[0] = 1.0;
        io.coef_dev[0] = dir_scale;
        io.nadd = 1;
    }
    for (int cj = 0; cj < py && cj < ny; ++cj)
        for (int ci = 0; ci < px && ci < nx; ++ci) {
            const int members = ((nx - ci + px - 1) / px) * ((ny - cj + py - 1) / py);
            const int gb = (members + AT - 1) / AT;
            for (int q = 0; q < ncomp; ++q) {
                seed_kernel<<<eg, AT, 0, s>>>(A->cseed, nx, ny, ncomp, q, ci, cj, px, py);
                StencilIO jo = io;
                jo.dir = A->cseed;
                if ((r = rok_host::launch_stencil(c, jo)) != ROK_OK) return r;
                gather_kernel<<<gb, AT, 0, s>>>(A->cg, A->cD, ub, nx, ny, ncomp, q, ci, cj, px, py, perx, pery);
                c->launches += 2;
            }
        }
    vjp_apply_kernel<<<eg, AT, 0, s>>>(o, A->cg, N);
    c->launches++;
    if (dst_mu && !lor && C.viscous) {
        // d f / d mu = f(y; mu = 1) - f(y; mu = 0): the residual is affine in mu
        StencilIO fo = io;
        fo.out = A->cD;
        if ((r = curv_stencil_with(c, with_mu(C, 1.0), fo)) != ROK_OK) return r;
        fo.out = A->cseed;
        fo.sub = A->cD;
        fo.s1 = -1.0;
        if ((r = curv_stencil_with(c, with_mu(C, 0.0), fo)) != ROK_OK) return r;
        CU(c->ops->dot2(ub, A->cseed, nullptr, nullptr, N, A->cpart, c->P, nullptr, s));
        tree_add_kernel<<<1, AT, 0, s>>>(A->cpart, c->P, mu_factor, mu_dev, dst_mu);
        c->launches += 2;
    }
    CU(cudaGetLastError());
    return ROK_OK;
}

// ---- residual VJP on curvilinear grids: hand-written reverse sweep ----------
//
// The residual of a curvilinear grid (Sec. 3.2) is f_c = -(sum of the outward
// face fluxes F_f l_f) / V_c, each face flux the Roe flux of the MUSCL states
// through the face normal minus the viscous flux, whose gradients come from
// the diamond around the face (the two cells and the two vertices, a vertex
// value the mean of its four cells).  Boundary cells read ghosts: a periodic
// image, a wall mirror (velocity negated) or the free stream; a corner ghost
// applies the rule of the i-direction first, then that of the j-direction.
// Pass 1 (one thread per face) takes Fbar = l_f (ubar_R / V_R - ubar_L / V_L)
// back through one face: the Roe flux in the face's (normal, tangential)
// frame by the reverse sweep of the uniform grids, rotated back, and the
// viscous flux by hand; it stores 17 values a face: the adjoints of the two
// MUSCL states (8), of the cell differences and the vertex differences of
// u, v, T (6), of the face velocity (2) and of the face viscosity (1).
// Pass 2 (one thread per cell) gathers, in a fixed order, what every face
// gave to the cell and to each ghost that images it (mirrored adjoints
// negate u and v), and maps primitive adjoints to conserved ones.
constexpr int kCurvFaceVals = 17;

// source of an extended index e of a direction of n cells with boundary
// conditions lo / hi: the interior index, whether a wall mirrors it, or the
// free stream
struct ExtSrc {
    int i;
    bool flip, inf;
};
__device__ __forceinline__ ExtSrc ext_src1(int e, int n, int lo, int hi)
{
    if (e < 0) {
        if (lo == ROK_BC_PERIODIC) return {e + n, false, false};
        if (lo == ROK_BC_WALL) return {-1 - e, true, false};
        return {0, false, true};
    }
    if (e >= n) {
        if (hi == ROK_BC_PERIODIC) return {e - n, false, false};
        if (hi == ROK_BC_WALL) return {2 * n - 1 - e, true, false};
        return {0, false, true};
    }
    return {e, false, false};
}

// primitives (rho, u, v, p, T) of extended cell (ei, ej), ghosts included
__device__ __forceinline__ void ext_prim(const StencilConsts &C, const double *__restrict__ pr, size_t nc, int ei,
                                         int ej, double *w)
{
    const ExtSrc si = ext_src1(ei, C.nx, C.bc[0], C.bc[1]);
    bool flip = si.flip, inf = si.inf;
    int sj = 0;
    if (!inf) {
        const ExtSrc s2 = ext_src1(ej, C.ny, C.bc[2], C.bc[3]);
        flip = flip != s2.flip;
        inf = s2.inf;
        sj = s2.i;
    }
    if (inf) {
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = C.prim_inf[k];
    } else {
        const size_t c = (size_t)sj * C.nx + si.i;
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = pr[k * nc + c];
    }
    if (flip) {
        w[1] = -w[1];
        w[2] = -w[2];
    }
}

// u, v, T at vertex (vi, vj): the mean of its four cells, summed ((a + b) + c) + d
__device__ __forceinline__ void vertex_uvT(const StencilConsts &C, const double *__restrict__ pr, size_t nc, int vi,
                                           int vj, double *o)
{
    double a[5], b[5], c[5], d[5];
    ext_prim(C, pr, nc, vi - 1, vj - 1, a);
    ext_prim(C, pr, nc, vi, vj - 1, b);
    ext_prim(C, pr, nc, vi - 1, vj, c);
    ext_prim(C, pr, nc, vi, vj, d);
    o[0] = 0.25 * (((a[1] + b[1]) + c[1]) + d[1]);
    o[1] = 0.25 * (((a[2] + b[2]) + c[2]) + d[2]);
    o[2] = 0.25 * (((a[4] + b[4]) + c[4]) + d[4]);
}

// Pass 1 of a curvilinear grid: faces of direction D (0: i-faces, face (i, j)
// between cells (i-1, j) and (i, j), (nx+1) ny of them; 1: j-faces, face (i, j)
// between (i, j-1) and (i, j), nx (ny+1) of them).  fa[q * nf + f], q < 17
// (q < 8 without viscosity); one partial of ubar . df/dmu per CTA.
template <bool VISC, bool SUTH, int D>
__global__ void __launch_bounds__(FT, 7)
    curv_vjp_face_kernel(const StencilConsts C, const CurvGeom G, const double *__restrict__ pr,
                         const double *__restrict__ ub, double *__restrict__ fa, double *__restrict__ mupart)
{
    static_assert(FT == 64, "the CTA sum below adds two warp sums");
    __shared__ double sh[2];
    const int nx = C.nx, ny = C.ny;
    const size_t nc = (size_t)nx * ny;
    const int fw = D == 0 ? nx + 1 : nx;   // faces per row
    const size_t nf = D == 0 ? (size_t)(nx + 1) * ny : (size_t)nx * (ny + 1);
    const size_t t = (size_t)blockIdx.x * FT + threadIdx.x;
    double mu_c = 0.0;
    if (t < nf) {
        const int i = (int)(t % fw), j = (int)(t / fw);
        // the four cells along the grid line, the face between the middle two
        double m2[5], m1[5], p1[5], p2[5];
        if (D == 0) {
            ext_prim(C, pr, nc, i - 2, j, m2);
            ext_prim(C, pr, nc, i - 1, j, m1);
            ext_prim(C, pr, nc, i, j, p1);
            ext_prim(C, pr, nc, i + 1, j, p2);
        } else {
            ext_prim(C, pr, nc, i, j - 2, m2);
            ext_prim(C, pr, nc, i, j - 1, m1);
            ext_prim(C, pr, nc, i, j, p1);
            ext_prim(C, pr, nc, i, j + 1, p2);
        }
        const double nxf = D == 0 ? G.in_x[t] : G.jn_x[t], nyf = D == 0 ? G.in_y[t] : G.jn_y[t];
        const double len = D == 0 ? G.il[t] : G.jl[t];
        // Fbar = l (ubar_R / V_R - ubar_L / V_L) over the interior neighbours
        const int li = D == 0 ? i - 1 : i, lj = D == 0 ? j : j - 1;
        const bool lin = li >= 0 && lj >= 0, rin = i < nx && j < ny;
        const size_t lc = lin ? (size_t)lj * nx + li : 0, rc = rin ? (size_t)j * nx + i : 0;
        double Fb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double r = rin ? ub[k * nc + rc] * G.inv_vol[rc] : 0.0;
            const double l = lin ? ub[k * nc + lc] * G.inv_vol[lc] : 0.0;
            Fb[k] = len * (r - l);
        }
        double WL[4], WR[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) muscl(m2[k], m1[k], p1[k], p2[k], C.c_lo, C.c_hi, WL[k], WR[k]);
        // Roe flux in the frame (n, t), t = (-ny, nx): the x-direction flux of the
        // rotated states, rotated back (the flux is invariant under rotation)
        {
            const double Lr[4] = {WL[0], WL[1] * nxf + WL[2] * nyf, -WL[1] * nyf + WL[2] * nxf, WL[3]};
            const double Rr[4] = {WR[0], WR[1] * nxf + WR[2] * nyf, -WR[1] * nyf + WR[2] * nxf, WR[3]};
            const double Fbr[4] = {Fb[0], Fb[1] * nxf + Fb[2] * nyf, -Fb[1] * nyf + Fb[2] * nxf, Fb[3]};
            double Lb[4], Rb[4];
            roe_vjp<0>(Lr, Rr, C, Fbr, Lb, Rb);
            fa[0 * nf + t] = Lb[0];
            fa[1 * nf + t] = Lb[1] * nxf - Lb[2] * nyf;
            fa[2 * nf + t] = Lb[1] * nyf + Lb[2] * nxf;
            fa[3 * nf + t] = Lb[3];
            fa[4 * nf + t] = Rb[0];
            fa[5 * nf + t] = Rb[1] * nxf - Rb[2] * nyf;
            fa[6 * nf + t] = Rb[1] * nyf + Rb[2] * nxf;
            fa[7 * nf + t] = Rb[3];
        }
        if (VISC) {
            // diamond gradients: g = dC (c0, c2) + dV (c1, c3) for u, v, T; dC
            // across the face (cells), dV along it (vertex P3 minus vertex P1)
            double va[3], vb[3];
            if (D == 0) {
                vertex_uvT(C, pr, nc, i, j, va);
                vertex_uvT(C, pr, nc, i, j + 1, vb);
            } else {
                vertex_uvT(C, pr, nc, i + 1, j, va);
                vertex_uvT(C, pr, nc, i, j, vb);
            }
            const double c0 = D == 0 ? G.ic0[t] : G.jc0[t], c1 = D == 0 ? G.ic1[t] : G.jc1[t];
            const double c2 = D == 0 ? G.ic2[t] : G.jc2[t], c3 = D == 0 ? G.ic3[t] : G.jc3[t];
            const double dC[3] = {p1[1] - m1[1], p1[2] - m1[2], p1[4] - m1[4]};
            const double dV[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
            const double ux = dC[0] * c0 + dV[0] * c1, uy = dC[0] * c2 + dV[0] * c3;
            const double vx = dC[1] * c0 + dV[1] * c1, vy = dC[1] * c2 + dV[1] * c3;
            const double Tx = dC[2] * c0 + dV[2] * c1, Ty = dC[2] * c2 + dV[2] * c3;
            // face viscosity mu_ref gf (gf = 1 for a constant viscosity)
            double gf = 1.0;
            if (SUTH) {
                double dgl, dgr;
                gf = 0.5 * (suth_g(C, m1[4], dgl) + suth_g(C, p1[4], dgr));
            }
            const double mu = SUTH ? C.mu * gf : C.mu;
            const double div = ux + vy;
            const double sxx = 2.0 * ux - C.c23 * div, syy = 2.0 * vy - C.c23 * div, sxy = uy + vx;
            const double snx = sxx * nxf + sxy * nyf, sny = sxy * nxf + syy * nyf;
            const double dTn = Tx * nxf + Ty * nyf;
            const double uf = 0.5 * (m1[1] + p1[1]), vf = 0.5 * (m1[2] + p1[2]);
            // F -= Fv: Fv = mu (0, snx, sny, uf snx + vf sny + kfac dTn)
            const double Fv1b = -Fb[1], Fv2b = -Fb[2], Fv3b = -Fb[3];
            const double snxb = mu * (Fv1b + uf * Fv3b), snyb = mu * (Fv2b + vf * Fv3b);
            const double dTnb = (mu * C.kfac) * Fv3b;
            const double mufb = (Fv1b * snx + Fv2b * sny) + Fv3b * ((uf * snx + vf * sny) + C.kfac * dTn);
            const double sxxb = snxb * nxf, syyb = snyb * nyf, sxyb = snxb * nyf + snyb * nxf;
            const double uxb = 2.0 * sxxb - C.c23 * (sxxb + syyb), vyb = 2.0 * syyb - C.c23 * (sxxb + syyb);
            const double uyb = sxyb, vxb = sxyb, Txb = dTnb * nxf, Tyb = dTnb * nyf;
            fa[8 * nf + t] = uxb * c0 + uyb * c2;    // dC of u
            fa[9 * nf + t] = vxb * c0 + vyb * c2;    // dC of v
            fa[10 * nf + t] = Txb * c0 + Tyb * c2;   // dC of T
            fa[11 * nf + t] = uxb * c1 + uyb * c3;   // dV of u
            fa[12 * nf + t] = vxb * c1 + vyb * c3;   // dV of v
            fa[13 * nf + t] = Txb * c1 + Tyb * c3;   // dV of T
            fa[14 * nf + t] = mu * snx * Fv3b;       // face u
            fa[15 * nf + t] = mu * sny * Fv3b;       // face v
            fa[16 * nf + t] = mufb;                  // face viscosity
            mu_c = SUTH ? mufb * gf : mufb;          // d mu_f / d mu_ref = gf
        }
    }
    const double s = lane_tree(mu_c);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) mupart[blockIdx.x] = sh[0] + sh[1];
}

// the extended indices of a direction (n >= 2 cells, boundary conditions
// lo / hi) that image interior index i: itself and the ghosts copied or
// mirrored from it (at most one on each side: the two ghost layers of a side
// come from different interior indices)
__device__ __forceinline__ int ext_images(int i, int n, int lo, int hi, int *e, bool *flip)
{
    int k = 0;
    e[k] = i;
    flip[k++] = false;
#pragma unroll
    for (int g = 1; g <= 2; ++g) {
        if (lo == ROK_BC_PERIODIC && i == n - g) { e[k] = -g; flip[k++] = false; }
        if (lo == ROK_BC_WALL && i == g - 1) { e[k] = -g; flip[k++] = true; }
        if (hi == ROK_BC_PERIODIC && i == g - 1) { e[k] = n - 1 + g; flip[k++] = false; }
        if (hi == ROK_BC_WALL && i == n - g) { e[k] = n - 1 + g; flip[k++] = true; }
    }
    return k;
}

// Pass 2 of a curvilinear grid: g = J^T ubar at each cell from the face values
// (fx: i-faces, fy: j-faces); out1 += s1 g, out2 += s2 g
template <bool VISC, bool SUTH>
__global__ void __launch_bounds__(AT) curv_vjp_cell_kernel(const StencilConsts C, const double *__restrict__ pr,
                                                           const double *__restrict__ fx,
                                                           const double *__restrict__ fy, const VjpOut o)
{
    const int nx = C.nx, ny = C.ny;
    const size_t nc = (size_t)nx * ny;
    const size_t nfx = (size_t)(nx + 1) * ny, nfy = (size_t)nx * (ny + 1);
    const size_t t = (size_t)blockIdx.x * AT + threadIdx.x;
    if (t >= nc) return;
    const int i = (int)(t % nx), j = (int)(t / nx);
    // face values, 0 where the face does not exist
    auto FX = [&](int q, int a, int b) -> double {
        return (a >= 0 && a <= nx && b >= 0 && b < ny) ? fx[q * nfx + (size_t)b * (nx + 1) + a] : 0.0;
    };
    auto FY = [&](int q, int a, int b) -> double {
        return (a >= 0 && a < nx && b >= 0 && b <= ny) ? fy[q * nfy + (size_t)b * nx + a] : 0.0;
    };
    const double a1 = (1.0 + C.c_lo) - C.c_hi;
    int ex[3], ey[3];
    bool flx[3], fly[3];
    const int nix = ext_images(i, nx, C.bc[0], C.bc[1], ex, flx);
    const int niy = ext_images(j, ny, C.bc[2], C.bc[3], ey, fly);
    double Pb[4] = {0.0, 0.0, 0.0, 0.0}, Tb = 0.0, mub = 0.0;
    for (int a = 0; a < nix; ++a)
        for (int b = 0; b < niy; ++b) {
            const int ei = ex[a], ej = ey[b];
            double pb[4] = {0.0, 0.0, 0.0, 0.0}, tb = 0.0;
            // MUSCL: the cell is m2 of face e+2, m1 of face e+1, p1 of face e, p2 of face e-1
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double s = -C.c_lo * FX(k, ei + 2, ej);
                s = s + (a1 * FX(k, ei + 1, ej) + C.c_hi * FX(k + 4, ei + 1, ej));
                s = s + (C.c_hi * FX(k, ei, ej) + a1 * FX(k + 4, ei, ej));
                s = s - C.c_lo * FX(k + 4, ei - 1, ej);
                s = s - C.c_lo * FY(k, ei, ej + 2);
                s = s + (a1 * FY(k, ei, ej + 1) + C.c_hi * FY(k + 4, ei, ej + 1));
                s = s + (C.c_hi * FY(k, ei, ej) + a1 * FY(k + 4, ei, ej));
                s = s - C.c_lo * FY(k + 4, ei, ej - 1);
                pb[k] = s;
            }
            if (VISC) {
                // right cell of faces (ei, ej) [i] and (ei, ej) [j], left cell of
                // faces (ei + 1, ej) [i] and (ei, ej + 1) [j]
                pb[1] += ((FX(8, ei, ej) - FX(8, ei + 1, ej)) + 0.5 * (FX(14, ei, ej) + FX(14, ei + 1, ej))) +
                         ((FY(8, ei, ej) - FY(8, ei, ej + 1)) + 0.5 * (FY(14, ei, ej) + FY(14, ei, ej + 1)));
                pb[2] += ((FX(9, ei, ej) - FX(9, ei + 1, ej)) + 0.5 * (FX(15, ei, ej) + FX(15, ei + 1, ej))) +
                         ((FY(9, ei, ej) - FY(9, ei, ej + 1)) + 0.5 * (FY(15, ei, ej) + FY(15, ei, ej + 1)));
                tb += (FX(10, ei, ej) - FX(10, ei + 1, ej)) + (FY(10, ei, ej) - FY(10, ei, ej + 1));
                if (SUTH)
                    mub += 0.5 * ((FX(16, ei, ej) + FX(16, ei + 1, ej)) + (FY(16, ei, ej) + FY(16, ei, ej + 1)));
                // vertex (vi, vj) is P1 of i-face (vi, vj) and of j-face (vi - 1, vj),
                // P3 of i-face (vi, vj - 1) and of j-face (vi, vj); the cell is one
                // of the four around vertices (ei, ej), (ei+1, ej), (ei, ej+1), (ei+1, ej+1)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double s = 0.0;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int vi = ei + (v & 1), vj = ej + (v >> 1);
                        s += ((FX(11 + q, vi, vj - 1) - FX(11 + q, vi, vj)) +
                              (FY(11 + q, vi, vj) - FY(11 + q, vi - 1, vj)));
                    }
                    if (q < 2) pb[1 + q] += 0.25 * s;
                    else tb += 0.25 * s;
                }
            }
            const double sg = (flx[a] != fly[b]) ? -1.0 : 1.0;   // a mirror image negates u and v
            Pb[0] += pb[0];
            Pb[1] += sg * pb[1];
            Pb[2] += sg * pb[2];
            Pb[3] += pb[3];
            Tb += tb;
        }
    double P[4], T;
    prim_load(pr, nc, t, P, T);
    if (SUTH) {
        double dg;
        suth_g(C, T, dg);
        Tb += mub * (C.mu * dg);
    }
    const double rho = P[0], u = P[1], v = P[2];
    const double rinv = 1.0 / rho;
    // T = p / rho
    Pb[3] += Tb * rinv;
    Pb[0] -= Tb * T * rinv;
    double qb[4];
    qb[0] = (Pb[0] - (u * Pb[1] + v * Pb[2]) * rinv) + C.gm1 * 0.5 * (u * u + v * v) * Pb[3];
    qb[1] = Pb[1] * rinv - C.gm1 * u * Pb[3];
    qb[2] = Pb[2] * rinv - C.gm1 * v * Pb[3];
    qb[3] = C.gm1 * Pb[3];
    const double s1 = o.s1dev ? o.s1 * *o.s1dev : o.s1;
    const double s2 = o.s2dev ? o.s2 * *o.s2dev : o.s2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t e = (size_t)k * nc + t;
        if (o.out1) o.out1[e] = o.out1[e] + s1 * qb[k];
        if (o.out2) o.out2[e] = o.out2[e] + s2 * qb[k];
    }
}

// the reverse sweep covers curvilinear grids of at least 2 x 2 cells; smaller
// ones and Lorenz-96 take the compressed Jacobian
bool curv_sweep(const rok_ctx *c) { return c->curv && c->C.nx >= 2 && c->C.ny >= 2; }
bool colored(const rok_ctx *c) { return c->kind == ROK_LORENZ96 || (c->curv && !curv_sweep(c)); }

rok_status vjp_curv(rok_ctx *c, AdjWork *A, const double *ystate, const double *ub, const VjpOut &o,
                    double *dst_mu, double mu_factor, const double *mu_dev, const double *dir,
                    const double *dir_scale)
{
    const StencilConsts &C = c->C;
    const size_t nc = c->nc;
    const size_t nfx = (size_t)(C.nx + 1) * C.ny, nfy = (size_t)C.nx * (C.ny + 1);
    const int nb = (int)((nc + AT - 1) / AT);
    const int gx = (int)((nfx + FT - 1) / FT), gy = (int)((nfy + FT - 1) / FT);
    double *fxa = A->cfaces, *fya = A->cfaces + kCurvFaceVals * nfx;
    cudaStream_t s = c->stream;
    prim_kernel<<<nb, AT, 0, s>>>(C, ystate, dir, dir_scale, A->prims);
    if (C.viscous && C.sutherland) {
        curv_vjp_face_kernel<true, true, 0><<<gx, FT, 0, s>>>(C, c->G, A->prims, ub, fxa, A->cmupart);
        curv_vjp_face_kernel<true, true, 1><<<gy, FT, 0, s>>>(C, c->G, A->prims, ub, fya, A->cmupart + gx);
        curv_vjp_cell_kernel<true, true><<<nb, AT, 0, s>>>(C, A->prims, fxa, fya, o);
    } else if (C.viscous) {
        curv_vjp_face_kernel<true, false, 0><<<gx, FT, 0, s>>>(C, c->G, A->prims, ub, fxa, A->cmupart);
        curv_vjp_face_kernel<true, false, 1><<<gy, FT, 0, s>>>(C, c->G, A->prims, ub, fya, A->cmupart + gx);
        curv_vjp_cell_kernel<true, false><<<nb, AT, 0, s>>>(C, A->prims, fxa, fya, o);
    } else {
        curv_vjp_face_kernel<false, false, 0><<<gx, FT, 0, s>>>(C, c->G, A->prims, ub, fxa, A->cmupart);
        curv_vjp_face_kernel<false, false, 1><<<gy, FT, 0, s>>>(C, c->G, A->prims, ub, fya, A->cmupart + gx);
        curv_vjp_cell_kernel<false, false><<<nb, AT, 0, s>>>(C, A->prims, fxa, fya, o);
    }
    c->launches += 4;
    if (dst_mu && C.viscous) {
        tree_add_kernel<<<1, AT, 0, s>>>(A->cmupart, gx + gy, mu_factor, mu_dev, dst_mu);
        c->launches++;
    }
    CU(cudaGetLastError());
    return ROK_OK;
}

// residual VJP launches: out1 += s1 g, out2 += s2 g with g = J(ystate)^T ubar;
// dst_mu += mu_factor (* mu_dev) ubar . df/dmu(ystate)
rok_status vjp(rok_ctx *c, AdjWork *A, const double *ystate, const double *ub, const VjpOut &o, double *dst_mu,
               double mu_factor, const double *mu_dev, const double *dir = nullptr, const double *dir_scale = nullptr)
{
    if (curv_sweep(c)) return vjp_curv(c, A, ystate, ub, o, dst_mu, mu_factor, mu_dev, dir, dir_scale);
    if (colored(c)) return vjp_colored(c, A, ystate, ub, o, dst_mu, mu_factor, mu_dev, dir, dir_scale);
    const StencilConsts &C = c->C;
    const size_t nc = (size_t)C.nx * C.ny;
    const int nb = (int)((nc + AT - 1) / AT);
    const int nf = (int)((nc + FT - 1) / FT);
    double *fxa = A->faces, *fya = A->faces + kFaceVals * nc;
    cudaStream_t s = c->stream;
    prim_kernel<<<nb, AT, 0, s>>>(C, ystate, dir, dir_scale, A->prims);
    if (C.viscous && C.sutherland) {
        vjp_face_kernel<true, true, 0><<<nf, FT, 0, s>>>(C, A->prims, ub, fxa, A->mupart);
        vjp_face_kernel<true, true, 1><<<nf, FT, 0, s>>>(C, A->prims, ub, fya, A->mupart + nf);
        vjp_cell_kernel<true, true><<<nb, AT, 0, s>>>(C, A->prims, fxa, fya, o);
    } else if (C.viscous) {
        vjp_face_kernel<true, false, 0><<<nf, FT, 0, s>>>(C, A->prims, ub, fxa, A->mupart);
        vjp_face_kernel<true, false, 1><<<nf, FT, 0, s>>>(C, A->prims, ub, fya, A->mupart + nf);
        vjp_cell_kernel<true, false><<<nb, AT, 0, s>>>(C, A->prims, fxa, fya, o);
    } else {
        vjp_face_kernel<false, false, 0><<<nf, FT, 0, s>>>(C, A->prims, ub, fxa, A->mupart);
        vjp_face_kernel<false, false, 1><<<nf, FT, 0, s>>>(C, A->prims, ub, fya, A->mupart + nf);
        vjp_cell_kernel<false, false><<<nb, AT, 0, s>>>(C, A->prims, fxa, fya, o);
    }
    c->launches += 4;
    if (dst_mu && C.viscous) {
        tree_add_kernel<<<1, AT, 0, s>>>(A->mupart, 2 * nf, mu_factor, mu_dev, dst_mu);
        c->launches++;
    }
    CU(cudaGetLastError());
    return ROK_OK;
}

// the reverse of a step: every grid, problem kind and basis, but not the
// exact-JVP step (the derivative of J(y) v in y is a second derivative of f)
rok_status step_reverse_supported(const rok_ctx *c) { return c->exact_jvp ? ROK_ERR_UNSUPPORTED : ROK_OK; }

void free_work(AdjWork *A)
{
    if (!A) return;
    cudaFree(A->Vb);
    for (int i = 0; i < 4; ++i) cudaFree(A->kb[i]);
    cudaFree(A->yb); cudaFree(A->Fb); cudaFree(A->F1b); cudaFree(A->F1acc);
    cudaFree(A->wb); cudaFree(A->wcur); cudaFree(A->wlast); cudaFree(A->Yt); cudaFree(A->y1);
    cudaFree(A->pA); cudaFree(A->pB); cudaFree(A->pM);
    cudaFree(A->faces); cudaFree(A->prims); cudaFree(A->mupart); cudaFree(A->as);
    cudaFree(A->cseed); cudaFree(A->cD); cudaFree(A->cg); cudaFree(A->cpart);
    cudaFree(A->cfaces); cudaFree(A->cmupart);
    cudaFreeHost(A->h_st); cudaFreeHost(A->h_mub);
    delete A;
}

rok_status ensure_work(rok_ctx *c, bool full)
{
    if (c->adj && (!full || c->adj->Vb)) return ROK_OK;
    AdjWork *A = c->adj ? c->adj : new AdjWork();
    c->adj = A;
    const size_t N = c->N, nc = c->nc;
    A->N = N;
    A->P = c->P;
    A->M = c->mmax;
    auto al = [&](double **p, size_t n) { return cudaMalloc(p, n * sizeof(double)) == cudaSuccess; };
    bool ok = true;
    if (!A->prims) {
        // face values of the uniform-grid sweep (curvilinear grids keep theirs in cfaces)
        const bool uniform = !c->curv && c->kind != ROK_LORENZ96;
        A->nmu = 2 * (int)((nc + FT - 1) / FT);
        ok = al(&A->prims, 5 * nc) && al(&A->mupart, A->nmu) && (!uniform || al(&A->faces, 2 * kFaceVals * nc)) &&
             cudaMalloc(&A->as, sizeof(AdjState)) == cudaSuccess &&
             cudaMallocHost(&A->h_mub, sizeof(double)) == cudaSuccess;
    }
    if (ok && colored(c) && !A->cseed)
        ok = al(&A->cseed, N) && al(&A->cD, N) && al(&A->cg, N) && al(&A->cpart, 2 * (size_t)c->P);
    if (ok && curv_sweep(c) && !A->cfaces) {
        const size_t nfx = (size_t)(c->C.nx + 1) * c->C.ny, nfy = (size_t)c->C.nx * (c->C.ny + 1);
        ok = al(&A->cfaces, kCurvFaceVals * (nfx + nfy)) &&
             al(&A->cmupart, (nfx + FT - 1) / FT + (nfy + FT - 1) / FT);
    }
    if (ok && full) {
        ok = al(&A->Vb, (size_t)(c->mmax > 0 ? c->mmax : 1) * N) && al(&A->yb, N) && al(&A->Fb, N) &&
             al(&A->F1b, N) && al(&A->F1acc, N) && al(&A->wb, N) && al(&A->wcur, N) && al(&A->wlast, N) &&
             al(&A->Yt, N) && al(&A->y1, N) && al(&A->pA, 2 * (size_t)c->P) && al(&A->pB, 2 * (size_t)c->P) &&
             al(&A->pM, (size_t)(c->mmax > 0 ? c->mmax : 1) * c->P) &&
             cudaMallocHost(&A->h_st, sizeof(StepState)) == cudaSuccess;
        for (int i = 0; i < 4 && ok; ++i) ok = al(&A->kb[i], N);
    }
    if (!ok) {
        free_work(A);
        c->adj = nullptr;
        return ROK_ERR_NOMEM;
    }
    return ROK_OK;
}

inline int egrid(const rok_ctx *c) { return c->egrid; }

// co-resident CTAs of mgsrev_column_kernel (0 without cooperative launch)
int rev_column_ctas()
{
    int dev = 0, coop = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgsrev_column_kernel<2>, RT, 0) != cudaSuccess) return 0;
    return per * sms;
}

}  // namespace

void rok_free_adjoint(rok_ctx *c)
{
    if (c && c->adj) {
        free_work(c->adj);
        c->adj = nullptr;
    }
}

// ---- the two halves of the reverse step ------------------------------------------

// The step from y_n once more, keeping what its reverse reads: the basis V, H
// and the LU of (I - h gamma H), lambda_i and phi_i (all in the StepState), the
// F_i and k_i (in the context), and the last column's orthogonalised w, which
// the step itself does not keep (in A->wlast).  y_{n+1} is left in A->y1;
// *m_out = the Krylov dimension built.  Synchronises once (status, m).
static rok_status step_internals(rok_ctx *c, const double *y, double h, int M, int *m_out)
{
    AdjWork *A = c->adj;
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    AdjState *as = A->as;
    cudaStream_t s = c->stream;
    const LinalgOps &ops = *c->ops;
    rok_status r;
    CU(cudaMemcpyAsync(A->y1, y, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(launch_begin(st, h, kRokGamma, M, s));
    if ((r = rok_host::enqueue_step_body(c, A->y1, M)) != ROK_OK) return r;
    CU(cudaMemcpyAsync(A->h_st, st, offsetof(StepState, H), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (A->h_st->status) {
        CU(launch_set_int(&st->status, 0, s));
        return (A->h_st->status & kStatusTimeout) ? ROK_ERR_TIMEOUT : ROK_ERR_NONFINITE;
    }
    const int m = A->h_st->meff;
    *m_out = m;
    // binary32 basis: widened exactly into the binary64 basis array, on which
    // the recomputed last column below and the reverse run.  The classical
    // Gram-Schmidt of the FMA build and MGS give the same V and H in exact
    // arithmetic, so the reverse of MGS is the derivative of either (at the
    // rounded basis).
    if (c->fp32 && m > 0) CU(launch_f2d(c->Vf, c->V, (size_t)m * N, s));
    // the last column's orthogonalised w (not kept by the step): its JVP and MGS
    // passes again, H entries to scratch
    if (m > 0) {
        StencilIO io = rok_host::plain_io(c, y, A->wlast);
        io.add[0] = c->V + (size_t)(m - 1) * N;
        io.coef[0] = 1.0;
        io.coef_dev[0] = &st->eps;
        io.nadd = 1;
        io.sub = c->F[0];
        io.s1_dev = &st->inv_eps;
        if ((r = rok_host::launch_stencil(c, io)) != ROK_OK) return r;
        CU(launch_set_int(&st->active, 1, s));
        CU(ops.dot2(c->V, A->wlast, A->wlast, A->wlast, N, A->pA, P, nullptr, s));
        double *pin = A->pA, *pout = A->pB;
        for (int i = 1; i <= m; ++i) {
            const double *vnext = i < m ? c->V + (size_t)i * N : nullptr;
            CU(ops.mgs(A->wlast, c->V + (size_t)(i - 1) * N, vnext, N, pin, P, &as->scratch[0], pout, i == 1, st, s));
            double *t = pin; pin = pout; pout = t;
        }
        c->launches += 2 + m;
    }
    return ROK_OK;
}

// The reverse of the step from y_n, its internals in place (step_internals, or
// a tape copied back): ybar_out = (dy_{n+1}/dy_n)^T ybar_in, mubar += the
// step's viscosity part.
static rok_status step_reverse(rok_ctx *c, const double *y, double h, int m, const double *ybar_in,
                               double *ybar_out, double *mubar)
{
    AdjWork *A = c->adj;
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    AdjState *as = A->as;
    cudaStream_t s = c->stream;
    const LinalgOps &ops = *c->ops;
    const int eg = egrid(c);
    rok_status r;
    // 2. stages in reverse: y_{n+1} = y_n + sum b_i k_i
    CU(cudaMemsetAsync(as, 0, sizeof(AdjState), s));
    CU(cudaMemcpyAsync(A->yb, ybar_in, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < 4; ++i) {
        lin2_kernel<<<eg, AT, 0, s>>>(A->kb[i], nullptr, 0.0, ybar_in, kRokB[i], nullptr, N);
        c->launches++;
    }
    for (int i = 3; i >= 0; --i) {
        if (m > 0) {
            CU(ops.multidot(A->kb[i], c->V, 0, N, N, A->pM, P, st, s));
            GamRowA gr;
            for (int j = 0; j < 4; ++j) gr.g[j] = kRokGammaOff[i][j];
            stage_rev_kernel<<<1, AT, 0, s>>>(i, gr, A->pM, P, st, as);
            fbar_kernel<<<eg, AT, 0, s>>>(A->Fb, A->kb[i], h, c->V, N, N, as->phib[i], st);
            c->launches += 3;
        } else {
            lin2_kernel<<<eg, AT, 0, s>>>(A->Fb, nullptr, 0.0, A->kb[i], h, nullptr, N);
            c->launches++;
        }
        if (i == 0) {
            CU(cudaMemcpyAsync(A->F1b, A->Fb, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
            continue;
        }
        // Y_i = y + sum_j alpha_ij k_j ; F_i = f(Y_i)
        const double *kv[4];
        double cf[4];
        int cnt = 0;
        for (int j = 0; j < i; ++j)
            if (kRokAlpha[i][j] != 0.0) { kv[cnt] = c->K[j]; cf[cnt] = kRokAlpha[i][j]; cnt++; }
        CU(ops.axpy_n(A->Yt, y, kv, cf, cnt, N, nullptr, eg, s));
        c->launches++;
        // g = J(Y_i)^T Fbar: ybar += g, kbar_j += alpha_ij g (one alpha per row here; others by a copy)
        int jlast = -1;
        for (int j = 0; j < i; ++j)
            if (kRokAlpha[i][j] != 0.0) jlast = j;
        VjpOut o{A->yb, 1.0, nullptr, jlast >= 0 ? A->kb[jlast] : nullptr, jlast >= 0 ? kRokAlpha[i][jlast] : 0.0,
                 nullptr};
        if (cnt > 1) {
            // general tableau: keep g in wb, then add it to every k_j
            CU(cudaMemsetAsync(A->wb, 0, N * sizeof(double), s));
            VjpOut og{A->wb, 1.0, nullptr, nullptr, 0.0, nullptr};
            if ((r = vjp(c, A, A->Yt, A->Fb, og, &as->mub, 1.0, nullptr)) != ROK_OK) return r;
            lin2_kernel<<<eg, AT, 0, s>>>(A->yb, A->yb, 1.0, A->wb, 1.0, nullptr, N);
            for (int j = 0; j < i; ++j)
                if (kRokAlpha[i][j] != 0.0)
                    lin2_kernel<<<eg, AT, 0, s>>>(A->kb[j], A->kb[j], 1.0, A->wb, kRokAlpha[i][j], nullptr, N);
        } else if ((r = vjp(c, A, A->Yt, A->Fb, o, &as->mub, 1.0, nullptr)) != ROK_OK) {
            return r;
        }
    }

    // 3. Arnoldi in reverse
    if (m > 0) {
        assemble_vb_kernel<<<eg, AT, 0, s>>>(A->Vb, N, N, A->kb[0], A->kb[1], A->kb[2], A->kb[3], c->F[0], c->F[1],
                                             c->F[2], c->F[3], st, as);
        CU(cudaMemsetAsync(A->F1acc, 0, N * sizeof(double), s));
        c->launches++;
        // arrival counters of the cooperative reverse launches: column j takes j
        CU(cudaMemsetAsync(c->colcnt, 0, column_counter_offset(m) * sizeof(unsigned), s));
        unsigned *cnt = c->colcnt;
        for (int j = m - 1; j >= 0; --j) {
            const double *vj = c->V + (size_t)j * N;
            if (j + 1 < m) {
                const double *v1 = c->V + (size_t)(j + 1) * N;
                double *vb1 = A->Vb + (size_t)(j + 1) * N;
                CU(ops.dot2(v1, vb1, nullptr, nullptr, N, A->pA, P, nullptr, s));
                // wbar from the normalisation's reverse, and wcur = h_{j+1,j} v_{j+1}
                normrev_kernel<<<eg, AT, 0, s>>>(A->wb, nullptr, vb1, v1, N, A->pA, P,
                                                 &st->H[(j + 1) * kMaxKrylov + j], &as->Hb[(j + 1) * kMaxKrylov + j],
                                                 A->wcur);
                c->launches += 2;
            } else {
                CU(cudaMemsetAsync(A->wb, 0, N * sizeof(double), s));
                CU(cudaMemcpyAsync(A->wcur, A->wlast, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
            }
            if (A->rev_ctas < 0) A->rev_ctas = rev_column_ctas();
            const int G = P < A->rev_ctas ? P : A->rev_ctas;
            CU(ops.dot2(vj, A->wb, nullptr, nullptr, N, A->pA, P, nullptr, s));
            c->launches++;
            if (c->persistent && G > 0 && (P + G - 1) / G <= kColChunks) {
                // all j + 1 reverse passes in one cooperative launch
                double *wbp = A->wb, *pa = A->pA, *pb = A->pB;
                const double *wcp = A->wcur, *Vp = c->V;
                double *Vbp = A->Vb;
                size_t ldv = N, nn = N;
                int jj = j, PP = P;
                unsigned *cntp = cnt;
                StepState *stp = st;
                const AdjState *asp = as;
                void *args[] = {&wbp, &wcp, &Vbp, &Vp, &ldv, &nn, &jj, &PP, &pa, &pb, &cntp, &stp, &asp};
                // one chunk per CTA when the grid covers them all (the one-chunk
                // kernel needs fewer registers, so it is co-resident wherever
                // the two-chunk one is)
                const void *fn = G >= P ? (const void *)mgsrev_column_kernel<1> : (const void *)mgsrev_column_kernel<2>;
                CU(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(RT), args, 0, s));
                cnt += j;
                c->launches++;
            } else {
                double *pin = A->pA, *pout = A->pB;
                for (int i = j; i >= 0; --i) {
                    const double *vi = c->V + (size_t)i * N;
                    const double *vprev = i > 0 ? c->V + (size_t)(i - 1) * N : nullptr;
                    mgsrev_kernel<<<P, RT, 0, s>>>(A->wb, A->wcur, A->Vb + (size_t)i * N, vi, vprev, N, pin, P,
                                                   &st->H[i * kMaxKrylov + j], &as->Hb[i * kMaxKrylov + j], pout);
                    c->launches++;
                    double *t = pin; pin = pout; pout = t;
                }
            }
            // w_0 = (f(y + eps v_j) - F1) / eps (the state formed in the primitives pass)
            VjpOut o{A->Vb + (size_t)j * N, 1.0, nullptr, A->yb, 1.0, &st->inv_eps};
            if ((r = vjp(c, A, y, A->wb, o, &as->mub, 1.0, &st->inv_eps, vj, &st->eps)) != ROK_OK) return r;
            lin2_kernel<<<eg, AT, 0, s>>>(A->F1acc, A->F1acc, 1.0, A->wb, 1.0, nullptr, N);
            c->launches++;
        }
        // v_1 = F1 / beta
        CU(ops.dot2(c->V, A->Vb, nullptr, nullptr, N, A->pA, P, nullptr, s));
        normrev_kernel<<<eg, AT, 0, s>>>(A->F1b, A->F1b, A->Vb, c->V, N, A->pA, P, &st->beta, nullptr, nullptr);
        lin2_kernel<<<eg, AT, 0, s>>>(A->F1b, A->F1b, 1.0, A->F1acc, -1.0, &st->inv_eps, N);
        c->launches += 3;
    }
    // 4. F1 = f(y_n)
    VjpOut o{A->yb, 1.0, nullptr, nullptr, 0.0, nullptr};
    if ((r = vjp(c, A, y, A->F1b, o, &as->mub, 1.0, nullptr)) != ROK_OK) return r;
    CU(cudaMemcpyAsync(ybar_out, A->yb, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (mubar) {
        CU(cudaMemcpyAsync(A->h_mub, &as->mub, sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        *mubar = c->C.viscous ? *A->h_mub : 0.0;
    }
    CU(cudaGetLastError());
    return ROK_OK;
}


// ---- tapes: one step's internals kept for its reverse ----------------------------
//
// [0, 256)         TapeHeader
// [256, ...)       the StepState after step_internals
// then 10 + M vectors of N float64, each on a 256-byte boundary: y_n, F_1..F_4,
// k_1..k_4, the last column's orthogonalised w, and the basis v_1..v_m (m <= M)
constexpr unsigned long long kTapeMagic = 0x45504154344b4f52ull;   // bytes "ROK4TAPE"
constexpr size_t kTapeAlign = 256;

struct TapeHeader {
    unsigned long long magic;
    unsigned long long n;   // state entries
    int M, m;               // Krylov dimension asked for / built
    double h;
};

struct TapeLayout {
    size_t st, vec, stride, bytes;
};

static size_t tape_round(size_t b) { return (b + kTapeAlign - 1) / kTapeAlign * kTapeAlign; }

static TapeLayout tape_layout(size_t N, int M)
{
    TapeLayout L;
    L.st = kTapeAlign;
    L.vec = L.st + tape_round(sizeof(StepState));
    L.stride = tape_round(N * sizeof(double));
    L.bytes = L.vec + (size_t)(10 + M) * L.stride;
    return L;
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

extern "C" {

rok_status rok_vjp(rok_ctx *c, const double *y, const double *ubar, double *ybar, double *mubar)
{
    if (!c || !y || !ubar || !ybar || ybar == y || ybar == ubar) return ROK_ERR_INVALID_ARG;
    rok_status r;
    if ((r = ensure_work(c, false)) != ROK_OK) return r;
    AdjWork *A = c->adj;
    CU(cudaMemsetAsync(ybar, 0, c->N * sizeof(double), c->stream));
    if (mubar) CU(cudaMemsetAsync(&A->as->mub, 0, sizeof(double), c->stream));
    VjpOut o{ybar, 1.0, nullptr, nullptr, 0.0, nullptr};
    if ((r = vjp(c, A, y, ubar, o, mubar ? &A->as->mub : nullptr, 1.0, nullptr)) != ROK_OK) return r;
    if (mubar) {
        if (!c->C.viscous) {
            *mubar = 0.0;
            return ROK_OK;
        }
        CU(cudaMemcpyAsync(A->h_mub, &A->as->mub, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        *mubar = *A->h_mub;
    }
    return ROK_OK;
}

rok_status rok_step_vjp(rok_ctx *c, const double *y, double h, int M, const double *ybar_in, double *ybar_out,
                        double *mubar)
{
    if (!c || !y || !ybar_in || !ybar_out || M < 0 || M > c->mmax || !(h > 0.0) || !isfinite(h))
        return ROK_ERR_INVALID_ARG;
    if (ybar_out == y) return ROK_ERR_INVALID_ARG;
    rok_status r = step_reverse_supported(c);
    if (r != ROK_OK) return r;
    if ((r = ensure_work(c, true)) != ROK_OK) return r;
    int m = 0;
    if ((r = step_internals(c, y, h, M, &m)) != ROK_OK) return r;
    return step_reverse(c, y, h, m, ybar_in, ybar_out, mubar);
}

rok_status rok_tape_bytes(rok_ctx *c, int M, size_t *bytes)
{
    if (!c || !bytes || M < 0 || M > c->mmax) return ROK_ERR_INVALID_ARG;
    *bytes = tape_layout(c->N, M).bytes;
    return ROK_OK;
}

rok_status rok_step_record(rok_ctx *c, double *y, double h, int M, void *tape)
{
    if (!c || !y || !tape || M < 0 || M > c->mmax || !(h > 0.0) || !isfinite(h)) return ROK_ERR_INVALID_ARG;
    const size_t N = c->N, vb = N * sizeof(double);
    const TapeLayout L = tape_layout(N, M);
    if ((uintptr_t)tape % kTapeAlign || overlaps(y, vb, tape, L.bytes)) return ROK_ERR_INVALID_ARG;
    rok_status r = step_reverse_supported(c);
    if (r != ROK_OK) return r;
    if ((r = ensure_work(c, true)) != ROK_OK) return r;
    AdjWork *A = c->adj;
    cudaStream_t s = c->stream;
    int m = 0;
    if ((r = step_internals(c, y, h, M, &m)) != ROK_OK) return r;
    char *t = (char *)tape;
    auto vec = [&](int k) { return t + L.vec + (size_t)k * L.stride; };
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    CU(cudaMemcpyAsync(t + L.st, c->st, sizeof(StepState), dd, s));
    CU(cudaMemcpyAsync(vec(0), y, vb, dd, s));
    for (int i = 0; i < 4; ++i) {
        CU(cudaMemcpyAsync(vec(1 + i), c->F[i], vb, dd, s));
        CU(cudaMemcpyAsync(vec(5 + i), c->K[i], vb, dd, s));
    }
    if (m > 0) {
        CU(cudaMemcpyAsync(vec(9), A->wlast, vb, dd, s));
        CU(cudaMemcpy2DAsync(vec(10), L.stride, c->V, vb, vb, m, dd, s));
    }
    // a pageable source: the call returns once the header has been staged
    const TapeHeader hd{kTapeMagic, (unsigned long long)N, M, m, h};
    CU(cudaMemcpyAsync(tape, &hd, sizeof hd, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(y, A->y1, vb, dd, s));
    c->last = rok_step_info{};
    c->last.residual_evals = 1 + M + 3;
    c->last.jvps = M;
    CU(cudaGetLastError());
    return ROK_OK;
}

rok_status rok_step_vjp_tape(rok_ctx *c, const void *tape, const double *ybar_in, double *ybar_out, double *mubar)
{
    if (!c || !tape || !ybar_in || !ybar_out || (uintptr_t)tape % kTapeAlign) return ROK_ERR_INVALID_ARG;
    rok_status r = step_reverse_supported(c);
    if (r != ROK_OK) return r;
    if ((r = ensure_work(c, true)) != ROK_OK) return r;
    AdjWork *A = c->adj;
    const size_t N = c->N, vb = N * sizeof(double);
    cudaStream_t s = c->stream;
    TapeHeader hd;
    CU(cudaMemcpyAsync(&hd, tape, sizeof hd, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hd.magic != kTapeMagic || hd.n != (unsigned long long)N || hd.M < 0 || hd.M > c->mmax || hd.m < 0 ||
        hd.m > hd.M || !(hd.h > 0.0) || !isfinite(hd.h))
        return ROK_ERR_INVALID_ARG;
    const TapeLayout L = tape_layout(N, hd.M);
    if (overlaps(ybar_out, vb, tape, L.bytes)) return ROK_ERR_INVALID_ARG;
    const char *t = (const char *)tape;
    auto vec = [&](int k) { return t + L.vec + (size_t)k * L.stride; };
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    CU(cudaMemcpyAsync(c->st, t + L.st, sizeof(StepState), dd, s));
    for (int i = 0; i < 4; ++i) {
        CU(cudaMemcpyAsync(c->F[i], vec(1 + i), vb, dd, s));
        CU(cudaMemcpyAsync(c->K[i], vec(5 + i), vb, dd, s));
    }
    if (hd.m > 0) {
        CU(cudaMemcpyAsync(A->wlast, vec(9), vb, dd, s));
        CU(cudaMemcpy2DAsync(c->V, vb, vec(10), L.stride, vb, hd.m, dd, s));
    }
    return step_reverse(c, (const double *)vec(0), hd.h, hd.m, ybar_in, ybar_out, mubar);
}

}  // extern "C"
