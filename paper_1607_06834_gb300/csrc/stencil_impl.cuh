// Finite-volume residual stencil of the compressible Euler / Navier-Stokes
// equations (Sec. 3.2, Eq. Nav_Stokes; scheme of Sec. 4.2: unlimited MUSCL,
// Roe flux, central viscous flux), one CTA per TX x TY tile of cells.
//
// This file is compiled twice, in stencil_fast.cu (FMA contraction allowed)
// and stencil_strict.cu (--fmad=false), each time inside its own namespace
// ROK_NS.  Every expression is written out in one fixed order; the strict
// build therefore produces the IEEE result of that order, which is the order
// of a plain CPU evaluation of the same formulas.
//
// With ROK_STENCIL_DEVICE_ONLY defined, only the device functions (MUSCL,
// Roe flux, primitives) are compiled, for reuse by the adjoint kernels.
//
// Tile pipeline (the kernel is FP64-ALU bound on GB300, so the design
// minimises FP64 work: primitives once per loaded cell, each face once):
//   1. load the (TX+4) x (TY+4) cells of the tile and its 2-cell halo, form the
//      state base + sum c_t add_t (stage states and y + eps v are built here),
//      convert to primitives (rho, u, v, p, T[, mu]) in shared memory;
//   2. every face of the tile: MUSCL left/right states, Roe flux, viscous flux,
//      stored in shared memory;
//   3. every cell: balance of its four faces, epilogue (JVP quotient, AXPY),
//      store, non-finite check.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dual.cuh"
#include "rok_internal.h"

namespace rok {
namespace ROK_NS {

// Tile shape: TXv x TYv cells per CTA, NTv threads (one or more cells per
// thread); the tile with its 2-cell halo is EW x EH cells.
template <int TXv, int TYv, int NTv = TXv * TYv>
struct Shape {
    static constexpr int TX = TXv, TY = TYv, NT = NTv, EW = TXv + 4, EH = TYv + 4;
    static_assert((TXv * TYv) % NTv == 0, "whole cells per thread");
};
using Shape32x8 = Shape<32, 8>;
using CurvShape = Shape<16, 16>;

// the curvilinear kernel's tiles (the uniform one: CartShape below)
constexpr int TX = CurvShape::TX;
constexpr int TY = CurvShape::TY;
constexpr int NT = CurvShape::NT;
constexpr int EW = CurvShape::EW;
constexpr int EH = CurvShape::EH;

template <class S>
__device__ __forceinline__ S harten(S lam, S delta)
{
    S a = fabs(lam);
    if (val(a) < val(delta)) a = (a * a + delta * delta) / (2.0 * delta);
    return a;
}

template <class S>
__device__ __forceinline__ void muscl(S m2, S m1, S p1, S p2, double c_lo,
                                      double c_hi, S &wl, S &wr)
{
    S dl = m1 - m2, dc = p1 - m1, dr = p2 - p1;
    wl = (m1 + c_lo * dl) + c_hi * dc;
    wr = (p1 - c_lo * dr) - c_hi * dc;
}

// the same reconstruction from the three cell differences dl = m1 - m2,
// dc = p1 - m1, dr = p2 - p1 (computed once per cell and shared by the faces)
template <class S>
__device__ __forceinline__ void muscl_d(S m1, S p1, S dl, S dc, S dr, double c_lo, double c_hi, S &wl, S &wr)
{
    wl = (m1 + c_lo * dl) + c_hi * dc;
    wr = (p1 - c_lo * dr) - c_hi * dc;
}

// Roe-averaged quantities common to every face orientation.  e = rho H = E + p;
// the sqrt(rho)-weighted averages use one reciprocal:
//   wl = rL sR / (sL sR (sL + sR)),  H~ = (eL sR + eR sL) / (sL sR (sL + sR)).
template <class S>
struct RoeAvg {
    S eL, eR, rt, ut, vt, Ht, kt, ct, inv_c2;
};

template <class S>
__device__ __forceinline__ RoeAvg<S> roe_avg(const S *L, const S *R, const StencilConsts &C)
{
    RoeAvg<S> a;
    S rL = L[0], uL = L[1], vL = L[2], pL = L[3];
    S rR = R[0], uR = R[1], vR = R[2], pR = R[3];
    a.eL = (pL * C.inv_gm1 + rL * (0.5 * (uL * uL + vL * vL))) + pL;
    a.eR = (pR * C.inv_gm1 + rR * (0.5 * (uR * uR + vR * vR))) + pR;
#ifdef ROK_STENCIL_FAST
    S sL = rL * rsqrt(rL), sR = rR * rsqrt(rR);
#else
    S sL = sqrt(rL), sR = sqrt(rR);
#endif
    a.rt = sL * sR;
    S den = 1.0 / (a.rt * (sL + sR));
    S wl = (rL * sR) * den, wr = (rR * sL) * den;
    a.ut = wl * uL + wr * uR;
    a.vt = wl * vL + wr * vR;
    a.Ht = (a.eL * sR + a.eR * sL) * den;
    a.kt = 0.5 * (a.ut * a.ut + a.vt * a.vt);
    S ct2 = C.gm1 * (a.Ht - a.kt);
#ifdef ROK_STENCIL_FAST
    // one reciprocal square root gives both c~ and 1/c~^2 (the FMA build only:
    // other rounding than sqrt and division, fewer FP64 instructions)
    S rc = rsqrt(ct2);
    a.ct = ct2 * rc;
    a.inv_c2 = rc * rc;
#else
    a.ct = sqrt(ct2);
    a.inv_c2 = 1.0 / ct2;
#endif
    return a;
}

// Roe flux through an x-face (unit normal (1, 0)).  Exact specialisation of the
// general-normal formula: only products by 1 or 0 and additions of a zero are
// removed, which leave the IEEE result of the general form unchanged (e.g.
// du - dqn nx = du - du = +0, so the shear term of D1 vanishes exactly).
template <class S>
__device__ __forceinline__ void roe_x(const S *L, const S *R, const StencilConsts &C, S *F)
{
    RoeAvg<S> a = roe_avg(L, R, C);
    S rL = L[0], uL = L[1], vL = L[2], pL = L[3];
    S rR = R[0], uR = R[1], vR = R[2], pR = R[3];
    S drho = rR - rL, dp = pR - pL, du = uR - uL, dv = vR - vL;
    S rcdq = a.rt * a.ct * du;
    S a1 = 0.5 * (dp - rcdq) * a.inv_c2;
    S a2 = drho - dp * a.inv_c2;
    S a3 = 0.5 * (dp + rcdq) * a.inv_c2;
    S delta = C.efix * (fabs(a.ut) + a.ct);
    S l1 = harten(a.ut - a.ct, delta);
    S l2 = fabs(a.ut);
    S l3 = harten(a.ut + a.ct, delta);
    S A1 = l1 * a1, A2 = l2 * a2, A3 = l3 * a3, As = l2 * a.rt;
    S sA = A1 + A3, dA = A3 - A1;
    S D0 = sA + A2;
    S D1 = a.ut * D0 + a.ct * dA;
    S D2 = a.vt * D0 + As * dv;
    S D3 = ((a.Ht * sA + a.kt * A2) + (a.ct * a.ut) * dA) + As * ((a.ut * du + a.vt * dv) - a.ut * du);
    S mL = rL * uL, mR = rR * uR;
    F[0] = 0.5 * ((mL + mR) - D0);
    F[1] = 0.5 * (((mL * uL + pL) + (mR * uR + pR)) - D1);
    F[2] = 0.5 * ((mL * vL + mR * vR) - D2);
    F[3] = 0.5 * ((uL * a.eL + uR * a.eR) - D3);
}

// Roe flux through a y-face (unit normal (0, 1)), exact specialisation as above.
template <class S>
__device__ __forceinline__ void roe_y(const S *L, const S *R, const StencilConsts &C, S *F)
{
    RoeAvg<S> a = roe_avg(L, R, C);
    S rL = L[0], uL = L[1], vL = L[2], pL = L[3];
    S rR = R[0], uR = R[1], vR = R[2], pR = R[3];
    S drho = rR - rL, dp = pR - pL, du = uR - uL, dv = vR - vL;
    S rcdq = a.rt * a.ct * dv;
    S a1 = 0.5 * (dp - rcdq) * a.inv_c2;
    S a2 = drho - dp * a.inv_c2;
    S a3 = 0.5 * (dp + rcdq) * a.inv_c2;
    S delta = C.efix * (fabs(a.vt) + a.ct);
    S l1 = harten(a.vt - a.ct, delta);
    S l2 = fabs(a.vt);
    S l3 = harten(a.vt + a.ct, delta);
    S A1 = l1 * a1, A2 = l2 * a2, A3 = l3 * a3, As = l2 * a.rt;
    S sA = A1 + A3, dA = A3 - A1;
    S D0 = sA + A2;
    S D1 = a.ut * D0 + As * du;
    S D2 = a.vt * D0 + a.ct * dA;
    S D3 = ((a.Ht * sA + a.kt * A2) + (a.ct * a.vt) * dA) + As * ((a.ut * du + a.vt * dv) - a.vt * dv);
    S mL = rL * vL, mR = rR * vR;
    F[0] = 0.5 * ((mL + mR) - D0);
    F[1] = 0.5 * ((mL * uL + mR * uR) - D1);
    F[2] = 0.5 * (((mL * vL + pL) + (mR * vR + pR)) - D2);
    F[3] = 0.5 * ((vL * a.eL + vR * a.eR) - D3);
}

// Roe flux for a general unit normal (nx, ny) (curvilinear grids).
template <class S>
__device__ __forceinline__ void roe_n(const S *L, const S *R, double nx, double ny,
                                      const StencilConsts &C, S *F)
{
    S rL = L[0], uL = L[1], vL = L[2], pL = L[3];
    S rR = R[0], uR = R[1], vR = R[2], pR = R[3];
    S qnL = uL * nx + vL * ny;
    S qnR = uR * nx + vR * ny;
    RoeAvg<S> a = roe_avg(L, R, C);
    S qnt = a.ut * nx + a.vt * ny;
    S drho = rR - rL, dp = pR - pL, du = uR - uL, dv = vR - vL, dqn = qnR - qnL;
    S rcdq = a.rt * a.ct * dqn;
    S a1 = 0.5 * (dp - rcdq) * a.inv_c2;
    S a2 = drho - dp * a.inv_c2;
    S a3 = 0.5 * (dp + rcdq) * a.inv_c2;
    S delta = C.efix * (fabs(qnt) + a.ct);
    S l1 = harten(qnt - a.ct, delta);
    S l2 = fabs(qnt);
    S l3 = harten(qnt + a.ct, delta);
    S A1 = l1 * a1, A2 = l2 * a2, A3 = l3 * a3, As = l2 * a.rt;
    S sA = A1 + A3, dA = A3 - A1;
    S D0 = sA + A2;
    S D1 = (a.ut * D0 + (a.ct * nx) * dA) + As * (du - dqn * nx);
    S D2 = (a.vt * D0 + (a.ct * ny) * dA) + As * (dv - dqn * ny);
    S D3 = ((a.Ht * sA + a.kt * A2) + (a.ct * qnt) * dA) + As * ((a.ut * du + a.vt * dv) - qnt * dqn);
    S mL = rL * qnL, mR = rR * qnR;
    S FL1 = mL * uL + pL * nx, FR1 = mR * uR + pR * nx;
    S FL2 = mL * vL + pL * ny, FR2 = mR * vR + pR * ny;
    F[0] = 0.5 * ((mL + mR) - D0);
    F[1] = 0.5 * ((FL1 + FR1) - D1);
    F[2] = 0.5 * ((FL2 + FR2) - D2);
    F[3] = 0.5 * ((qnL * a.eL + qnR * a.eR) - D3);
}

#ifdef ROK_STENCIL_FAST
// ---- FMA build of the uniform-grid faces: fewer FP64 instructions -------------
// GB300 issues FP64 at 2 lane-operations per SM per clock, against 64 for
// 32-bit integers, and the stencil is bound by FP64 issue.  The FMA build
// therefore evaluates the same formulas with fewer FP64 operations (other
// rounding, within a few ulp of the flux scale):
//   * faces hold G = 2F, so the factor 1/2 of the central and upwind parts is
//     dropped and the cell balance uses 0.5/dx, 0.5/dy;
//   * the viscous coefficients carry mu, the grid spacing and the factor 2
//     (face_coefs);
//   * rho H = p gamma/(gamma-1) + rho k; the Roe averages from one
//     reciprocal square root z = 1/sqrt(rho_L rho_R) and one reciprocal
//     (w_L = 1/(1 + rho_R z)), the averaged velocity as q_R - w_L (q_R - q_L);
//   * halving and the comparison of non-negative numbers on the integer pipe;
//   * reciprocals from the hardware estimate and one Newton step.

// x / 2 by lowering the exponent field by one.  Exact for every x whose half
// is a normal number; a result below the normal range flushes to a signed
// zero (as the flush-to-zero modes do), infinities and NaNs pass unchanged.
__device__ __forceinline__ double half(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    const bool keep = e == 0x7ffu;
    const bool normal = e - 2u < 0x7fdu;   // 2 <= e <= 0x7fe
    const int h = normal ? hi - 0x00100000 : (keep ? hi : (hi & (int)0x80000000));
    return __hiloint2double(h, normal || keep ? lo : 0);
}
__device__ __forceinline__ Dual half(Dual x) { return {half(x.v), half(x.d)}; }

// x / 4 in the same way (exponent field lowered by two)
__device__ __forceinline__ double quarter(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    const bool keep = e == 0x7ffu;
    const bool normal = e - 3u < 0x7fcu;   // 3 <= e <= 0x7fe
    const int h = normal ? hi - 0x00200000 : (keep ? hi : (hi & (int)0x80000000));
    return __hiloint2double(h, normal || keep ? lo : 0);
}

// 1/x: the hardware estimate r0 (rcp.approx.ftz.f64, relative error e0) and one
// third-order Newton step for f(r) = 1/r - x: with e = 1 - x r0,
// 1/x = r0 (1 + e + e^2 + ...), so r0 + r0 (e + e^2) has relative error
// O(e0^3) below the final rounding (Householder's method of order 2).
__device__ __forceinline__ double rcp(double x)
{
    double r0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(x));
    const double e = fma(-x, r0, 1.0);
    return fma(r0, fma(e, e, e), r0);
}
__device__ __forceinline__ Dual rcp(Dual x)
{
    const double r = rcp(x.v);
    return {r, -(x.d * r) * r};
}


// a < b for non-negative (or +0) binary64 values: the bit patterns order alike
__device__ __forceinline__ bool less_nonneg(double a, double b)
{
    return __double_as_longlong(a) < __double_as_longlong(b);
}

// |x| by clearing the sign bit (the result feeds an integer comparison)
__device__ __forceinline__ double abs_bits(double x) { return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x)); }
__device__ __forceinline__ Dual abs_bits(Dual x) { return __double2hiint(x.v) < 0 ? -x : x; }

template <class S>
__device__ __forceinline__ S harten2(S lam, S delta)
{
    S a = abs_bits(lam);
    if (less_nonneg(val(a), val(delta))) a = (a * a + delta * delta) / (2.0 * delta);
    return a;
}

// The sum and difference of the two acoustic wave terms of the Roe
// dissipation, sA = l1 a1 + l3 a3 and dA = l3 a3 - l1 a1, with
// a1,3 = (dp -+ rho~ c~ dn) / (2 c~^2) and l1,3 = |u~ -+ c~| after Harten's
// fix (delta = efix (|u~| + c~)).  Where the face is subsonic and the fix idle
// (c~ - |u~| >= delta, i.e. c~ efix_k >= |u~|), l1,3 = c~ -+ u~, and with
// c~ / c~^2 = 1 / c~ the two reduce to sA = (dp + u~ rho~ dn) / c~ and
// dA = rho~ dn + u~ dp / c~^2 (7 FP64 instructions instead of 15).  The
// choice is made face by face (a warp whose faces differ runs both forms), so
// a face's arithmetic does not depend on the faces sharing its warp; rc = 1/c~.
template <class S>
__device__ __forceinline__ void acoustic_sums(S un, S ct, S rc, S inv_c2, S rt, S dn, S dp, S l2,
                                              const StencilConsts &C, S &sA, S &dA)
{
    // both sides non-negative for efix <= 1 (a negative product, efix > 1,
    // orders below by its sign bit: the general form)
    if (!less_nonneg(val(ct * C.efix_k), val(l2))) {
        sA = rc * ((un * rt) * dn + dp);
        dA = (inv_c2 * un) * dp + rt * dn;
    } else {
        const S delta = C.efix * (l2 + ct);
        const S hc = half(inv_c2);
        const S rcdq = (rt * ct) * dn;
        const S a1 = (dp - rcdq) * hc, a3 = (dp + rcdq) * hc;
        const S l1 = harten2(un - ct, delta), l3 = harten2(un + ct, delta);
        const S A1 = l1 * a1, A3 = l3 * a3;
        sA = A1 + A3;
        dA = A3 - A1;
    }
}

// Doubled Roe flux G = 2F through a face of a uniform grid with unit normal
// e_DIR (DIR 0: x, 1: y): the same flux as roe_x / roe_y, component N the
// normal and T the tangential momentum.  With VX the doubled viscous flux
// (vn, vt, ve: normal momentum, tangential momentum, energy; visc2_terms) is
// subtracted too, vn and ve inside the dissipation sums where a product
// becomes a fused multiply-add (one FP64 instruction fewer each).
template <bool VX, class S>
__device__ __forceinline__ void roe2_nt(S rL, S nL, S tL, S pL, S rR, S nR, S tR, S pR, const StencilConsts &C,
                                        S &g0, S &gn, S &gt, S &g3, S vn, S vt, S ve)
{
    // Roe average from one reciprocal square root z = 1/sqrt(rho_L rho_R)
    // (sX = sqrt(rho_X)): rho~ = rho_L rho_R z = sL sR; a = rho_R z = sR / sL;
    // the left weight sL / (sL + sR) = 1 / (1 + a); and
    // H~ = (eL / sL + eR / sR) / (sL + sR) = wl z (eL a + eR)
    const S eL = pL * C.gg + rL * half(nL * nL + tL * tL);   // rho H = E + p
    const S eR = pR * C.gg + rR * half(nR * nR + tR * tR);
    const S prr = rL * rR;
    const S z = rsqrt(prr);
    const S rt = prr * z;
    const S a = rR * z;
    const S wl = rcp(a + 1.0);   // the right weight is 1 - wl
    const S drho = rR - rL, dp = pR - pL, dn = nR - nL, dt = tR - tL;
    const S nt = nR - wl * dn, tt = tR - wl * dt;
    const S Ht = (wl * z) * (eL * a + eR);
    const S kt = half(nt * nt + tt * tt);
    const S ct2 = C.gm1 * (Ht - kt);
    const S rc = rsqrt(ct2);
    const S ct = ct2 * rc, inv_c2 = rc * rc;
    // wave strengths and speeds (Harten's fix on the acoustic waves)
    const S a2 = drho - dp * inv_c2;
    const S l2 = fabs(nt);
    S sA, dA;
    acoustic_sums(nt, ct, rc, inv_c2, rt, dn, dp, l2, C, sA, dA);
    const S A2 = l2 * a2, As = l2 * rt;
    const S D0 = sA + A2;
    const S Asdt = As * dt;
    const S Dn = nt * D0 + (VX ? ct * dA + vn : ct * dA);
    const S Dt = VX ? tt * D0 + Asdt + vt : tt * D0 + Asdt;
    const S D3 = Ht * sA + (kt * A2 + ((ct * nt) * dA + (VX ? tt * Asdt + ve : tt * Asdt)));
    const S mL = rL * nL, mR = rR * nR;
    g0 = (mL + mR) - D0;
    gn = mL * nL + (mR * nR + ((pL + pR) - Dn));
    gt = mL * tL + (mR * tR - Dt);
    g3 = nL * eL + (nR * eR - D3);
}

template <int DIR, bool VX, class S>
__device__ __forceinline__ void roe2(const S *L, const S *R, const StencilConsts &C, S *G, S vn, S vt, S ve)
{
    constexpr int N = 1 + DIR, T = 2 - DIR;
    roe2_nt<VX>(L[0], L[N], L[T], L[3], R[0], R[N], R[T], R[3], C, G[0], G[N], G[T], G[3], vn, vt, ve);
}

// Doubled viscous flux terms of a uniform-grid face (coefficients of
// face_coefs), for roe2 to subtract: dnn, dtn, dTn differences across the
// face, dnt, dtt four-cell differences along it, sn, st the sums of the two
// cells' normal and tangential velocities, mus the sum of their viscosities
// (Sutherland's law only); vn, vt the momentum and ve the energy terms.
template <bool SUTH, class S>
__device__ __forceinline__ void visc2_terms(S dnn, S dtn, S dTn, S dnt, S dtt, S sn, S st, S mus, const double *vk,
                                            S &vn, S &vt, S &ve)
{
    S tnn = dnn * vk[0] + dtt * vk[1];
    S tnt = dnt * vk[2] + dtn * vk[3];
    S q = dTn * vk[4];
    if (SUTH) {
        tnn = tnn * mus;
        tnt = tnt * mus;
        q = q * mus;
    }
    vn = tnn;
    vt = tnt;
    ve = half(sn) * tnn + (half(st) * tnt + q);
}
// Doubled Roe flux G = 2F through a face with unit normal (nx, ny) (curvilinear
// grids): the flux of roe_n.
template <bool VX, class S>
__device__ __forceinline__ void roe_n2(const S *L, const S *R, double nx, double ny, const StencilConsts &C, S *G,
                                       S v1, S v2, S v3)
{
    const S rL = L[0], uL = L[1], vL = L[2], pL = L[3];
    const S rR = R[0], uR = R[1], vR = R[2], pR = R[3];
    const S qnL = uL * nx + vL * ny, qnR = uR * nx + vR * ny;
    const S eL = pL * C.gg + rL * half(uL * uL + vL * vL);
    const S eR = pR * C.gg + rR * half(uR * uR + vR * vR);
    // Roe average from one reciprocal square root, as in roe2
    const S prr = rL * rR;
    const S z = rsqrt(prr);
    const S rt = prr * z;
    const S a = rR * z;
    const S wl = rcp(a + 1.0);   // the right weight is 1 - wl
    const S drho = rR - rL, dp = pR - pL, du = uR - uL, dv = vR - vL, dqn = qnR - qnL;
    const S ut = uR - wl * du, vt = vR - wl * dv;
    const S Ht = (wl * z) * (eL * a + eR);
    const S kt = half(ut * ut + vt * vt);
    const S ct2 = C.gm1 * (Ht - kt);
    const S rc = rsqrt(ct2);
    const S ct = ct2 * rc, inv_c2 = rc * rc;
    const S qnt = ut * nx + vt * ny;
    const S a2 = drho - dp * inv_c2;
    const S l2 = fabs(qnt);
    S sA, dA;
    acoustic_sums(qnt, ct, rc, inv_c2, rt, dqn, dp, l2, C, sA, dA);
    const S A2 = l2 * a2, As = l2 * rt;
    const S D0 = sA + A2;
    const S cdA = ct * dA;
    // with VX the viscous terms v1, v2, v3 (visc_n2_terms) join the products by As
    const S sx = du - dqn * nx, sy = dv - dqn * ny, s3 = (ut * du + vt * dv) - qnt * dqn;
    const S D1 = ut * D0 + (cdA * nx + (VX ? As * sx + v1 : As * sx));
    const S D2 = vt * D0 + (cdA * ny + (VX ? As * sy + v2 : As * sy));
    const S D3 = Ht * sA + (kt * A2 + (qnt * cdA + (VX ? As * s3 + v3 : As * s3)));
    const S mL = rL * qnL, mR = rR * qnR, pLR = pL + pR;
    G[0] = (mL + mR) - D0;
    G[1] = mL * uL + (mR * uR + (pLR * nx - D1));
    G[2] = mL * vL + (mR * vR + (pLR * ny - D2));
    G[3] = qnL * eL + (qnR * eR - D3);
}

// Doubled viscous flux terms of a curvilinear face, for roe_n2 to subtract
// (v1, v2 the momentum and v3 the energy terms).  The gradients
// come from the difference across the face (dC*) and four times the difference
// of the two vertex averages along it (dV*: the middle pair of cells cancels),
// with the metric terms c0, c1q = c1 / 4, c2, c3q = c3 / 4; su, sv the sums of
// the two cells' velocities, mus of their viscosities (Sutherland's law only).
template <bool SUTH, class S>
__device__ __forceinline__ void visc_n2_terms(double nx, double ny, double c0, double c1q, double c2, double c3q,
                                              S dCu, S dCv, S dCT, S dVu, S dVv, S dVT, S su, S sv, S mus,
                                              const StencilConsts &C, S &v1, S &v2, S &v3)
{
    const S ux = dCu * c0 + dVu * c1q, uy = dCu * c2 + dVu * c3q;
    const S vx = dCv * c0 + dVv * c1q, vy = dCv * c2 + dVv * c3q;
    const S Tx = dCT * c0 + dVT * c1q, Ty = dCT * c2 + dVT * c3q;
    S txx = ux * C.vc[0] + vy * C.vc[1];
    S tyy = vy * C.vc[0] + ux * C.vc[1];
    S txy = (uy + vx) * C.vc[2];
    S q = (Tx * nx + Ty * ny) * C.vc[3];
    if (SUTH) {
        txx = txx * mus;
        tyy = tyy * mus;
        txy = txy * mus;
        q = q * mus;
    }
    const S tnx = txx * nx + txy * ny, tny = txy * nx + tyy * ny;
    v1 = tnx;
    v2 = tny;
    v3 = half(su) * tnx + (half(sv) * tny + q);
}
#endif  // ROK_STENCIL_FAST

// shared-memory tile of primitive variables (halo included)
template <class S, class SH = CurvShape>
struct Tile {
    S r[SH::EH][SH::EW], u[SH::EH][SH::EW], v[SH::EH][SH::EW], p[SH::EH][SH::EW], T[SH::EH][SH::EW],
        mu[SH::EH][SH::EW];
};
// differences of the four reconstructed primitives between a cell and its
// lower neighbour along x (dx, the tile's rows 2 .. TY+1 only: dx[k][ly - 2][lx])
// and y (dy, the tile's columns 2 .. TX+1 only: dy[k][ly][lx - 2]) -- the ones
// the faces read
template <class S, class SH = CurvShape>
struct Diffs {
    S dx[4][SH::TY][SH::EW], dy[4][SH::EH][SH::TX];
};

// FMA build, viscous faces: sums over the two cells beside a face of its
// tangential neighbour rows / columns, shared by the faces above and below:
// px[q][ly - 1][fx] = w[ly][fx + 1] + w[ly][fx + 2] (rows 1 .. TY+2),
// qy[q][lx - 1][fy] = w[fy + 1][lx] + w[fy + 2][lx] (columns 1 .. TX+2), w = u, v
template <class S, class SH = CurvShape>
struct PairSums {
    S px[2][SH::TY + 2][SH::TX + 1], qy[2][SH::TX + 2][SH::TY + 1];
};

// shared-memory bytes of the pair sums (FMA build, viscous kernels only)
template <bool VISC, class S, class SH>
constexpr size_t pair_sums_bytes()
{
#ifdef ROK_STENCIL_FAST
    return VISC ? sizeof(PairSums<S, SH>) : 0;
#else
    return 0;
#endif
}

template <class S, class SH = CurvShape>
struct Faces {
    S fx[4][SH::TY][SH::TX + 1];
    S fy[4][SH::TY + 1][SH::TX];
};

template <class S, class SH>
__device__ __forceinline__ S pick(const Tile<S, SH> &t, int k, int y, int x)
{
    return k == 0 ? t.r[y][x] : (k == 1 ? t.u[y][x] : (k == 2 ? t.v[y][x] : t.p[y][x]));
}

template <bool SUTH, class S, class SH>
__device__ __forceinline__ void store_prim(Tile<S, SH> &t, int ly, int lx, S rho, S mx, S my,
                                           S E, bool mirror, const StencilConsts &C)
{
#ifdef ROK_STENCIL_FAST
    S rinv = rcp(rho);
    S u = mx * rinv;
    S v = my * rinv;
    S p = C.gm1 * E - C.gm1h * (mx * u + my * v);
#else
    S rinv = 1.0 / rho;
    S u = mx * rinv;
    S v = my * rinv;
    S p = C.gm1 * (E - 0.5 * (mx * u + my * v));
#endif
    S T = p * rinv;
    t.r[ly][lx] = rho;
    t.u[ly][lx] = mirror ? -u : u;
    t.v[ly][lx] = mirror ? -v : v;
    t.p[ly][lx] = p;
    t.T[ly][lx] = T;
    if (SUTH) {
        S tt = T * C.inv_tref;
        t.mu[ly][lx] = C.mu * (tt * sqrt(tt)) * ((1.0 + C.suth_s) / (tt + C.suth_s));
    }
}

// state entry e: base + sum_t c_t add_t (+ cf addf); for dual numbers the
// tangent is the direction of the exact JVP (dir or its binary32 form dirf)
__device__ __forceinline__ double load_value(const StencilIO &io, const double (&cf)[kMaxAdd], double cff, size_t e)
{
    double q = io.base[e];
    for (int t = 0; t < io.nadd; ++t) q = q + cf[t] * io.add[t][e];
    if (io.addf) q = q + cff * (double)io.addf[e];
    return q;
}

template <class S>
__device__ __forceinline__ S load_state(const StencilIO &io, const double (&cf)[kMaxAdd], double cff, size_t e);

template <>
__device__ __forceinline__ double load_state<double>(const StencilIO &io, const double (&cf)[kMaxAdd], double cff,
                                                     size_t e)
{
    return load_value(io, cf, cff, e);
}

template <>
__device__ __forceinline__ Dual load_state<Dual>(const StencilIO &io, const double (&cf)[kMaxAdd], double cff, size_t e)
{
    return {load_value(io, cf, cff, e), io.dir ? io.dir[e] : (double)io.dirf[e]};
}

template <class S>
__device__ __forceinline__ S lift(double x);
template <>
__device__ __forceinline__ double lift<double>(double x) { return x; }
template <>
__device__ __forceinline__ Dual lift<Dual>(double x) { return {x, 0.0}; }

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// a per-instance scalar `sb` bytes after the pointer (batches; 0 otherwise)
template <class T>
__device__ __forceinline__ T *at_bytes(T *p, size_t sb)
{
    return reinterpret_cast<T *>(reinterpret_cast<typename std::conditional<std::is_const<T>::value, const char,
                                                                             char>::type *>(p) + sb);
}

// ---- stage 3: balance + epilogue ---------------------------------------------
// the launch output: t = (sub ? r - sub : r) * s1, out = add_out ? add_out + s2 t : t,
// r the residual value (or the JVP tangent)
// the part after the scaling by s1: out = add_out ? add_out + s2 t : t
__device__ __forceinline__ void epilogue_finish(const StencilIO &io, double s2, size_t e, double t, size_t sb = 0)
{
    double o = io.add_out ? io.add_out[e] + s2 * t : t;
    io.out[e] = o;
    if ((__double2hiint(o) & 0x7ff00000) == 0x7ff00000)   // infinity or NaN
        atomicOr(at_bytes(io.status, sb), kStatusNonfinite);
}

__device__ __forceinline__ void epilogue_store(const StencilIO &io, double s1, double s2, size_t e, double r,
                                               size_t sb = 0)
{
    double t = io.sub ? (r - io.sub[e]) : r;
    epilogue_finish(io, s2, e, t * s1, sb);
}

__device__ __forceinline__ void coefs(const StencilIO &io, double (&cf)[kMaxAdd], double &cff, double &s1, double &s2,
                                      size_t sb = 0)
{
#pragma unroll
    for (int t = 0; t < kMaxAdd; ++t) cf[t] = io.coef_dev[t] ? io.coef[t] * *at_bytes(io.coef_dev[t], sb) : io.coef[t];
    cff = io.coef_f_dev ? io.coef_f * *at_bytes(io.coef_f_dev, sb) : io.coef_f;
    s1 = io.s1_dev ? io.s1 * *at_bytes(io.s1_dev, sb) : io.s1;
    s2 = io.s2_dev ? io.s2 * *at_bytes(io.s2_dev, sb) : io.s2;
}

#ifndef ROK_STENCIL_DEVICE_ONLY
// ============================ uniform periodic grid ============================
// One TX x TY tile with lower-left cell (i0, j0) of an nx x ny periodic grid.
// Batches pass the instance's first entry `off` in the flat vectors and the
// byte offset `sb` of its per-instance scalars (eps, 1/eps, status, flag).
template <bool VISC, bool SUTH, class S, class SH>
__device__ __forceinline__ void cart_tile(const StencilConsts &C, const StencilIO &io, int i0, int j0,
                                          unsigned char *smem_raw, size_t off = 0, size_t sb = 0)
{
    constexpr int TX = SH::TX, TY = SH::TY, NT = SH::NT, EW = SH::EW, EH = SH::EH;
    if (io.active && *at_bytes(io.active, sb) == 0) return;
    Tile<S, SH> &tl = *reinterpret_cast<Tile<S, SH> *>(smem_raw);
    Faces<S, SH> &fc = *reinterpret_cast<Faces<S, SH> *>(smem_raw + sizeof(Tile<S, SH>));
    Diffs<S, SH> &df = *reinterpret_cast<Diffs<S, SH> *>(smem_raw + sizeof(Tile<S, SH>) + sizeof(Faces<S, SH>));
#ifdef ROK_STENCIL_FAST
    PairSums<S, SH> &ps = *reinterpret_cast<PairSums<S, SH> *>(smem_raw + sizeof(Tile<S, SH>) +
                                                               sizeof(Faces<S, SH>) + sizeof(Diffs<S, SH>));
#endif

    const int nx = C.nx, ny = C.ny;
    const size_t nc = (size_t)nx * ny;
    const int tid = threadIdx.x;
    double cf[kMaxAdd], cff, s1, s2;
    coefs(io, cf, cff, s1, s2, sb);
    for (int idx = tid; idx < EW * EH; idx += NT) {
        int lx = idx % EW, ly = idx / EW;
        int gi = wrapi(i0 + lx - 2, nx), gj = wrapi(j0 + ly - 2, ny);
        size_t c = off + (size_t)gj * nx + gi;
        S rho = load_state<S>(io, cf, cff, c);
        S mx = load_state<S>(io, cf, cff, nc + c);
        S my = load_state<S>(io, cf, cff, 2 * nc + c);
        S E = load_state<S>(io, cf, cff, 3 * nc + c);
        store_prim<SUTH, S, SH>(tl, ly, lx, rho, mx, my, E, false, C);
    }
    __syncthreads();
    // cell differences the faces read: along x in the tile's rows (lx >= 1),
    // along y in the tile's columns (ly >= 1)
    constexpr int NDX = (EW - 1) * TY, NDY = TX * (EH - 1);
#ifdef ROK_STENCIL_FAST
    constexpr int NPX = VISC ? 2 * (TY + 2) * (TX + 1) : 0, NQY = VISC ? 2 * (TX + 2) * (TY + 1) : 0;
#else
    constexpr int NPX = 0, NQY = 0;
#endif
    for (int idx = tid; idx < NDX + NDY + NPX + NQY; idx += NT) {
        if (idx < NDX) {
            const int ly = 2 + idx / (EW - 1), lx = 1 + idx % (EW - 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) df.dx[k][ly - 2][lx] = pick(tl, k, ly, lx) - pick(tl, k, ly, lx - 1);
        } else if (idx < NDX + NDY) {
            const int j = idx - NDX;
            const int ly = 1 + j / TX, lx = 2 + j % TX;
#pragma unroll
            for (int k = 0; k < 4; ++k) df.dy[k][ly][lx - 2] = pick(tl, k, ly, lx) - pick(tl, k, ly - 1, lx);
        }
#ifdef ROK_STENCIL_FAST
        else if (idx < NDX + NDY + NPX) {
            const int j = idx - NDX - NDY, q = j / ((TY + 2) * (TX + 1)), r = j % ((TY + 2) * (TX + 1));
            const int row = r / (TX + 1), fx = r % (TX + 1);
            ps.px[q][row][fx] = pick(tl, 1 + q, row + 1, fx + 1) + pick(tl, 1 + q, row + 1, fx + 2);
        } else {
            const int j = idx - NDX - NDY - NPX, q = j / ((TX + 2) * (TY + 1)), r = j % ((TX + 2) * (TY + 1));
            const int col = r / (TY + 1), fy = r % (TY + 1);
            ps.qy[q][col][fy] = pick(tl, 1 + q, fy + 1, col + 1) + pick(tl, 1 + q, fy + 2, col + 1);
        }
#endif
    }
    __syncthreads();

#ifdef ROK_STENCIL_FAST
    // One face per thread, x- and y-faces in one sequence of full warp batches
    // ((TX+1) TY + TX (TY+1) faces: 17 x 32 for 16 x 16 tiles, where batches of
    // one orientation each need 18, two of them half full: an FP64 warp
    // instruction costs the same with 16 lanes as with 32).  The orientation
    // is a per-lane value: it selects the cells, the shared-memory rows of the
    // differences and pair sums, the normal and tangential velocity and the
    // output array; the arithmetic is the same for both.
    {
        constexpr int NFX_ = (TX + 1) * TY, NF = NFX_ + TX * (TY + 1);
        auto face = [&](int f) {
            const bool yd = f >= NFX_;
            const int g = yd ? f - NFX_ : f;
            const int fx = yd ? g % TX : g % (TX + 1), fy = yd ? g / TX : g / (TX + 1);
            // the cells on the minus and plus side (tile coordinates)
            const int ym = yd ? fy + 1 : fy + 2, xm = yd ? fx + 2 : fx + 1;
            const int yp = fy + 2, xp = fx + 2;
            // differences along the face normal: dl, dc, dr at d[0], d[ds], d[2 ds]
            const int ds = yd ? TX : 1;
            S WL[4], WR[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const S *d = yd ? &df.dy[k][ym][xm - 2] : &df.dx[k][ym - 2][xm];
                muscl_d(pick(tl, k, ym, xm), pick(tl, k, yp, xp), d[0], d[ds], d[2 * ds], C.c_lo, C.c_hi, WL[k],
                        WR[k]);
            }
            S vn = lift<S>(0.0), vt = lift<S>(0.0), ve = lift<S>(0.0);
            if (VISC) {
                // normal / tangential velocity: u / v on x-faces, v / u on y-faces
                const S *dn = yd ? &df.dy[2][ym][xm - 2] : &df.dx[1][ym - 2][xm];
                const S *dt = yd ? &df.dy[1][ym][xm - 2] : &df.dx[2][ym - 2][xm];
                const int ps_stride = yd ? TY + 1 : TX + 1;
                const S *pn = yd ? &ps.qy[1][xm][fy] : &ps.px[0][ym][fx];
                const S *pt = yd ? &ps.qy[0][xm][fy] : &ps.px[1][ym][fx];
                visc2_terms<SUTH>(dn[ds], dt[ds], tl.T[yp][xp] - tl.T[ym][xm], pn[0] - pn[-2 * ps_stride],
                                  pt[0] - pt[-2 * ps_stride], pn[-ps_stride], pt[-ps_stride],
                                  SUTH ? tl.mu[ym][xm] + tl.mu[yp][xp] : lift<S>(0.0), C.vk[yd ? 1 : 0], vn, vt,
                                  ve);
            }
            S g0, gn, gt, g3;
            roe2_nt<VISC>(WL[0], yd ? WL[2] : WL[1], yd ? WL[1] : WL[2], WL[3], WR[0], yd ? WR[2] : WR[1],
                          yd ? WR[1] : WR[2], WR[3], C, g0, gn, gt, g3, vn, vt, ve);
            S *out = yd ? &fc.fy[0][fy][fx] : &fc.fx[0][fy][fx];
            const int ks = yd ? (TY + 1) * TX : TY * (TX + 1);
            out[0] = g0;
            out[ks] = yd ? gt : gn;
            out[2 * ks] = yd ? gn : gt;
            out[3 * ks] = g3;
        };
        for (int bt = tid >> 5; bt < (NF + 31) / 32; bt += NT / 32) {
            const int f = bt * 32 + (tid & 31);
            if (f < NF) face(f);
        }
    }
#else
    // one face per thread, in warp-sized batches with the x-face batches first:
    // warp w takes batches w, w + NT/32, ...  Every batch has one orientation
    // (a warp-uniform branch), and the partial x batch and the last y batch
    // fall to different warps.
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    constexpr int BX = (NFX + 31) / 32, BY = (NFY + 31) / 32;
    auto xface = [&](int f) {
        int fx = f % (TX + 1), fy = f / (TX + 1);
        int y = fy + 2, xl = fx + 1, xr = fx + 2;
        S WL[4], WR[4], F[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            muscl_d(pick(tl, k, y, xl), pick(tl, k, y, xr), df.dx[k][y - 2][xl], df.dx[k][y - 2][xr], df.dx[k][y - 2][xr + 1],
                    C.c_lo, C.c_hi, WL[k], WR[k]);
#ifdef ROK_STENCIL_FAST
        S vn = lift<S>(0.0), vt = lift<S>(0.0), ve = lift<S>(0.0);
        if (VISC)
            visc2_terms<SUTH>(df.dx[1][y - 2][xr], df.dx[2][y - 2][xr], tl.T[y][xr] - tl.T[y][xl],
                              ps.px[0][y][fx] - ps.px[0][y - 2][fx], ps.px[1][y][fx] - ps.px[1][y - 2][fx],
                              ps.px[0][y - 1][fx], ps.px[1][y - 1][fx],
                              SUTH ? tl.mu[y][xl] + tl.mu[y][xr] : lift<S>(0.0), C.vk[0], vn, vt, ve);
        roe2<0, VISC>(WL, WR, C, F, vn, vt, ve);
#else
        roe_x(WL, WR, C, F);
        if (VISC) {
            S ux = (tl.u[y][xr] - tl.u[y][xl]) * C.rdx;
            S uy = ((tl.u[y + 1][xl] + tl.u[y + 1][xr]) - (tl.u[y - 1][xl] + tl.u[y - 1][xr])) * C.q_rdy;
            S vx = (tl.v[y][xr] - tl.v[y][xl]) * C.rdx;
            S vy = ((tl.v[y + 1][xl] + tl.v[y + 1][xr]) - (tl.v[y - 1][xl] + tl.v[y - 1][xr])) * C.q_rdy;
            S Tx = (tl.T[y][xr] - tl.T[y][xl]) * C.rdx;
            S mu_f = SUTH ? 0.5 * (tl.mu[y][xl] + tl.mu[y][xr]) : lift<S>(C.mu);
            S u_f = 0.5 * (tl.u[y][xl] + tl.u[y][xr]);
            S v_f = 0.5 * (tl.v[y][xl] + tl.v[y][xr]);
            S div = ux + vy;
            S txx = mu_f * (2.0 * ux - C.c23 * div);
            S txy = mu_f * (uy + vx);
            S kf = mu_f * C.kfac;
            F[1] = F[1] - txx;
            F[2] = F[2] - txy;
            F[3] = F[3] - ((u_f * txx + v_f * txy) + kf * Tx);
        }
#endif
#pragma unroll
        for (int k = 0; k < 4; ++k) fc.fx[k][fy][fx] = F[k];
    };
    auto yface = [&](int f) {
        int fx = f % TX, fy = f / TX;
        int x = fx + 2, yb = fy + 1, yt = fy + 2;
        S WL[4], WR[4], F[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            muscl_d(pick(tl, k, yb, x), pick(tl, k, yt, x), df.dy[k][yb][x - 2], df.dy[k][yt][x - 2], df.dy[k][yt + 1][x - 2],
                    C.c_lo, C.c_hi, WL[k], WR[k]);
#ifdef ROK_STENCIL_FAST
        S vn = lift<S>(0.0), vt = lift<S>(0.0), ve = lift<S>(0.0);
        if (VISC)
            visc2_terms<SUTH>(df.dy[2][yt][x - 2], df.dy[1][yt][x - 2], tl.T[yt][x] - tl.T[yb][x],
                              ps.qy[1][x][fy] - ps.qy[1][x - 2][fy], ps.qy[0][x][fy] - ps.qy[0][x - 2][fy],
                              ps.qy[1][x - 1][fy], ps.qy[0][x - 1][fy],
                              SUTH ? tl.mu[yb][x] + tl.mu[yt][x] : lift<S>(0.0), C.vk[1], vn, vt, ve);
        roe2<1, VISC>(WL, WR, C, F, vn, vt, ve);
#else
        roe_y(WL, WR, C, F);
        if (VISC) {
            S uy = (tl.u[yt][x] - tl.u[yb][x]) * C.rdy;
            S ux = ((tl.u[yb][x + 1] + tl.u[yt][x + 1]) - (tl.u[yb][x - 1] + tl.u[yt][x - 1])) * C.q_rdx;
            S vy = (tl.v[yt][x] - tl.v[yb][x]) * C.rdy;
            S vx = ((tl.v[yb][x + 1] + tl.v[yt][x + 1]) - (tl.v[yb][x - 1] + tl.v[yt][x - 1])) * C.q_rdx;
            S Ty = (tl.T[yt][x] - tl.T[yb][x]) * C.rdy;
            S mu_f = SUTH ? 0.5 * (tl.mu[yb][x] + tl.mu[yt][x]) : lift<S>(C.mu);
            S u_f = 0.5 * (tl.u[yb][x] + tl.u[yt][x]);
            S v_f = 0.5 * (tl.v[yb][x] + tl.v[yt][x]);
            S div = ux + vy;
            S tyy = mu_f * (2.0 * vy - C.c23 * div);
            S txy = mu_f * (uy + vx);
            S kf = mu_f * C.kfac;
            F[1] = F[1] - txy;
            F[2] = F[2] - tyy;
            F[3] = F[3] - ((u_f * txy + v_f * tyy) + kf * Ty);
        }
#endif
#pragma unroll
        for (int k = 0; k < 4; ++k) fc.fy[k][fy][fx] = F[k];
    };
    for (int bt = tid >> 5; bt < BX + BY; bt += NT / 32) {
        const int lane = tid & 31;
        if (bt < BX) {
            const int f = bt * 32 + lane;
            if (f < NFX) xface(f);
        } else {
            const int f = (bt - BX) * 32 + lane;
            if (f < NFY) yface(f);
        }
    }
#endif
    __syncthreads();

#ifdef ROK_STENCIL_FAST
    const double bx = C.hrdx, by = C.hrdy;   // the faces hold 2F
#else
    const double bx = C.rdx, by = C.rdy;
#endif
#pragma unroll
    for (int cell = tid; cell < TX * TY; cell += NT) {
        const int tx = cell % TX, ty = cell / TX;
        const int gi = i0 + tx, gj = j0 + ty;
        if (gi < nx && gj < ny) {
            size_t c = off + (size_t)gj * nx + gi;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                S dX = fc.fx[k][ty][tx + 1] - fc.fx[k][ty][tx];
                S dY = fc.fy[k][ty + 1][tx] - fc.fy[k][ty][tx];
#ifdef ROK_STENCIL_FAST
                if constexpr (std::is_same<S, double>::value) {
                    // r - sub = -(dX bx + (dY by + sub)): two FMAs
                    const size_t e = k * nc + c;
                    const double t = io.sub ? -(dX * bx + (dY * by + io.sub[e])) : -(dX * bx + dY * by);
                    epilogue_finish(io, s2, e, t * s1, sb);
                    continue;
                }
#endif
                S r = -(dX * bx + dY * by);
                epilogue_store(io, s1, s2, k * nc + c, result(r), sb);
            }
        }
    }
}

// tile shape of the single-grid uniform kernel: 16 x 16 (fewer halo faces and
// cells per tile than 32 x 8; 1 % faster at 512^2 and 1024^2)
using CartShape = Shape<16, 16>;

template <bool VISC, bool SUTH, class S, int MINB>
__global__ void __launch_bounds__(CartShape::NT, MINB) cart_kernel(const StencilConsts C, const StencilIO io)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cart_tile<VISC, SUTH, S, CartShape>(C, io, blockIdx.x * CartShape::TX, blockIdx.y * CartShape::TY, smem_raw);
}

// Many independent uniform periodic grids of one physics group in one launch:
// CTA b computes tile b - tile_first[k] of instance k = tile_inst[b].  The
// instances share the gas model and scheme constants (C); grid size, spacing
// and viscosity are per instance.  Vectors are flat: instance k's entries start
// at element inst[k].off; the per-instance scalars (eps, 1/eps, status,
// active flag) sit stride_bytes apart, starting at the pointers in io.
template <bool VISC, bool SUTH, class SH, int MINB>
__global__ void __launch_bounds__(SH::NT, MINB) cart_batch_kernel(const StencilConsts C, const StencilIO io,
                                                                   const BatchTiles bt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int k = bt.tile_inst[b];
    const BatchInst I = bt.inst[k];
    StencilConsts Ck = C;
    Ck.nx = I.nx;
    Ck.ny = I.ny;
    Ck.rdx = I.rdx;
    Ck.rdy = I.rdy;
    Ck.q_rdx = I.q_rdx;
    Ck.q_rdy = I.q_rdy;
    Ck.mu = I.mu;
    Ck.hrdx = I.hrdx;
    Ck.hrdy = I.hrdy;
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int q = 0; q < 5; ++q) Ck.vk[d][q] = I.vk[d][q];
    const int t = b - bt.tile_first[k];
    const int ntx = (I.nx + SH::TX - 1) / SH::TX;
    cart_tile<VISC, SUTH, double, SH>(Ck, io, (t % ntx) * SH::TX, (t / ntx) * SH::TY, smem_raw, I.off,
                                      (size_t)k * bt.stride_bytes);
}

// ============================== curvilinear grid ===============================
// Ghost cells follow the boundary rules: j-ghosts of interior columns first,
// then i-ghosts of every row (ghost rows included); periodic wraps, a wall
// mirrors (rho, -u, -v, p), the far field is the free stream.
template <bool VISC, bool SUTH, class S, int MINB>
__global__ void __launch_bounds__(NT, MINB) curv_kernel(const StencilConsts C, const CurvGeom G, const StencilIO io)
{
    if (io.active && *io.active == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tile<S> &tl = *reinterpret_cast<Tile<S> *>(smem_raw);
    Faces<S> &fc = *reinterpret_cast<Faces<S> *>(smem_raw + sizeof(Tile<S>));
    Diffs<S> &df = *reinterpret_cast<Diffs<S> *>(smem_raw + sizeof(Tile<S>) + sizeof(Faces<S>));

    const int nx = C.nx, ny = C.ny;
    const size_t nc = (size_t)nx * ny;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tid = threadIdx.x;
    double cf[kMaxAdd], cff, s1, s2;
    coefs(io, cf, cff, s1, s2);

    for (int idx = tid; idx < EW * EH; idx += NT) {
        int lx = idx % EW, ly = idx / EW;
        int gi = i0 + lx - 2, gj = j0 + ly - 2;
        bool mirror = false, inf = false;
        if (gi < 0 || gi >= nx) {
            int b = gi < 0 ? C.bc[0] : C.bc[1];
            if (b == ROK_BC_PERIODIC) gi = wrapi(gi, nx);
            else if (b == ROK_BC_WALL) { gi = gi < 0 ? -gi - 1 : 2 * nx - 1 - gi; mirror = !mirror; }
            else inf = true;
        }
        if (!inf && (gj < 0 || gj >= ny)) {
            int b = gj < 0 ? C.bc[2] : C.bc[3];
            if (b == ROK_BC_PERIODIC) gj = wrapi(gj, ny);
            else if (b == ROK_BC_WALL) { gj = gj < 0 ? -gj - 1 : 2 * ny - 1 - gj; mirror = !mirror; }
            else inf = true;
        }
        // a tile cell past the last valid index of a partial tile may still be out
        // of range after the rules above; clamp it (its faces are never used)
        gi = min(max(gi, 0), nx - 1);
        gj = min(max(gj, 0), ny - 1);
        if (inf) {
            tl.r[ly][lx] = lift<S>(C.prim_inf[0]);
            tl.u[ly][lx] = lift<S>(mirror ? -C.prim_inf[1] : C.prim_inf[1]);
            tl.v[ly][lx] = lift<S>(mirror ? -C.prim_inf[2] : C.prim_inf[2]);
            tl.p[ly][lx] = lift<S>(C.prim_inf[3]);
            tl.T[ly][lx] = lift<S>(C.prim_inf[4]);
            if (SUTH) tl.mu[ly][lx] = lift<S>(C.prim_inf[5]);
        } else {
            size_t c = (size_t)gj * nx + gi;
            S rho = load_state<S>(io, cf, cff, c);
            S mx = load_state<S>(io, cf, cff, nc + c);
            S my = load_state<S>(io, cf, cff, 2 * nc + c);
            S E = load_state<S>(io, cf, cff, 3 * nc + c);
            store_prim<SUTH, S>(tl, ly, lx, rho, mx, my, E, mirror, C);
        }
    }
    __syncthreads();
    // the cell differences the faces' MUSCL reconstruction reads (as in cart_tile)
    constexpr int NDX = (EW - 1) * TY, NDY = TX * (EH - 1);
    for (int idx = tid; idx < NDX + NDY; idx += NT) {
        if (idx < NDX) {
            const int ly = 2 + idx / (EW - 1), lx = 1 + idx % (EW - 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) df.dx[k][ly - 2][lx] = pick(tl, k, ly, lx) - pick(tl, k, ly, lx - 1);
        } else {
            const int j = idx - NDX;
            const int ly = 1 + j / TX, lx = 2 + j % TX;
#pragma unroll
            for (int k = 0; k < 4; ++k) df.dy[k][ly][lx - 2] = pick(tl, k, ly, lx) - pick(tl, k, ly - 1, lx);
        }
    }
    __syncthreads();

#ifdef ROK_STENCIL_FAST
    // i- and j-faces in one sequence of full warp batches, the orientation a
    // per-lane value (as in cart_tile): it selects the cells, the difference
    // rows, the tangential neighbours (+1 row on i-faces, -1 column on j-faces,
    // the sign convention of the metric terms), the metric arrays and the output
    {
        constexpr int NFX_ = (TX + 1) * TY, NF = NFX_ + TX * (TY + 1);
        auto face = [&](int f) {
            const bool yd = f >= NFX_;
            const int g = yd ? f - NFX_ : f;
            const int fx = yd ? g % TX : g % (TX + 1), fy = yd ? g / TX : g / (TX + 1);
            const int gi = i0 + fx, gj = j0 + fy;
            if (yd ? (gi >= nx || gj > ny) : (gi > nx || gj >= ny)) return;
            const size_t fi = yd ? (size_t)gj * nx + gi : (size_t)gj * (nx + 1) + gi;
            const int ym = yd ? fy + 1 : fy + 2, xm = yd ? fx + 2 : fx + 1;
            const int yp = fy + 2, xp = fx + 2;
            const int ds = yd ? TX : 1;
            const int ty = yd ? 0 : 1, txo = yd ? -1 : 0;   // tangential step
            S WL[4], WR[4], F[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const S *d = yd ? &df.dy[k][ym][xm - 2] : &df.dx[k][ym - 2][xm];
                muscl_d(pick(tl, k, ym, xm), pick(tl, k, yp, xp), d[0], d[ds], d[2 * ds], C.c_lo, C.c_hi, WL[k],
                        WR[k]);
            }
            const double nxf = yd ? G.jn_x[fi] : G.in_x[fi], nyf = yd ? G.jn_y[fi] : G.in_y[fi];
            S v1 = lift<S>(0.0), v2 = lift<S>(0.0), v3 = lift<S>(0.0);
            if (VISC) {
                auto across = [&](const S (&w)[EH][EW]) { return w[yp][xp] - w[ym][xm]; };
                auto along = [&](const S (&w)[EH][EW]) {
                    return (w[ym + ty][xm + txo] + w[yp + ty][xp + txo]) - (w[ym - ty][xm - txo] + w[yp - ty][xp - txo]);
                };
                visc_n2_terms<SUTH>(nxf, nyf, yd ? G.jc0[fi] : G.ic0[fi], quarter(yd ? G.jc1[fi] : G.ic1[fi]),
                                    yd ? G.jc2[fi] : G.ic2[fi], quarter(yd ? G.jc3[fi] : G.ic3[fi]), across(tl.u),
                                    across(tl.v), across(tl.T), along(tl.u), along(tl.v), along(tl.T),
                                    tl.u[ym][xm] + tl.u[yp][xp], tl.v[ym][xm] + tl.v[yp][xp],
                                    SUTH ? tl.mu[ym][xm] + tl.mu[yp][xp] : lift<S>(0.0), C, v1, v2, v3);
            }
            roe_n2<VISC>(WL, WR, nxf, nyf, C, F, v1, v2, v3);
            const double len = half(yd ? G.jl[fi] : G.il[fi]);   // the face holds 2F
            S *out = yd ? &fc.fy[0][fy][fx] : &fc.fx[0][fy][fx];
            const int ks = yd ? (TY + 1) * TX : TY * (TX + 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) out[k * ks] = F[k] * len;
        };
        for (int bt = tid >> 5; bt < (NF + 31) / 32; bt += NT / 32) {
            const int f = bt * 32 + (tid & 31);
            if (f < NF) face(f);
        }
    }
#else
    // faces in warp-sized batches spread over the warps (as in cart_tile)
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    constexpr int BX = (NFX + 31) / 32, BY = (NFY + 31) / 32;
    auto xface = [&](int f) {
        int fx = f % (TX + 1), fy = f / (TX + 1);
        int gi = i0 + fx, gj = j0 + fy;
        if (gi > nx || gj >= ny) return;
        size_t fi = (size_t)gj * (nx + 1) + gi;
        int y = fy + 2, xl = fx + 1, xr = fx + 2;
        S WL[4], WR[4], F[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            muscl_d(pick(tl, k, y, xl), pick(tl, k, y, xr), df.dx[k][y - 2][xl], df.dx[k][y - 2][xr], df.dx[k][y - 2][xr + 1],
                    C.c_lo, C.c_hi, WL[k], WR[k]);
        double nxf = G.in_x[fi], nyf = G.in_y[fi];
#ifdef ROK_STENCIL_FAST
        S v1 = lift<S>(0.0), v2 = lift<S>(0.0), v3 = lift<S>(0.0);
        if (VISC)
            visc_n2_terms<SUTH>(nxf, nyf, G.ic0[fi], quarter(G.ic1[fi]), G.ic2[fi], quarter(G.ic3[fi]),
                          tl.u[y][xr] - tl.u[y][xl], tl.v[y][xr] - tl.v[y][xl], tl.T[y][xr] - tl.T[y][xl],
                          (tl.u[y + 1][xl] + tl.u[y + 1][xr]) - (tl.u[y - 1][xl] + tl.u[y - 1][xr]),
                          (tl.v[y + 1][xl] + tl.v[y + 1][xr]) - (tl.v[y - 1][xl] + tl.v[y - 1][xr]),
                          (tl.T[y + 1][xl] + tl.T[y + 1][xr]) - (tl.T[y - 1][xl] + tl.T[y - 1][xr]),
                          tl.u[y][xl] + tl.u[y][xr], tl.v[y][xl] + tl.v[y][xr],
                          SUTH ? tl.mu[y][xl] + tl.mu[y][xr] : lift<S>(0.0), C, v1, v2, v3);
        roe_n2<VISC>(WL, WR, nxf, nyf, C, F, v1, v2, v3);
        const double len = half(G.il[fi]);   // the face holds 2F
#else
        roe_n(WL, WR, nxf, nyf, C, F);
        if (VISC) {
            double c0 = G.ic0[fi], c1 = G.ic1[fi], c2 = G.ic2[fi], c3 = G.ic3[fi];
            S g[6];
            // vertex (i, j) = P1 from rows y-1, y; vertex (i, j+1) = P3 from rows y, y+1
            {
                S a = 0.25 * (((tl.u[y - 1][xl] + tl.u[y - 1][xr]) + tl.u[y][xl]) + tl.u[y][xr]);
                S b = 0.25 * (((tl.u[y][xl] + tl.u[y][xr]) + tl.u[y + 1][xl]) + tl.u[y + 1][xr]);
                S dC = tl.u[y][xr] - tl.u[y][xl], dV = b - a;
                g[0] = dC * c0 + dV * c1;
                g[1] = dC * c2 + dV * c3;
            }
            {
                S a = 0.25 * (((tl.v[y - 1][xl] + tl.v[y - 1][xr]) + tl.v[y][xl]) + tl.v[y][xr]);
                S b = 0.25 * (((tl.v[y][xl] + tl.v[y][xr]) + tl.v[y + 1][xl]) + tl.v[y + 1][xr]);
                S dC = tl.v[y][xr] - tl.v[y][xl], dV = b - a;
                g[2] = dC * c0 + dV * c1;
                g[3] = dC * c2 + dV * c3;
            }
            {
                S a = 0.25 * (((tl.T[y - 1][xl] + tl.T[y - 1][xr]) + tl.T[y][xl]) + tl.T[y][xr]);
                S b = 0.25 * (((tl.T[y][xl] + tl.T[y][xr]) + tl.T[y + 1][xl]) + tl.T[y + 1][xr]);
                S dC = tl.T[y][xr] - tl.T[y][xl], dV = b - a;
                g[4] = dC * c0 + dV * c1;
                g[5] = dC * c2 + dV * c3;
            }
            S mu_f = SUTH ? 0.5 * (tl.mu[y][xl] + tl.mu[y][xr]) : lift<S>(C.mu);
            S u_f = 0.5 * (tl.u[y][xl] + tl.u[y][xr]);
            S v_f = 0.5 * (tl.v[y][xl] + tl.v[y][xr]);
            S div = g[0] + g[3];
            S txx = mu_f * (2.0 * g[0] - C.c23 * div);
            S tyy = mu_f * (2.0 * g[3] - C.c23 * div);
            S txy = mu_f * (g[1] + g[2]);
            S tnx = txx * nxf + txy * nyf;
            S tny = txy * nxf + tyy * nyf;
            S kf = mu_f * C.kfac;
            S dTn = g[4] * nxf + g[5] * nyf;
            F[1] = F[1] - tnx;
            F[2] = F[2] - tny;
            F[3] = F[3] - ((u_f * tnx + v_f * tny) + kf * dTn);
        }
        const double len = G.il[fi];
#endif
#pragma unroll
        for (int k = 0; k < 4; ++k) fc.fx[k][fy][fx] = F[k] * len;
    };
    auto yface = [&](int f) {
        int fx = f % TX, fy = f / TX;
        int gi = i0 + fx, gj = j0 + fy;
        if (gi >= nx || gj > ny) return;
        size_t fi = (size_t)gj * nx + gi;
        int x = fx + 2, yb = fy + 1, yt = fy + 2;
        S WL[4], WR[4], F[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            muscl_d(pick(tl, k, yb, x), pick(tl, k, yt, x), df.dy[k][yb][x - 2], df.dy[k][yt][x - 2], df.dy[k][yt + 1][x - 2],
                    C.c_lo, C.c_hi, WL[k], WR[k]);
        double nxf = G.jn_x[fi], nyf = G.jn_y[fi];
#ifdef ROK_STENCIL_FAST
        S v1 = lift<S>(0.0), v2 = lift<S>(0.0), v3 = lift<S>(0.0);
        if (VISC)
            visc_n2_terms<SUTH>(nxf, nyf, G.jc0[fi], quarter(G.jc1[fi]), G.jc2[fi], quarter(G.jc3[fi]),
                          tl.u[yt][x] - tl.u[yb][x], tl.v[yt][x] - tl.v[yb][x], tl.T[yt][x] - tl.T[yb][x],
                          (tl.u[yb][x - 1] + tl.u[yt][x - 1]) - (tl.u[yb][x + 1] + tl.u[yt][x + 1]),
                          (tl.v[yb][x - 1] + tl.v[yt][x - 1]) - (tl.v[yb][x + 1] + tl.v[yt][x + 1]),
                          (tl.T[yb][x - 1] + tl.T[yt][x - 1]) - (tl.T[yb][x + 1] + tl.T[yt][x + 1]),
                          tl.u[yb][x] + tl.u[yt][x], tl.v[yb][x] + tl.v[yt][x],
                          SUTH ? tl.mu[yb][x] + tl.mu[yt][x] : lift<S>(0.0), C, v1, v2, v3);
        roe_n2<VISC>(WL, WR, nxf, nyf, C, F, v1, v2, v3);
        const double len = half(G.jl[fi]);   // the face holds 2F
#else
        roe_n(WL, WR, nxf, nyf, C, F);
        if (VISC) {
            double c0 = G.jc0[fi], c1 = G.jc1[fi], c2 = G.jc2[fi], c3 = G.jc3[fi];
            S g[6];
            // vertex (i+1, j) = P1 from columns x, x+1; vertex (i, j) = P3 from columns x-1, x
            {
                S a = 0.25 * (((tl.u[yb][x] + tl.u[yb][x + 1]) + tl.u[yt][x]) + tl.u[yt][x + 1]);
                S b = 0.25 * (((tl.u[yb][x - 1] + tl.u[yb][x]) + tl.u[yt][x - 1]) + tl.u[yt][x]);
                S dC = tl.u[yt][x] - tl.u[yb][x], dV = b - a;
                g[0] = dC * c0 + dV * c1;
                g[1] = dC * c2 + dV * c3;
            }
            {
                S a = 0.25 * (((tl.v[yb][x] + tl.v[yb][x + 1]) + tl.v[yt][x]) + tl.v[yt][x + 1]);
                S b = 0.25 * (((tl.v[yb][x - 1] + tl.v[yb][x]) + tl.v[yt][x - 1]) + tl.v[yt][x]);
                S dC = tl.v[yt][x] - tl.v[yb][x], dV = b - a;
                g[2] = dC * c0 + dV * c1;
                g[3] = dC * c2 + dV * c3;
            }
            {
                S a = 0.25 * (((tl.T[yb][x] + tl.T[yb][x + 1]) + tl.T[yt][x]) + tl.T[yt][x + 1]);
                S b = 0.25 * (((tl.T[yb][x - 1] + tl.T[yb][x]) + tl.T[yt][x - 1]) + tl.T[yt][x]);
                S dC = tl.T[yt][x] - tl.T[yb][x], dV = b - a;
                g[4] = dC * c0 + dV * c1;
                g[5] = dC * c2 + dV * c3;
            }
            S mu_f = SUTH ? 0.5 * (tl.mu[yb][x] + tl.mu[yt][x]) : lift<S>(C.mu);
            S u_f = 0.5 * (tl.u[yb][x] + tl.u[yt][x]);
            S v_f = 0.5 * (tl.v[yb][x] + tl.v[yt][x]);
            S div = g[0] + g[3];
            S txx = mu_f * (2.0 * g[0] - C.c23 * div);
            S tyy = mu_f * (2.0 * g[3] - C.c23 * div);
            S txy = mu_f * (g[1] + g[2]);
            S tnx = txx * nxf + txy * nyf;
            S tny = txy * nxf + tyy * nyf;
            S kf = mu_f * C.kfac;
            S dTn = g[4] * nxf + g[5] * nyf;
            F[1] = F[1] - tnx;
            F[2] = F[2] - tny;
            F[3] = F[3] - ((u_f * tnx + v_f * tny) + kf * dTn);
        }
        const double len = G.jl[fi];
#endif
#pragma unroll
        for (int k = 0; k < 4; ++k) fc.fy[k][fy][fx] = F[k] * len;
    };
    for (int bt = tid >> 5; bt < BX + BY; bt += NT / 32) {
        const int lane = tid & 31;
        if (bt < BX) {
            const int f = bt * 32 + lane;
            if (f < NFX) xface(f);
        } else {
            const int f = (bt - BX) * 32 + lane;
            if (f < NFY) yface(f);
        }
    }
#endif
    __syncthreads();

    const int tx = tid % TX, ty = tid / TX;
    const int gi = i0 + tx, gj = j0 + ty;
    if (gi < nx && gj < ny) {
        size_t c = (size_t)gj * nx + gi;
        double iv = G.inv_vol[c];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            S dX = fc.fx[k][ty][tx + 1] - fc.fx[k][ty][tx];
            S dY = fc.fy[k][ty + 1][tx] - fc.fy[k][ty][tx];
            S r = -((dX + dY) * iv);
            epilogue_store(io, s1, s2, k * nc + c, result(r));
        }
    }
}

// Lorenz-96 (appendix): f_i = (u_{i+1} - u_{i-2}) u_{i-1} - u_i + F, periodic,
// with the stencil launch's state formation and epilogue (dual numbers: the
// exact JVP along io.dir / io.dirf).
template <class S>
__global__ void lorenz_kernel(const StencilConsts C, const StencilIO io, int n)
{
    if (io.active && *io.active == 0) return;
    double cf[kMaxAdd], cff, s1, s2;
    coefs(io, cf, cff, s1, s2);
    auto q = [&](int i) {
        i = (i % n + n) % n;
        return load_state<S>(io, cf, cff, (size_t)i);
    };
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        S r = ((q(i + 1) - q(i - 2)) * q(i - 1) - q(i)) + C.lorenz_f;
        epilogue_store(io, s1, s2, (size_t)i, result(r));
    }
}

cudaError_t launch_lorenz(const StencilConsts &c, const StencilIO &io, int n, cudaStream_t s)
{
    if (io.dir || io.dirf) lorenz_kernel<Dual><<<(n + 255) / 256, 256, 0, s>>>(c, io, n);
    else lorenz_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(c, io, n);
    return cudaGetLastError();
}

template <bool V, bool SU, class S>
static cudaError_t launch_cart_t(const StencilConsts &c, const StencilIO &io, cudaStream_t s)
{
    constexpr int MINB = sizeof(S) == sizeof(double) ? 3 : 1;
    const size_t smem = sizeof(Tile<S, CartShape>) + sizeof(Faces<S, CartShape>) + sizeof(Diffs<S, CartShape>) +
                        pair_sums_bytes<V, S, CartShape>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(cart_kernel<V, SU, S, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((c.nx + CartShape::TX - 1) / CartShape::TX, (c.ny + CartShape::TY - 1) / CartShape::TY);
    cart_kernel<V, SU, S, MINB><<<grid, CartShape::NT, smem, s>>>(c, io);
    return cudaGetLastError();
}

template <bool V, bool SU, class S>
static cudaError_t launch_curv_t(const StencilConsts &c, const CurvGeom &g, const StencilIO &io, cudaStream_t s)
{
    constexpr int MINB = sizeof(S) == sizeof(double) ? 3 : 1;
    const size_t smem = sizeof(Tile<S>) + sizeof(Faces<S>) + sizeof(Diffs<S>);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(curv_kernel<V, SU, S, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((c.nx + TX - 1) / TX, (c.ny + TY - 1) / TY);
    curv_kernel<V, SU, S, MINB><<<grid, NT, smem, s>>>(c, g, io);
    return cudaGetLastError();
}

// residual / FD-JVP launches use binary64 scalars; a launch with a direction
// (io.dir or io.dirf) runs the dual-number kernel and writes the exact JVP
cudaError_t launch_cart(const StencilConsts &c, const StencilIO &io, cudaStream_t s)
{
    const bool dual = io.dir || io.dirf;
    if (!c.viscous) return dual ? launch_cart_t<false, false, Dual>(c, io, s) : launch_cart_t<false, false, double>(c, io, s);
    if (c.sutherland)
        return dual ? launch_cart_t<true, true, Dual>(c, io, s) : launch_cart_t<true, true, double>(c, io, s);
    return dual ? launch_cart_t<true, false, Dual>(c, io, s) : launch_cart_t<true, false, double>(c, io, s);
}

template <bool V, bool SU, class SH>
static cudaError_t launch_cart_batch_t(const StencilConsts &c, const StencilIO &io, const BatchTiles &bt, int ntiles,
                                       cudaStream_t s)
{
    const size_t smem = sizeof(Tile<double, SH>) + sizeof(Faces<double, SH>) + sizeof(Diffs<double, SH>) +
                        pair_sums_bytes<V, double, SH>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(cart_batch_kernel<V, SU, SH, 3>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cart_batch_kernel<V, SU, SH, 3><<<ntiles, SH::NT, smem, s>>>(c, io, bt);
    return cudaGetLastError();
}

template <bool V, bool SU>
static cudaError_t launch_cart_batch_v(const StencilConsts &c, const StencilIO &io, const BatchTiles &bt, int ntiles,
                                       int shape, cudaStream_t s)
{
    switch (shape) {
    case kShape32x8: return launch_cart_batch_t<V, SU, Shape<32, 8>>(c, io, bt, ntiles, s);
    case kShape16x16: return launch_cart_batch_t<V, SU, Shape<16, 16>>(c, io, bt, ntiles, s);
    case kShape64x4: return launch_cart_batch_t<V, SU, Shape<64, 4>>(c, io, bt, ntiles, s);
    default: return cudaErrorInvalidValue;
    }
}

// batched residual / FD-JVP launch over the tiles of many grids (binary64 only)
cudaError_t launch_cart_batch(const StencilConsts &c, const StencilIO &io, const BatchTiles &bt, int ntiles, int shape,
                              cudaStream_t s)
{
    if (io.dir || io.dirf || io.addf) return cudaErrorInvalidValue;
    if (ntiles <= 0) return cudaSuccess;
    if (!c.viscous) return launch_cart_batch_v<false, false>(c, io, bt, ntiles, shape, s);
    if (c.sutherland) return launch_cart_batch_v<true, true>(c, io, bt, ntiles, shape, s);
    return launch_cart_batch_v<true, false>(c, io, bt, ntiles, shape, s);
}

cudaError_t launch_curv(const StencilConsts &c, const CurvGeom &g, const StencilIO &io, cudaStream_t s)
{
    const bool dual = io.dir || io.dirf;
    if (!c.viscous)
        return dual ? launch_curv_t<false, false, Dual>(c, g, io, s) : launch_curv_t<false, false, double>(c, g, io, s);
    if (c.sutherland)
        return dual ? launch_curv_t<true, true, Dual>(c, g, io, s) : launch_curv_t<true, true, double>(c, g, io, s);
    return dual ? launch_curv_t<true, false, Dual>(c, g, io, s) : launch_curv_t<true, false, double>(c, g, io, s);
}

#endif  // ROK_STENCIL_DEVICE_ONLY

}  // namespace ROK_NS
}  // namespace rok
