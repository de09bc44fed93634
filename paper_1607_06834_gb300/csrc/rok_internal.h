// Internal declarations of librok: parameter blocks shared by the host
// drivers and the kernels, launch helpers, status codes on the device.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "rok.h"

namespace rok {

constexpr int kMaxKrylov = 64;   // largest Krylov dimension / GMRES restart length
constexpr int kMaxAdd = 3;       // vectors added to the base state in one stencil load

// device status word bits (latched; read by rok_sync / info)
enum : int {
    kStatusNonfinite = 1,
    kStatusSingular = 2,
    kStatusTimeout = 4,    // a bounded device wait (arrival counter) gave up
};


// Constants of the finite-volume residual (Sec. 3.2).  Every derived constant is
// computed on the host by the same expression the plain CPU evaluation uses, so the
// strict-rounding stencil reproduces it bit for bit.
struct StencilConsts {
    int nx, ny;
    int bc[4];
    int viscous, sutherland;
    double gm1, inv_gm1;       // gamma - 1, 1 / (gamma - 1)
    double c_lo, c_hi;         // 0.25 (1 - kappa), 0.25 (1 + kappa)
    double efix;               // Harten coefficient
    double kfac, c23;          // gamma / ((gamma - 1) Pr), 2 / 3
    double g_over_pr;          // gamma / Pr (viscous time-step bound)
    double mu, inv_tref, suth_s;
    double rdx, rdy, q_rdx, q_rdy;  // 1/dx, 1/dy, 0.25/dx, 0.25/dy (uniform grids)
    double prim_inf[6];        // rho, u, v, p, T, mu of the free stream
    double lorenz_f;
    // FMA build of the stencil (faces hold G = 2F): gamma/(gamma-1), (gamma-1)/2,
    // 0.5/dx, 0.5/dy, the uniform-grid viscous coefficients of face_coefs() and
    // the curvilinear ones (m 4/3, -m 2/3, m, m k with m as in face_coefs)
    double gg, gm1h, hrdx, hrdy;
    double vk[2][5];
    double vc[4];
    double efix_k;             // (1 - efix) / (1 + efix): c~ efix_k >= |u~| <=> c~ - |u~| >= efix (|u~| + c~)
};

// Viscous coefficients of the doubled face flux G = 2F of a uniform grid, per
// face direction d (0: x-faces, 1: y-faces; n the face normal, t the tangent).
// With the cell differences across the face (dnn: normal velocity, dtn:
// tangential velocity, dTn: temperature) and the four-cell differences along it
// (dnt: normal velocity, dtt: tangential velocity):
//   2 tau_nn = m (vk0 dnn + vk1 dtt),  2 tau_nt = m (vk2 dnt + vk3 dtn),
//   2 k dT/dn = m vk4 dTn,
// where m = 1 and the factor 2 mu is folded in for a constant viscosity, and
// m = mu_L + mu_R (= 2 mu_face) with Sutherland's law (Sec. 3.2, Stokes'
// hypothesis: tau_nn = mu (4/3 du_n/dn - 2/3 du_t/dt)).
inline void face_coefs(double mu, bool sutherland, double kfac, double rdx, double rdy, double vk[2][5])
{
    const double m = sutherland ? 1.0 : 2.0 * mu;
    const double rdn[2] = {rdx, rdy}, qrdt[2] = {0.25 * rdy, 0.25 * rdx};
    for (int d = 0; d < 2; ++d) {
        vk[d][0] = m * (4.0 / 3.0) * rdn[d];
        vk[d][1] = -m * (2.0 / 3.0) * qrdt[d];
        vk[d][2] = m * qrdt[d];
        vk[d][3] = m * rdn[d];
        vk[d][4] = m * kfac * rdn[d];
    }
}

// the FMA-build constants from the fields above (gm1, inv_gm1, mu, kfac, rdx, rdy)
inline void set_fast_consts(StencilConsts &C)
{
    C.gg = C.inv_gm1 + 1.0;
    C.gm1h = 0.5 * C.gm1;
    C.efix_k = (1.0 - C.efix) / (1.0 + C.efix);
    C.hrdx = 0.5 * C.rdx;
    C.hrdy = 0.5 * C.rdy;
    face_coefs(C.mu, C.sutherland != 0, C.kfac, C.rdx, C.rdy, C.vk);
    const double m = C.sutherland ? 1.0 : 2.0 * C.mu;
    C.vc[0] = m * (4.0 / 3.0);
    C.vc[1] = -m * (2.0 / 3.0);
    C.vc[2] = m;
    C.vc[3] = m * C.kfac;
}

// Face metrics of a curvilinear grid (device arrays).
struct CurvGeom {
    // i-faces: (nx+1) * ny, index j*(nx+1)+i ; j-faces: nx * (ny+1), index j*nx+i
    const double *in_x, *in_y, *il, *ic0, *ic1, *ic2, *ic3;
    const double *jn_x, *jn_y, *jl, *jc0, *jc1, *jc2, *jc3;
    const double *inv_vol;     // nx * ny
};

// Inputs and epilogue of one stencil launch:
//   state = base + sum_t c_t add_t [+ cf addf]     (c_t from coef or *coef_dev;
//                                                  addf: a binary32 vector, read exactly)
//   t     = (sub ? r - sub : r) * s1              (s1 times *s1_dev if given)
//   out   = add_out ? add_out + s2 t : t          (s2 times *s2_dev if given)
// With a direction (dir or dirf) the stencil runs on dual numbers and r is the
// exact directional derivative J(state) dir instead of the residual.
struct StencilIO {
    const double *base;
    const double *add[kMaxAdd];
    double coef[kMaxAdd];
    const double *coef_dev[kMaxAdd];
    int nadd;
    const float *addf;         // nullable binary32 term (mixed-precision Krylov basis)
    double coef_f;
    const double *coef_f_dev;
    const double *dir;         // exact JVP: direction v (the launch then writes J(state) v)
    const float *dirf;         // ... or its binary32 form
    const double *sub;
    double s1;
    const double *s1_dev;
    const double *add_out;
    double s2;
    const double *s2_dev;
    double *out;
    int *status;
    const int *active;         // nullable device flag: 0 = skip the launch's work
};

// ---- batches of independent uniform periodic grids ----------------------------
// Per-instance constants of a batch (device array).  Flat vectors hold instance
// k's N_k = 4 nx ny entries at [off, off + N_k); off is a multiple of 2048, the
// entries of a reduction CTA, so that every CTA chunk belongs to one instance.
struct BatchInst {
    int nx, ny;
    size_t off, n;             // element offset and length N_k
    int chunk0, nchunks;       // first 2048-entry chunk and chunk count P_k
    double rdx, rdy, q_rdx, q_rdy, mu;
    double hrdx, hrdy, vk[2][5];   // FMA-build constants (face_coefs)
};

// Tile table of one batched stencil launch (device arrays): CTA b computes tile
// b - tile_first[k] of instance k = tile_inst[b]; per-instance scalars are
// stride_bytes apart.
struct BatchTiles {
    const int *tile_inst;
    const int *tile_first;
    const BatchInst *inst;
    size_t stride_bytes;
};

// tile shapes of the batched stencil (the autotuner picks one per physics group)
enum { kShape32x8 = 0, kShape16x16 = 1, kShape64x4 = 2, kNumShapes = 3 };
inline int shape_tx(int s) { return s == kShape16x16 ? 16 : (s == kShape64x4 ? 64 : 32); }
inline int shape_ty(int s) { return s == kShape16x16 ? 16 : (s == kShape64x4 ? 4 : 8); }

// stencil launchers, one set per rounding mode (separate translation units)
namespace fast {
cudaError_t launch_cart(const StencilConsts &c, const StencilIO &io, cudaStream_t s);
cudaError_t launch_curv(const StencilConsts &c, const CurvGeom &g, const StencilIO &io, cudaStream_t s);
cudaError_t launch_lorenz(const StencilConsts &c, const StencilIO &io, int n, cudaStream_t s);
cudaError_t launch_cart_batch(const StencilConsts &c, const StencilIO &io, const BatchTiles &bt, int ntiles,
                              int shape, cudaStream_t s);
}
namespace strict {
cudaError_t launch_cart(const StencilConsts &c, const StencilIO &io, cudaStream_t s);
cudaError_t launch_curv(const StencilConsts &c, const CurvGeom &g, const StencilIO &io, cudaStream_t s);
cudaError_t launch_lorenz(const StencilConsts &c, const StencilIO &io, int n, cudaStream_t s);
cudaError_t launch_cart_batch(const StencilConsts &c, const StencilIO &io, const BatchTiles &bt, int ntiles,
                              int shape, cudaStream_t s);
}

}  // namespace rok
