// Vector kernels of the ROK step on GB300: deterministic reductions, the
// modified-Gram-Schmidt Arnoldi passes (Sec. 2.3.3), the projected stage
// solves of Eq. ROK, stage vectors and combines.  Declarations shared by
// linalg.cu (definitions) and api.cu (host drivers).
#pragma once
#include <cuda_runtime.h>

#include "rok_internal.h"

namespace rok {

constexpr int kRedThreads = 256;

// Step state kept in device memory so that a whole step runs without host
// synchronisation (and can be captured in a CUDA graph).
struct StepState {
    double h, hg;             // step size, h * gamma
    double eps, inv_eps;      // finite-difference increment (Eq. matvecFD)
    double ynorm;             // ||y_n||
    double wnorm0;            // ||J v_j|| before orthogonalisation (breakdown test)
    double beta;              // ||f(y_n)||
    int active;               // Arnoldi still extending the basis
    int meff;                 // Krylov dimension built
    int status;               // latched error bits
    int pad;
    double H[(kMaxKrylov + 1) * kMaxKrylov];   // row-major, stride kMaxKrylov
    double LU[kMaxKrylov * kMaxKrylov];
    int piv[kMaxKrylov];
    double lam[4][kMaxKrylov];
    double cvec[4][kMaxKrylov];
    double phi[kMaxKrylov];
    double gcoef[kMaxKrylov + 1];  // host-provided coefficients (GMRES update)
};

// ---- launchers (linalg.cu) ---------------------------------------------------
void set_elem_blocks(int blocks);
cudaError_t launch_set_int(int *p, int v, cudaStream_t s);
// out partials[2*P]: [0, P) sum a0*b0, [P, 2P) sum a1*b1 (a1 may be NULL: skipped)
cudaError_t launch_dot2(const double *a0, const double *b0, const double *a1, const double *b1, size_t n,
                        double *partials, int P, const int *active, cudaStream_t s);
// h = sum(pin[0..P)); H entry <- h; w -= h vprev; pout <- partial dots of (vnext, w) or (w, w)
// if first: also st->wnorm0 = sqrt(sum(pin[P..2P)))
cudaError_t launch_mgs(double *w, const double *vprev, const double *vnext, size_t n, const double *pin,
                       int P, double *hout, double *pout, bool first, StepState *st, cudaStream_t s);
// hn = sqrt(sum pin[0..P)); breakdown / beta tests; v = w * (1/hn); hsub (nullable) <- hn
cudaError_t launch_normalize(const double *w, double *v, size_t n, const double *pin, int P, double *hsub,
                             int column, StepState *st, cudaStream_t s);
// multi-dot: pout[m*P + b] = partial of <V_m, F>, m < meff
cudaError_t launch_multidot(const double *F, const double *V, size_t ldv, size_t n, double *pout, int P,
                            const StepState *st, cudaStream_t s);
// stage i: phi = reduce(pin), rhs = h phi + h H sum_j gam_ij lam_j, lam_i = LU solve, cvec_i = lam_i - h phi
cudaError_t launch_stage_solve(int stage, const double *gam_row, const double *pin, int P, StepState *st,
                               cudaStream_t s);
// LU with partial pivoting of I - h g H (meff x meff)
cudaError_t launch_lu(StepState *st, cudaStream_t s);
// k = sum_m cvec[stage][m] V_m + h F
cudaError_t launch_stage_vec(double *k, const double *F, const double *V, size_t ldv, size_t n, int stage,
                             const StepState *st, cudaStream_t s);
// out = base + sum_t c_t v_t (c_t host; count <= 8); if guard: skip when st->status != 0
cudaError_t launch_axpy_n(double *out, const double *base, const double *const *v, const double *c, int count,
                          size_t n, const StepState *guard, cudaStream_t s);
// out = sum_{m<count} gcoef[m] V_m + base (GMRES update x += V y), coefficients on the device
cudaError_t launch_basis_combine(double *out, const double *base, const double *V, size_t ldv, size_t n,
                                 int count, const double *gcoef, cudaStream_t s);
// eps from reduced ||y||^2 (pin[0..P)) and ||v||^2 (pin[P..2P)) or vnorm = 1 when v_unit
cudaError_t launch_eps(const double *pin, int P, bool v_unit, double eps_given, StepState *st, cudaStream_t s);
// begin a step: h, hg, meff = M, active = (M > 0)
cudaError_t launch_begin(StepState *st, double h, double gamma, int M, cudaStream_t s);
// beta = sqrt(sum pin); if beta == 0: meff = 0, active = 0
cudaError_t launch_sum_sqrt(const double *pin, int P, double *dst, cudaStream_t s);
// dt from CFL: per-cell spectral-radius bound, max reduction
cudaError_t launch_cfl(const double *y, const StencilConsts &c, const double *geo_six, const double *geo_siy,
                       const double *geo_sjx, const double *geo_sjy, const double *geo_vol, double *pmax, int P,
                       cudaStream_t s);

}  // namespace rok
