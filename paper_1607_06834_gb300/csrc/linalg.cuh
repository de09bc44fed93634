// Vector kernels of the ROK step on GB300: deterministic reductions, the
// modified-Gram-Schmidt Arnoldi passes (Sec. 2.2.2), the projected stage
// solves of Eq. ROK, stage vectors and combines.  Declarations shared by
// linalg.cu (definitions) and api.cu (host drivers).
#pragma once
#include <cuda_runtime.h>

#include "rok_internal.h"

namespace rok {


// Arrival counters of the persistent Arnoldi column kernel: column j uses the
// j + 2 counters from column_counter_offset(j); an Arnoldi process of M columns
// zeroes the first column_counter_offset(M) before its first column.
inline size_t column_counter_offset(int j) { return (size_t)j * (j + 3) / 2; }

// Step state kept in device memory so that a whole step runs without host
// synchronisation (and can be captured in a CUDA graph).
// Restarted GMRES(m) of the comparators' stage solves, kept on the device so
// that a restart cycle runs without host round trips: Givens rotations of the
// Hessenberg columns (rotated in place in StepState::H), the rotated
// right-hand side g, the residual estimate and the stop flags.
struct GmresState {
    double cs[kMaxKrylov], sn[kMaxKrylov];
    double g[kMaxKrylov + 1];
    double bnorm, tol_abs;   // ||rhs||, tol ||rhs||
    double res;              // |g_{k}|: residual estimate of the current iterate
    int m;                   // restart length
    int k;                   // columns in the current cycle's least-squares system
    int its;                 // Arnoldi columns processed in this solve
    int live;                // the current cycle is still extending its basis
    int conv;                // converged (residual estimate <= tol ||rhs||)
    int pad;
};

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
    double phis[4][kMaxKrylov];    // phi of every stage (kept for the reverse step)
    double gcoef[kMaxKrylov + 1];  // coefficients of the GMRES update x += V gcoef
    GmresState gm;
    double gram[kMaxKrylov];       // <v_{i+1}, v_i> of the basis (FMA-build two-vector passes)
};

// ---- rounding-mode dependent vector kernels (linalg_impl.cuh, compiled twice) ----
struct LinalgOps {
    // partials[b] = <a0,b0>, partials[P+b] = <a1,b1> (a1 nullable) over CTA b's 2048 entries
    cudaError_t (*dot2)(const double *a0, const double *b0, const double *a1, const double *b1, size_t n,
                        double *partials, int P, const int *active, cudaStream_t s);
    // h = tree(pin); *hout = h; w -= h vprev; pout[b] = <vnext, w> (or <w, w> when vnext is NULL);
    // first: also st->wnorm0 = sqrt(tree(pin + P))
    cudaError_t (*mgs)(double *w, const double *vprev, const double *vnext, size_t n, const double *pin, int P,
                       double *hout, double *pout, bool first, StepState *st, cudaStream_t s);
    // hn = sqrt(tree(pin)); breakdown / beta tests; v = w * (1/hn); *hsub = hn (nullable)
    cudaError_t (*normalize)(const double *w, double *v, size_t n, const double *pin, int P, double *hsub,
                             int column, StepState *st, cudaStream_t s);
    // pout[m*P + b] = <V_m, F> over CTA b's entries, m < meff; V binary64 or (fp32) binary32
    cudaError_t (*multidot)(const double *F, const void *V, int fp32, size_t ldv, size_t n, double *pout, int P,
                            const StepState *st, cudaStream_t s);
    // stage i: phi, rhs = h phi + h H sum_j gam_ij lam_j, lam_i by LU, cvec_i = lam_i - h phi
    cudaError_t (*stage_solve)(int stage, const double *gam_row, const double *pin, int P, StepState *st,
                               cudaStream_t s);
    // LU with partial pivoting of I - h g H (meff x meff)
    cudaError_t (*lu)(StepState *st, cudaStream_t s);
    // k = sum_m cvec[stage][m] V_m + h F (V binary64 or binary32, arithmetic binary64)
    cudaError_t (*stage_vec)(double *k, const double *F, const void *V, int fp32, size_t ldv, size_t n, int stage,
                             const StepState *st, int grid, cudaStream_t s);
    // out = base + sum_q c_q v_q (count <= 8, host coefficients); skipped when guard->status != 0
    cudaError_t (*axpy_n)(double *out, const double *base, const double *const *v, const double *c, int count,
                          size_t n, const StepState *guard, int grid, cudaStream_t s);
    // out = base + sum_{m<count} gcoef[m] V_m (device coefficients; count_dev, when
    // not null, lowers count to *count_dev on the device)
    cudaError_t (*basis_combine)(double *out, const double *base, const double *V, size_t ldv, size_t n, int count,
                                 const double *gcoef, const int *count_dev, int grid, cudaStream_t s);
    // eps from tree(pin) = ||y||^2 and tree(pin + P) = ||v||^2 (or ||v|| = 1)
    cudaError_t (*eps)(const double *pin, int P, bool v_unit, double eps_given, StepState *st, cudaStream_t s);
    cudaError_t (*sum_sqrt)(const double *pin, int P, double *dst, cudaStream_t s);
    // One whole Arnoldi column j in a single cooperative launch (grid = ctas,
    // co-resident): h_ij = <v_i, w>, w -= h_ij v_i for i = 0..j (modified
    // Gram-Schmidt), then, when next != 0, h_{j+1,j} = ||w||, the breakdown test
    // and v_{j+1} = w * (1/h_{j+1,j}).  w and the next basis vector stay in
    // registers between passes; partA holds 4P partials, partB 2P; cnt[0 ..
    // j + 2) are the arrival counters of the partial generations, zero on entry
    // (column_counter_offset).  Strict build: the same arithmetic as dot2 + mgs
    // + normalize.  FMA build: two basis vectors a pass (MGS to rounding); the
    // columns of one basis run in order, and partA[2G, 3G) (G <= P its grid)
    // carries the partials of <v_{j+1}, v_j> from column j to column j + 1;
    // the breakdown test's scale ||J v_j|| is (sum_i h_ij^2 + h_{j+1,j}^2)^(1/2).
    // Returns cudaErrorNotSupported when the ctas cannot cover the P chunks
    // (caller falls back).
    // fp32: the basis V is binary32 and the Gram-Schmidt arithmetic binary32 (w rounded on load);
    // the FMA build orthogonalises by CGS2 then (two waits per column) and takes
    // partA as 2 (kMaxKrylov + 1) P binary32 partials (partB unused)
    cudaError_t (*arnoldi_column)(const double *w, void *V, int fp32, size_t ldv, size_t n, int j, int next, int P,
                                  double *partA, double *partB, unsigned *cnt, StepState *st, int ctas,
                                  cudaStream_t s);
    // co-resident CTAs of arnoldi_column on this device (0 if cooperative launch is unavailable)
    int (*arnoldi_column_ctas)(int sms);
    // v_1 = (T)F1 / ||(T)F1|| (T = binary64 or binary32); beta = 0: empty basis
    cudaError_t (*first_vector)(const double *F, void *V0, int fp32, size_t n, double *partials, int P,
                                StepState *st, cudaStream_t s);
    // partials[b] = sum over CTA b of (e_i / sc_i)^2, e = sum_q d_q k_q (count <= 8, in order),
    // sc_i = atol + rtol max(|y_i|, |ynew_i|): the weighted RMS norm of an error estimate
    cudaError_t (*err_sum)(const double *y, const double *ynew, const double *const *kv, const double *d, int count,
                           double atol, double rtol, size_t n, double *partials, int P, cudaStream_t s);
    // Restarted GMRES on the device.  gmres_start: ||rhs|| = sqrt(tree(pin)),
    // tol_abs = tol ||rhs||, counters reset (||rhs|| = 0: converged at x = 0).
    cudaError_t (*gmres_start)(const double *pin, int P, double tol, int m, StepState *st, cudaStream_t s);
    // gmres_cycle: beta = sqrt(tree(pin)), the norm of the cycle's starting
    // residual; converged when beta <= tol_abs, otherwise g = beta e_1, the
    // subdiagonal of H cleared and the Arnoldi flag set for the cycle.
    cudaError_t (*gmres_cycle)(const double *pin, int P, StepState *st, cudaStream_t s);
    // gmres_givens: column j of H (written by the Arnoldi column) rotated by the
    // earlier rotations, the new rotation, g updated, residual estimate; stops
    // the cycle (Arnoldi flag cleared) at convergence, breakdown or column m-1.
    cudaError_t (*gmres_givens)(int j, StepState *st, cudaStream_t s);
    // gmres_lsq: R y = g by back substitution into gcoef[0 .. k)
    cudaError_t (*gmres_lsq)(StepState *st, cudaStream_t s);
};

// Segment table of a batch (device arrays): chunk c of a flat vector belongs to
// instance chunk_inst[c]; st is the per-instance step state array.
struct BSeg {
    const int *chunk_inst;
    const BatchInst *inst;
    StepState *st;
    int nchunks;
};

// ---- batched forms of the ROK step kernels (same arithmetic per instance) ----
// cpc = 2048-entry chunks per CTA (grid = ceil(nchunks / cpc)); part/pin/pout hold
// one partial per chunk (two sets for dot2 and the first MGS pass).
struct BatchOps {
    cudaError_t (*dot2)(const double *a0, const double *b0, const double *a1, const double *b1, double *part,
                        const BSeg &sg, int use_active, int cpc, cudaStream_t s);
    // eps of every instance from ||y||^2 partials (unit direction)
    cudaError_t (*eps)(const double *part, const BSeg &sg, int ninst, cudaStream_t s);
    cudaError_t (*first_normalize)(const double *F, double *V0, const double *part, const BSeg &sg, int cpc,
                                   cudaStream_t s);
    // MGS pass i (1 <= i <= j + 1) of column j
    cudaError_t (*mgs)(double *w, const double *V, size_t ldv, int i, int j, const double *pin, double *pout,
                       const BSeg &sg, int cpc, cudaStream_t s);
    cudaError_t (*normalize)(const double *w, double *V, size_t ldv, int column, const double *pin, const BSeg &sg,
                             int cpc, cudaStream_t s);
    cudaError_t (*multidot)(const double *F, const double *V, size_t ldv, double *pout, const BSeg &sg, int cpc,
                            cudaStream_t s);
    cudaError_t (*stage_solve)(int stage, const double *gam_row, const double *pin, const BSeg &sg, int ninst,
                               cudaStream_t s);
    cudaError_t (*lu)(StepState *st, int ninst, cudaStream_t s);
    cudaError_t (*stage_vec)(double *k, const double *F, const double *V, size_t ldv, int stage, const BSeg &sg,
                             int cpc, cudaStream_t s);
    // y += sum_q b_q k_q (4 stage vectors), skipped for instances with a latched status
    cudaError_t (*update)(double *y, const double *const *kv, const double *b, const BSeg &sg, int cpc,
                          cudaStream_t s);
};

namespace fast {
extern const LinalgOps ops;
extern const BatchOps bops;
}
namespace strict {
extern const LinalgOps ops;
extern const BatchOps bops;
}

// number of CTAs (and partials) of a reduction over n entries: 2048 entries per CTA
inline int reduction_blocks(size_t n) { return n ? (int)((n + 2047) / 2048) : 1; }

// ---- rounding-independent helpers (linalg_common.cu) -----------------------------
cudaError_t launch_set_int(int *p, int v, cudaStream_t s);
// dst = (double) src, n entries (exact widening)
cudaError_t launch_f2d(const float *src, double *dst, size_t n, cudaStream_t s);
// begin a step: h, hg, meff = M, active = (M > 0)
cudaError_t launch_begin(StepState *st, double h, double gamma, int M, cudaStream_t s);
// the same for n instances, h[k] from a device array (latched status kept)
cudaError_t launch_begin_batch(StepState *st, const double *h, double gamma, int M, int n, cudaStream_t s);
// clear the latched status of n instances
cudaError_t launch_clear_status(StepState *st, int n, cudaStream_t s);
// dt from CFL: per-cell spectral-radius bound, max reduction (order independent)
cudaError_t launch_cfl(const double *y, const StencilConsts &c, const double *geo_six, const double *geo_siy,
                       const double *geo_sjx, const double *geo_sjy, const double *geo_vol, double *pmax, int P,
                       cudaStream_t s);

}  // namespace rok
