// The single-problem context (rok_ctx of include/rok.h): description, kernel
// constants, workspace and caches, shared by the host drivers of the forward
// step (api.cu) and of its reverse (adjoint.cu).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <utility>
#include <vector>

#include "linalg.cuh"
#include "rok_internal.h"

using namespace rok;

struct AdjWork;   // workspace of the reverse step (adjoint.cu), created on first use

struct rok_ctx {
    rok_problem_desc d;
    StencilConsts C;
    bool curv = false;
    bool strict = false;
    int kind = 0;
    size_t nc = 0, N = 0;
    int P = 0;                 // CTAs (partials) of a reduction over N entries
    int egrid = 0;             // CTAs of the element-wise kernels
    const LinalgOps *ops = nullptr;
    int mmax = 0;
    cudaStream_t stream = nullptr;
    // workspace
    double *V = nullptr;       // (mmax+1) x N basis (binary64; also the GMRES basis)
    float *Vf = nullptr;       // (mmax+1) x N binary32 basis of the mixed-precision ROK step
    bool fp32 = false;
    bool exact_jvp = false;    // Jacobian-vector products by dual numbers inside the steps
    double *F[4] = {};         // stage residuals
    double *K[4] = {};         // stage vectors
    double *w = nullptr, *t0 = nullptr, *t1 = nullptr, *t2 = nullptr;
    double *pA = nullptr, *pB = nullptr, *pM = nullptr;   // partial sums
    StepState *st = nullptr;
    unsigned *colcnt = nullptr; // arrival counters of the persistent Gram-Schmidt column kernels
    int col_ctas = 0;           // co-resident CTAs of that kernel (0: multi-kernel path)
    bool persistent = true;     // use the persistent column kernels where they fit
    StepState *h_st = nullptr;  // pinned mirror
    double *h_part = nullptr;   // pinned, >= 2P
    // curvilinear geometry (device)
    std::vector<double *> geo_bufs;
    CurvGeom G{};
    double *cfl_six = nullptr, *cfl_siy = nullptr, *cfl_sjx = nullptr, *cfl_sjy = nullptr, *cfl_vol = nullptr;
    // counters / timing
    long long launches = 0, stencil_launches = 0, stencil_timed = 0;
    double stencil_ms = 0.0;
    bool time_stencil = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
    // graph cache
    bool use_graph = false;
    std::map<std::pair<double *, int>, cudaGraphExec_t> graphs;
    std::map<std::pair<double *, int>, long long> graph_launches;
    bool capturing = false;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    rok_step_info last{};
    AdjWork *adj = nullptr;   // reverse-step workspace (adjoint.cu)
};

// free the reverse-step workspace (adjoint.cu)
void rok_free_adjoint(rok_ctx *c);
