// Batches of independent problems (include/rok.h, rok_batch_*): the ROK4 step of
// Sec. 2.2.2 (Eq. ROK) applied to many uniform periodic grids at once.  Every
// kernel launch covers all instances: the residual stencil walks a tile table
// that spans the grids of one physics group, the vector kernels walk 2048-entry
// chunks that each belong to one instance, and the small per-instance solves
// run one CTA (or warp) per instance.  The host only enqueues; a whole run of
// steps can be captured in one CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <map>
#include <tuple>
#include <vector>

#include "coefficients.h"
#include "linalg.cuh"
#include "rok_internal.h"

using namespace rok;

namespace {

constexpr int kGroups = 3;   // Euler, Navier-Stokes, Navier-Stokes with Sutherland's law
constexpr int kChunk = 2048; // entries of one reduction CTA chunk
const int kCpcCandidates[4] = {1, 2, 4, 8};

}  // namespace

struct rok_batch {
    int count = 0;
    bool strict = false;
    int mmax = 0;
    cudaStream_t stream = nullptr;
    const BatchOps *bops = nullptr;
    std::vector<BatchInst> inst;   // host copy
    std::vector<int> group;        // physics group per instance
    size_t total = 0;              // flat length
    int nchunks = 0;
    StencilConsts C[kGroups];      // shared constants per group (grid fields per instance)
    bool has_group[kGroups] = {false, false, false};
    double gamma_rok = kRokGamma;
    // device tables
    BatchInst *d_inst = nullptr;
    int *d_chunk_inst = nullptr;
    int *d_tiles = nullptr;                          // all tile tables, one allocation
    const int *tile_inst[kGroups][kNumShapes] = {};
    const int *tile_first[kGroups][kNumShapes] = {};
    int ntiles[kGroups][kNumShapes] = {};
    // workspace
    StepState *st = nullptr;
    double *V = nullptr;           // (mmax + 1) x total
    double *F[4] = {}, *K[4] = {};
    double *w = nullptr, *t0 = nullptr;
    double *pA = nullptr, *pB = nullptr, *pM = nullptr;
    double *d_h = nullptr;
    StepState *h_st = nullptr;     // pinned headers
    // launch shapes
    int tile[kGroups] = {kShape32x8, kShape32x8, kShape32x8};
    int cpc = 1, vcpc = 1;
    // graphs
    bool use_graph = false;
    std::map<std::tuple<double *, int, int>, cudaGraphExec_t> graphs;
    std::map<std::tuple<double *, int, int>, long long> graph_launches;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    long long launches = 0;
};

namespace {

#define CU(x)                                      \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return ROK_ERR_CUDA; \
    } while (0)

void free_batch(rok_batch *b)
{
    if (!b) return;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->gev[0]) cudaEventDestroy(b->gev[0]);
    if (b->gev[1]) cudaEventDestroy(b->gev[1]);
    cudaFree(b->d_inst);
    cudaFree(b->d_chunk_inst);
    cudaFree(b->d_tiles);
    cudaFree(b->st);
    cudaFree(b->V);
    for (int i = 0; i < 4; ++i) { cudaFree(b->F[i]); cudaFree(b->K[i]); }
    cudaFree(b->w); cudaFree(b->t0);
    cudaFree(b->pA); cudaFree(b->pB); cudaFree(b->pM);
    cudaFree(b->d_h);
    cudaFreeHost(b->h_st);
    delete b;
}

int group_of(const rok_problem_desc &d)
{
    if (d.kind == ROK_EULER2D) return 0;
    return d.sutherland_s > 0.0 ? 2 : 1;
}

// constants shared by a group, by the same expressions as rok_init
void group_consts(const rok_problem_desc &d, StencilConsts &C)
{
    memset(&C, 0, sizeof(C));
    C.nx = d.nx;
    C.ny = d.ny;
    for (int k = 0; k < 4; ++k) C.bc[k] = d.bc[k];
    C.viscous = d.kind == ROK_NS2D;
    C.sutherland = d.kind == ROK_NS2D && d.sutherland_s > 0.0;
    C.gm1 = d.gamma - 1.0;
    C.inv_gm1 = 1.0 / C.gm1;
    C.c_lo = 0.25 * (1.0 - d.muscl_kappa);
    C.c_hi = 0.25 * (1.0 + d.muscl_kappa);
    C.efix = d.entropy_fix;
    C.kfac = d.kind == ROK_NS2D ? d.gamma / (C.gm1 * d.prandtl) : 0.0;
    C.c23 = 2.0 / 3.0;
    C.g_over_pr = d.kind == ROK_NS2D ? d.gamma / d.prandtl : 0.0;
    C.mu = d.kind == ROK_NS2D ? d.mu : 0.0;
    C.inv_tref = C.sutherland ? 1.0 / d.t_ref : 0.0;
    C.suth_s = d.sutherland_s;
    C.gg = C.inv_gm1 + 1.0;
    C.gm1h = 0.5 * C.gm1;
    C.efix_k = (1.0 - C.efix) / (1.0 + C.efix);
}

// instances of one group share the gas model and scheme constants
bool same_group_consts(const rok_problem_desc &a, const rok_problem_desc &b)
{
    if (group_of(a) != group_of(b)) return true;
    bool same = a.gamma == b.gamma && a.muscl_kappa == b.muscl_kappa && a.entropy_fix == b.entropy_fix;
    if (a.kind == ROK_NS2D) same = same && a.prandtl == b.prandtl;
    if (group_of(a) == 2) same = same && a.t_ref == b.t_ref && a.sutherland_s == b.sutherland_s;
    return same;
}

BSeg seg(const rok_batch *b)
{
    BSeg s;
    s.chunk_inst = b->d_chunk_inst;
    s.inst = b->d_inst;
    s.st = b->st;
    s.nchunks = b->nchunks;
    return s;
}

StencilIO io_plain(rok_batch *b, const double *y, double *out)
{
    StencilIO io;
    memset(&io, 0, sizeof(io));
    io.base = y;
    io.s1 = 1.0;
    io.s2 = 1.0;
    io.out = out;
    io.status = &b->st[0].status;
    return io;
}

// one stencil pass over every instance: one launch per physics group present;
// `only` >= 0 restricts it to one group (tuning)
rok_status stencil(rok_batch *b, const StencilIO &io, int only = -1, int shape_override = -1)
{
    for (int g = 0; g < kGroups; ++g) {
        if (!b->has_group[g] || (only >= 0 && g != only)) continue;
        const int s = shape_override >= 0 ? shape_override : b->tile[g];
        BatchTiles bt;
        bt.tile_inst = b->tile_inst[g][s];
        bt.tile_first = b->tile_first[g][s];
        bt.inst = b->d_inst;
        bt.stride_bytes = sizeof(StepState);
        cudaError_t e = b->strict ? strict::launch_cart_batch(b->C[g], io, bt, b->ntiles[g][s], s, b->stream)
                                  : fast::launch_cart_batch(b->C[g], io, bt, b->ntiles[g][s], s, b->stream);
        if (e != cudaSuccess) return ROK_ERR_CUDA;
        b->launches++;
    }
    return ROK_OK;
}

// One ROK4 step of every instance, enqueue only (h from the device array).
rok_status enqueue_step(rok_batch *b, double *y, int M)
{
    const BatchOps &o = *b->bops;
    const BSeg sg = seg(b);
    const size_t ldv = b->total;
    const int n = b->count;
    cudaStream_t s = b->stream;
    rok_status r;
    CU(launch_begin_batch(b->st, b->d_h, b->gamma_rok, M, n, s));
    b->launches++;
    // F1 = f(y_n); eps from ||y_n||
    if ((r = stencil(b, io_plain(b, y, b->F[0]))) != ROK_OK) return r;
    CU(o.dot2(y, y, nullptr, nullptr, b->pA, sg, 0, b->cpc, s));
    CU(o.eps(b->pA, sg, n, s));
    b->launches += 2;
    if (M > 0) {
        // v_1 = F1 / ||F1||
        CU(o.dot2(b->F[0], b->F[0], nullptr, nullptr, b->pA, sg, 0, b->cpc, s));
        CU(o.first_normalize(b->F[0], b->V, b->pA, sg, b->vcpc, s));
        b->launches += 2;
        for (int j = 0; j < M; ++j) {
            // w = (f(y + eps v_j) - F1) / eps, then modified Gram-Schmidt
            StencilIO io = io_plain(b, y, b->w);
            io.add[0] = b->V + (size_t)j * ldv;
            io.coef[0] = 1.0;
            io.coef_dev[0] = &b->st[0].eps;
            io.nadd = 1;
            io.sub = b->F[0];
            io.s1_dev = &b->st[0].inv_eps;
            io.active = &b->st[0].active;
            if ((r = stencil(b, io)) != ROK_OK) return r;
            CU(o.dot2(b->V, b->w, b->w, b->w, b->pA, sg, 1, b->cpc, s));
            b->launches++;
            double *pin = b->pA, *pout = b->pB;
            for (int i = 1; i <= j + 1; ++i) {
                CU(o.mgs(b->w, b->V, ldv, i, j, pin, pout, sg, b->cpc, s));
                b->launches++;
                double *t = pin; pin = pout; pout = t;
            }
            if (j + 1 < M) {
                CU(o.normalize(b->w, b->V, ldv, j + 1, pin, sg, b->cpc, s));
                b->launches++;
            }
        }
        CU(o.lu(b->st, n, s));
        b->launches++;
    }
    for (int i = 0; i < 4; ++i) {
        if (i > 0) {
            StencilIO io = io_plain(b, y, b->F[i]);
            for (int j = 0; j < i; ++j)
                if (kRokAlpha[i][j] != 0.0) {
                    io.add[io.nadd] = b->K[j];
                    io.coef[io.nadd] = kRokAlpha[i][j];
                    io.nadd++;
                }
            if ((r = stencil(b, io)) != ROK_OK) return r;
        }
        if (M > 0) {
            CU(o.multidot(b->F[i], b->V, ldv, b->pM, sg, b->cpc, s));
            CU(o.stage_solve(i, kRokGammaOff[i], b->pM, sg, n, s));
            b->launches += 2;
        }
        CU(o.stage_vec(b->K[i], b->F[i], b->V, ldv, i, sg, b->vcpc, s));
        b->launches++;
    }
    const double *kv[4] = {b->K[0], b->K[1], b->K[2], b->K[3]};
    CU(o.update(y, kv, kRokB, sg, b->vcpc, s));
    b->launches++;
    return ROK_OK;
}

rok_status status_of(int bits)
{
    if (bits & (kStatusNonfinite | kStatusSingular)) return ROK_ERR_NONFINITE;
    if (bits & kStatusTimeout) return ROK_ERR_TIMEOUT;
    return ROK_OK;
}

// Tile tables of every (group, shape): instances in order, tiles of an instance
// row by row.
rok_status build_tiles(rok_batch *b)
{
    std::vector<int> all;
    size_t pos[kGroups][kNumShapes][2];
    for (int g = 0; g < kGroups; ++g)
        for (int s = 0; s < kNumShapes; ++s) {
            std::vector<int> ti, tf(b->count, -1);
            for (int k = 0; k < b->count; ++k) {
                if (b->group[k] != g) continue;
                const int tx = (b->inst[k].nx + shape_tx(s) - 1) / shape_tx(s);
                const int ty = (b->inst[k].ny + shape_ty(s) - 1) / shape_ty(s);
                tf[k] = (int)ti.size();
                for (int t = 0; t < tx * ty; ++t) ti.push_back(k);
            }
            b->ntiles[g][s] = (int)ti.size();
            pos[g][s][0] = all.size();
            all.insert(all.end(), ti.begin(), ti.end());
            pos[g][s][1] = all.size();
            all.insert(all.end(), tf.begin(), tf.end());
        }
    if (cudaMalloc(&b->d_tiles, all.size() * sizeof(int)) != cudaSuccess) return ROK_ERR_NOMEM;
    CU(cudaMemcpy(b->d_tiles, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
    for (int g = 0; g < kGroups; ++g)
        for (int s = 0; s < kNumShapes; ++s) {
            b->tile_inst[g][s] = b->d_tiles + pos[g][s][0];
            b->tile_first[g][s] = b->d_tiles + pos[g][s][1];
        }
    return ROK_OK;
}

bool valid_cpc(int c) { return c == 1 || c == 2 || c == 4 || c == 8; }

void clear_graphs(rok_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->graph_launches.clear();
}

// mean device time of `reps` runs of fn on the batch stream, after one warm-up
template <class Fn>
rok_status time_ms(rok_batch *b, int reps, Fn fn, float *out)
{
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    rok_status r = fn();
    if (r == ROK_OK) {
        cudaEventRecord(e0, b->stream);
        for (int i = 0; i < reps && r == ROK_OK; ++i) r = fn();
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) r = ROK_ERR_CUDA;
        float ms = 0.0f;
        if (r == ROK_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = ROK_ERR_CUDA;
        *out = ms / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
}

}  // namespace

extern "C" {

rok_status rok_batch_init(rok_batch **out, const rok_problem_desc *descs, int count, void *stream)
{
    if (!out || !descs || count < 1) return ROK_ERR_INVALID_ARG;
    *out = nullptr;
    for (int k = 0; k < count; ++k) {
        const rok_problem_desc &d = descs[k];
        if (d.kind != ROK_EULER2D && d.kind != ROK_NS2D) return ROK_ERR_INVALID_ARG;
        if (d.nx < 2 || d.ny < 2 || (long long)d.nx * d.ny > (1LL << 26)) return ROK_ERR_INVALID_ARG;
        if (d.xv || d.yv) return ROK_ERR_UNSUPPORTED;
        for (int s = 0; s < 4; ++s)
            if (d.bc[s] != ROK_BC_PERIODIC) return ROK_ERR_UNSUPPORTED;
        if (!(d.lx > 0.0) || !(d.ly > 0.0) || !(d.gamma > 1.0)) return ROK_ERR_INVALID_ARG;
        if (d.kind == ROK_NS2D && (!(d.prandtl > 0.0) || d.mu < 0.0)) return ROK_ERR_INVALID_ARG;
        if (d.kind == ROK_NS2D && d.sutherland_s > 0.0 && !(d.t_ref > 0.0)) return ROK_ERR_INVALID_ARG;
        if (d.rounding != ROK_ROUND_FAST && d.rounding != ROK_ROUND_STRICT) return ROK_ERR_INVALID_ARG;
        if (d.krylov_max < 0 || d.krylov_max > kMaxKrylov) return ROK_ERR_INVALID_ARG;
        if (d.basis != ROK_BASIS_FP64 && d.basis != ROK_BASIS_FP32) return ROK_ERR_INVALID_ARG;
        if (d.jvp != ROK_JVP_FD && d.jvp != ROK_JVP_EXACT) return ROK_ERR_INVALID_ARG;
        if (d.rounding != descs[0].rounding || d.krylov_max != descs[0].krylov_max) return ROK_ERR_INVALID_ARG;
        for (int q = 0; q < k; ++q)
            if (!same_group_consts(d, descs[q])) return ROK_ERR_INVALID_ARG;
    }
    for (int k = 0; k < count; ++k)
        if (descs[k].basis != ROK_BASIS_FP64 || descs[k].jvp != ROK_JVP_FD) return ROK_ERR_UNSUPPORTED;

    rok_batch *b = new rok_batch();
    b->count = count;
    b->strict = descs[0].rounding == ROK_ROUND_STRICT;
    b->mmax = descs[0].krylov_max;
    b->stream = (cudaStream_t)stream;
    b->bops = b->strict ? &strict::bops : &fast::bops;
    b->inst.resize(count);
    b->group.resize(count);
    size_t off = 0;
    int chunk = 0;
    std::vector<int> chunk_inst;
    for (int k = 0; k < count; ++k) {
        const rok_problem_desc &d = descs[k];
        BatchInst &I = b->inst[k];
        memset(&I, 0, sizeof(I));
        I.nx = d.nx;
        I.ny = d.ny;
        I.n = 4 * (size_t)d.nx * d.ny;
        I.off = off;
        I.chunk0 = chunk;
        I.nchunks = (int)((I.n + kChunk - 1) / kChunk);
        const double dx = d.lx / d.nx, dy = d.ly / d.ny;
        I.rdx = 1.0 / dx;
        I.rdy = 1.0 / dy;
        I.q_rdx = 0.25 * I.rdx;
        I.q_rdy = 0.25 * I.rdy;
        I.mu = d.kind == ROK_NS2D ? d.mu : 0.0;
        I.hrdx = 0.5 * I.rdx;
        I.hrdy = 0.5 * I.rdy;
        if (d.kind == ROK_NS2D)
            face_coefs(I.mu, d.sutherland_s > 0.0, d.gamma / ((d.gamma - 1.0) * d.prandtl), I.rdx, I.rdy, I.vk);
        off += (size_t)I.nchunks * kChunk;
        chunk += I.nchunks;
        for (int c = 0; c < I.nchunks; ++c) chunk_inst.push_back(k);
        const int g = group_of(d);
        b->group[k] = g;
        if (!b->has_group[g]) {
            group_consts(d, b->C[g]);
            b->has_group[g] = true;
        }
    }
    b->total = off;
    b->nchunks = chunk;

    const size_t N = b->total;
    auto al = [&](double **p, size_t n) { return cudaMalloc(p, n * sizeof(double)) == cudaSuccess; };
    bool ok = cudaMalloc(&b->d_inst, count * sizeof(BatchInst)) == cudaSuccess &&
              cudaMalloc(&b->d_chunk_inst, b->nchunks * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->st, count * sizeof(StepState)) == cudaSuccess &&
              al(&b->V, (size_t)(b->mmax + 1) * N) && al(&b->w, N) && al(&b->t0, N) &&
              al(&b->pA, 2 * (size_t)b->nchunks) && al(&b->pB, 2 * (size_t)b->nchunks) &&
              al(&b->pM, (size_t)(b->mmax > 0 ? b->mmax : 1) * b->nchunks) && al(&b->d_h, count) &&
              cudaMallocHost(&b->h_st, count * sizeof(StepState)) == cudaSuccess;
    for (int i = 0; i < 4 && ok; ++i) ok = al(&b->F[i], N) && al(&b->K[i], N);
    if (!ok) { free_batch(b); return ROK_ERR_NOMEM; }
    rok_status r = build_tiles(b);
    if (r != ROK_OK) { free_batch(b); return r; }
    if (cudaMemcpy(b->d_inst, b->inst.data(), count * sizeof(BatchInst), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_chunk_inst, chunk_inst.data(), b->nchunks * sizeof(int), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(b->st, 0, count * sizeof(StepState)) != cudaSuccess ||
        cudaMemset(b->d_h, 0, count * sizeof(double)) != cudaSuccess) {
        free_batch(b);
        return ROK_ERR_CUDA;
    }
    *out = b;
    return ROK_OK;
}

rok_status rok_batch_destroy(rok_batch *b)
{
    if (!b) return ROK_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return ROK_OK;
}

rok_status rok_batch_layout(const rok_batch *b, size_t *total, size_t *offsets)
{
    if (!b || !total) return ROK_ERR_INVALID_ARG;
    *total = b->total;
    if (offsets)
        for (int k = 0; k < b->count; ++k) offsets[k] = b->inst[k].off;
    return ROK_OK;
}

rok_status rok_batch_residual(rok_batch *b, const double *y, double *f)
{
    if (!b || !y || !f || y == f) return ROK_ERR_INVALID_ARG;
    return stencil(b, io_plain(b, y, f));
}

rok_status rok_batch_step(rok_batch *b, double *y, const double *h, int M, int nsteps, rok_step_info *info)
{
    if (!b || !y || !h || M < 0 || M > b->mmax || nsteps < 1) return ROK_ERR_INVALID_ARG;
    for (int k = 0; k < b->count; ++k)
        if (!(h[k] > 0.0) || !isfinite(h[k])) return ROK_ERR_INVALID_ARG;
    // pageable source: the copy is staged before the call returns
    CU(cudaMemcpyAsync(b->d_h, h, b->count * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    if (b->use_graph) {
        cudaStream_t user = b->stream;
        if (!b->gstream) {
            CU(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&b->gev[0], cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&b->gev[1], cudaEventDisableTiming));
        }
        CU(cudaEventRecord(b->gev[0], user));
        CU(cudaStreamWaitEvent(b->gstream, b->gev[0], 0));
        auto key = std::make_tuple(y, M, nsteps);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t g;
            const long long l0 = b->launches;
            b->stream = b->gstream;
            cudaError_t e = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal);
            rok_status r = ROK_OK;
            for (int step = 0; step < nsteps && e == cudaSuccess && r == ROK_OK; ++step) r = enqueue_step(b, y, M);
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(b->gstream, &g) : e;
            b->stream = user;
            if (r != ROK_OK) {
                if (e2 == cudaSuccess) cudaGraphDestroy(g);
                return r;
            }
            if (e2 != cudaSuccess) return ROK_ERR_CUDA;
            cudaGraphExec_t ge;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return ROK_ERR_CUDA;
            it = b->graphs.emplace(key, ge).first;
            b->graph_launches[key] = b->launches - l0;
            b->launches = l0;
        }
        CU(cudaGraphLaunch(it->second, b->gstream));
        CU(cudaEventRecord(b->gev[1], b->gstream));
        CU(cudaStreamWaitEvent(user, b->gev[1], 0));
        b->launches += b->graph_launches[key];
    } else {
        for (int step = 0; step < nsteps; ++step) {
            rok_status r = enqueue_step(b, y, M);
            if (r != ROK_OK) return r;
        }
    }
    if (!info) return ROK_OK;
    CU(cudaMemcpy2DAsync(b->h_st, sizeof(StepState), b->st, sizeof(StepState), offsetof(StepState, H), b->count,
                         cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    rok_status first = ROK_OK;
    bool any = false;
    for (int k = 0; k < b->count; ++k) {
        const StepState &s = b->h_st[k];
        rok_step_info &o = info[k];
        memset(&o, 0, sizeof(o));
        o.status = status_of(s.status);
        o.m_eff = s.meff;
        o.eps = s.eps;
        o.residual_evals = nsteps * (1 + M + 3);
        o.jvps = nsteps * M;
        if (o.status != ROK_OK && first == ROK_OK) first = (rok_status)o.status;
        any = any || s.status != 0;
    }
    if (any) {
        CU(launch_clear_status(b->st, b->count, b->stream));
        b->launches++;
    }
    return first;
}

rok_status rok_batch_tune(rok_batch *b, const double *y, rok_batch_tuning *out)
{
    if (!b || !y) return ROK_ERR_INVALID_ARG;
    rok_batch_tuning t;
    memset(&t, 0, sizeof(t));
    rok_status r;
    for (int g = 0; g < kGroups; ++g) {
        float best = -1.0f;
        for (int s = 0; s < kNumShapes; ++s) {
            t.stencil_ms[g][s] = -1.0f;
            if (!b->has_group[g]) continue;
            float ms = 0.0f;
            r = time_ms(b, 3, [&] { return stencil(b, io_plain(b, y, b->t0), g, s); }, &ms);
            if (r != ROK_OK) return r;
            t.stencil_ms[g][s] = ms;
            if (best < 0.0f || ms < best) {
                best = ms;
                t.tile[g] = s;
            }
        }
    }
    // vector passes on scratch data: one Arnoldi column (active flags set),
    // zero partials (h = 0)
    CU(launch_begin_batch(b->st, b->d_h, b->gamma_rok, 1, b->count, b->stream));
    CU(cudaMemsetAsync(b->pA, 0, 2 * (size_t)b->nchunks * sizeof(double), b->stream));
    const BSeg sg = seg(b);
    float best_m = -1.0f, best_v = -1.0f;
    for (int q = 0; q < 4; ++q) {
        const int c = kCpcCandidates[q];
        float ms = 0.0f;
        r = time_ms(b, 3, [&] {
            return b->bops->mgs(b->t0, b->V, b->total, 1, 0, b->pA, b->pB, sg, c, b->stream) == cudaSuccess
                       ? ROK_OK : ROK_ERR_CUDA; }, &ms);
        if (r != ROK_OK) return r;
        t.mgs_ms[q] = ms;
        if (best_m < 0.0f || ms < best_m) { best_m = ms; t.chunks_per_cta = c; }
        r = time_ms(b, 3, [&] {
            return b->bops->stage_vec(b->w, b->F[0], b->V, b->total, 0, sg, c, b->stream) == cudaSuccess
                       ? ROK_OK : ROK_ERR_CUDA; }, &ms);
        if (r != ROK_OK) return r;
        t.vec_ms[q] = ms;
        if (best_v < 0.0f || ms < best_v) { best_v = ms; t.vec_chunks_per_cta = c; }
    }
    CU(launch_clear_status(b->st, b->count, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    for (int g = 0; g < kGroups; ++g) b->tile[g] = t.tile[g];
    b->cpc = t.chunks_per_cta;
    b->vcpc = t.vec_chunks_per_cta;
    clear_graphs(b);
    if (out) *out = t;
    return ROK_OK;
}

rok_status rok_batch_set_tuning(rok_batch *b, const rok_batch_tuning *t)
{
    if (!b || !t) return ROK_ERR_INVALID_ARG;
    for (int g = 0; g < kGroups; ++g)
        if (t->tile[g] < 0 || t->tile[g] >= kNumShapes) return ROK_ERR_INVALID_ARG;
    if (!valid_cpc(t->chunks_per_cta) || !valid_cpc(t->vec_chunks_per_cta)) return ROK_ERR_INVALID_ARG;
    for (int g = 0; g < kGroups; ++g) b->tile[g] = t->tile[g];
    b->cpc = t->chunks_per_cta;
    b->vcpc = t->vec_chunks_per_cta;
    clear_graphs(b);
    return ROK_OK;
}

rok_status rok_batch_get_tuning(const rok_batch *b, rok_batch_tuning *t)
{
    if (!b || !t) return ROK_ERR_INVALID_ARG;
    memset(t, 0, sizeof(*t));
    for (int g = 0; g < kGroups; ++g) t->tile[g] = b->tile[g];
    t->chunks_per_cta = b->cpc;
    t->vec_chunks_per_cta = b->vcpc;
    return ROK_OK;
}

rok_status rok_batch_set_graph(rok_batch *b, int enable)
{
    if (!b) return ROK_ERR_INVALID_ARG;
    b->use_graph = enable != 0;
    return ROK_OK;
}

rok_status rok_batch_get_launches(rok_batch *b, long long *launches, int reset)
{
    if (!b || !launches) return ROK_ERR_INVALID_ARG;
    *launches = b->launches;
    if (reset) b->launches = 0;
    return ROK_OK;
}

}  // extern "C"
