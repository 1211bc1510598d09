// Host side of the C ABI declared in include/lbm.h: parameter validation and
// derivation, device buffers, kernel sequencing (with a CUDA graph for long
// runs), diagnostics, state exchange and checkpoints.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lbm.h"
#include "lbm_internal.h"

using namespace wblbm;

namespace {

constexpr double CS2 = 1.0 / 3.0;
constexpr int GRAPH_STEPS = 32;  // steps per captured graph (even: ping-pong)

// Lattice velocities, used on the host only by lbm_debug_poke to find where
// a population is stored.  D2Q9 in the order of Eq. eq:ci; D3Q19: rest,
// faces (+x, -x, +y, -y, +z, -z), edges (xy, xz, yz planes).
constexpr int HC2[9][3] = {{0, 0, 0},  {0, -1, 0}, {1, 0, 0},  {0, 1, 0}, {-1, 0, 0},
                           {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
constexpr int HC3[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                            {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {1, -1, 0}, {-1, 1, 0},
                            {-1, -1, 0}, {1, 0, 1}, {1, 0, -1},  {-1, 0, 1}, {-1, 0, -1},
                            {0, 1, 1},  {0, 1, -1}, {0, -1, 1},  {0, -1, -1}};

}  // namespace

struct lbm_ctx {
    lbm_grid grid;
    int lattice;
    lbm_params prm;
    double kappa, beta, tau_f, alpha;
    int Q, D;
    int nf;      // f arrays: Q, plus the low word of the rest population in FP32
    long long N;
    size_t esz;  // bytes per stored population value
    int codec;   // offset storage: OFFSET_F16 / OFFSET_BF16, else -1
    size_t fbytes, gbytes;  // bytes of one f / g state buffer
    float *scw;  // offset storage: target scales [2], then 2 words of scratch
    float *eqs;  // FP32 equilibrium shift {buffer 0, buffer 1, target, next target} (device)
    int own_state;  // f[], g[] and S were allocated here (not by the caller)
    int recentre;  // lbm_diagnostics moves the FP32 equilibrium shift (not under an adjoint)
    int nsm;
    void *f[2], *g[2], *S;
    int cur;     // f[cur], g[cur] hold the current state
    double *aux;         // N doubles (initial chemical potential)
    void *phiw;          // D3Q19: phi field written by the first pass of a step
    double *stage;       // (3 + D) N doubles, host moment staging (lazy)
    DiagPartial *partials;
    DiagPartial *dres;   // device: [0] on-demand diagnostics, [1] last fused
    DiagPartial *hres;   // pinned host copy of dres
    int npart;
    cudaStream_t stream;
    cudaStream_t cap;    // private stream used for graph capture
    cudaEvent_t diag_ev; // recorded after a fused diagnostics copy
    cudaEvent_t up_ev;   // recorded after lbm_init_phi's upload from host memory
    int diag_pending;
    long long last_diag_step;
    int has_last_diag;
    int device;
    long long step;
    int initialized;
    int err;             // sticky error (returned once, then cleared)
    LaunchShape shape;
    StepParams<double> pd;
    StepParams<float> pf;
    cudaGraphExec_t gexec;
    int gexec_valid;
};

namespace {

int fail_cuda(lbm_ctx *c, cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    if (c) c->err = LBM_ERR_CUDA;
    return LBM_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_);     \
    } while (0)

int take_err(lbm_ctx *c)
{
    int e = c->err;
    if (e != LBM_ERR_CUDA) c->err = LBM_OK;  // CUDA errors stay: the context is unusable
    return e;
}

int validate(const lbm_grid *g, int lattice, const lbm_params *p)
{
    return validate_problem(g, lattice, p);
}

template <typename T>
void fill_params(StepParams<T> &P, const lbm_ctx *c)
{
    const Derived d = {c->kappa, c->beta, c->tau_f, c->alpha};
    fill_step_params(P, c->grid, c->prm, d);
}

const void *params_ptr(const lbm_ctx *c)
{
    return c->prm.precision == LBM_FP64 ? (const void *)&c->pd : (const void *)&c->pf;
}

int set_device(lbm_ctx *ctx)
{
    CK(cudaSetDevice(ctx->device));
    return LBM_OK;
}

// one pass over the current state
int run_pass(lbm_ctx *ctx, int pass, cudaStream_t st, double *o_phi, double *o_p, double *o_u,
             double *o_mu)
{
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.f_src = ctx->f[ctx->cur];
    a.g_src = ctx->g[ctx->cur];
    a.f_dst = ctx->f[ctx->cur ^ 1];
    a.g_dst = ctx->g[ctx->cur ^ 1];
    a.S = ctx->S;
    a.S_out = ctx->S;
    a.out_phi = o_phi;
    a.out_p = o_p;
    a.out_u = o_u;
    a.out_mu = o_mu;
    a.partials = ctx->partials;
    a.eqs_src = ctx->eqs + ctx->cur;
    a.eqs_dst = ctx->eqs + (ctx->cur ^ 1);
    a.eqs_target = ctx->eqs + 2;
    a.flip = ctx->cur;
    if (ctx->codec >= 0)
        CK(d3q19_off_pass(ctx->codec, pass, &ctx->pf, a, ctx->shape, ctx->phiw, ctx->scw, st));
    else if (ctx->lattice == LBM_D3Q19)
        CK(d3q19_pass(ctx->prm.precision, pass, params_ptr(ctx), a, ctx->shape, ctx->phiw, st));
    else
        CK(d2q9_pass(ctx->prm.precision, pass, params_ptr(ctx), a, ctx->shape, st));
    return LBM_OK;
}

// D2Q9 pass over a state held in a snapshot (f | g | S contiguous, the
// adjoint's layout) instead of the context's buffers; a time step writes the
// next state into `next` (same layout).  The equilibrium shift stays at the
// context's (constant while an adjoint recorder is attached).
// moments (PASS_MACROS_T, D2Q9): phi, mu, p (N each) and u (2N) in the
// storage type, back to back from `moments`
int run_pass_snap(lbm_ctx *ctx, int pass, const char *snap, char *next, void *moments)
{
    const size_t fb = ctx->fbytes, gb = ctx->gbytes;
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.f_src = snap;
    a.g_src = snap + fb;
    a.S = (void *)(snap + fb + gb);
    if (next) {
        a.f_dst = next;
        a.g_dst = next + fb;
        a.S_out = next + fb + gb;
    }
    if (moments) {
        const size_t nb = (size_t)ctx->N * ctx->esz;
        char *m = static_cast<char *>(moments);
        a.mt_phi = m;
        a.mt_mu = m + nb;
        a.mt_p = m + 2 * nb;
        a.mt_u = m + 3 * nb;
    }
    a.partials = ctx->partials;
    a.eqs_src = ctx->eqs + ctx->cur;
    a.eqs_dst = ctx->eqs + (ctx->cur ^ 1);
    a.eqs_target = ctx->eqs + ctx->cur;
    CK(d2q9_pass(ctx->prm.precision, pass, params_ptr(ctx), a, ctx->shape, ctx->stream));
    return LBM_OK;
}

// offset storage: new target scales from the current state
int refresh_scales(lbm_ctx *ctx, cudaStream_t st)
{
    if (ctx->codec < 0) return LBM_OK;
    CK(offset_refresh(ctx->codec, ctx->N, ctx->Q, ctx->f[ctx->cur], ctx->g[ctx->cur],
                      (unsigned *)(ctx->scw + 2), ctx->scw, ctx->nsm, st));
    return LBM_OK;
}

const float OFFSET_INITIAL_SCALES[2] = {OFFSET_SCALE_FLOOR, OFFSET_SCALE_FLOOR};

// a new state (initial condition, set_state, load): equilibrium shift `a`
// for the state in buffer 0 and for new writes
int set_eq_shift(lbm_ctx *ctx, float a)
{
    if (a == 0.0f) {
        CK(cudaMemsetAsync(ctx->eqs, 0, 4 * sizeof(float), ctx->stream));
        return LBM_OK;
    }
    float v[4] = {a, a, a, a};
    CK(cudaMemcpyAsync(ctx->eqs, v, sizeof v, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // v is on the stack
    return LBM_OK;
}

// offset storage: targets back to the initial scales (before a new state is written)
int reset_scales(lbm_ctx *ctx)
{
    if (ctx->codec < 0) return LBM_OK;
    CK(cudaMemcpyAsync(ctx->scw, OFFSET_INITIAL_SCALES, sizeof OFFSET_INITIAL_SCALES,
                       cudaMemcpyHostToDevice, ctx->stream));
    return LBM_OK;
}

// A graph of GRAPH_STEPS plain steps starting from cur = 0 (ends at cur = 0).
int ensure_graph(lbm_ctx *ctx)
{
    if (ctx->gexec_valid) return LBM_OK;
    const int saved = ctx->cur;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    ctx->cur = 0;
    for (int k = 0; k < GRAPH_STEPS && rc == LBM_OK; ++k) {
        rc = run_pass(ctx, PASS_STATE, ctx->cap, nullptr, nullptr, nullptr, nullptr);
        ctx->cur ^= 1;
    }
    ctx->cur = saved;
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &graph);
    if (rc != LBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(e);
    e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    ctx->gexec_valid = 1;
    return LBM_OK;
}

void poll_diag(lbm_ctx *ctx, bool wait)
{
    if (!ctx->diag_pending) return;
    cudaError_t e = wait ? cudaEventSynchronize(ctx->diag_ev) : cudaEventQuery(ctx->diag_ev);
    if (e == cudaErrorNotReady) return;
    if (e != cudaSuccess) {
        ctx->err = LBM_ERR_CUDA;
        return;
    }
    ctx->diag_pending = 0;
    if (ctx->hres[1].nonfinite != 0.0 && ctx->err == LBM_OK) ctx->err = LBM_ERR_NONFINITE;
}

void fill_diag(const DiagPartial &r, long long step, lbm_diag *out)
{
    out->sum_phi = r.sum_phi;
    out->kinetic_energy = r.E;
    out->u_max = sqrt(r.u2max);
    out->mu_min = r.mu_min;
    out->mu_max = r.mu_max;
    out->budget = r.budget;
    out->step = step;
    out->nonfinite = r.nonfinite != 0.0;
}

void free_all(lbm_ctx *c)
{
    if (c->gexec_valid) cudaGraphExecDestroy(c->gexec);
    if (c->own_state) {
        void *st[] = {c->f[0], c->f[1], c->g[0], c->g[1], c->S};
        for (void *p : st)
            if (p) cudaFree(p);
    }
    void *dev[] = {c->aux, c->phiw, c->stage, c->partials, c->dres, c->scw, c->eqs};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (c->hres) cudaFreeHost(c->hres);
    if (c->diag_ev) cudaEventDestroy(c->diag_ev);
    if (c->up_ev) cudaEventDestroy(c->up_ev);
    if (c->cap) cudaStreamDestroy(c->cap);
}

}  // namespace

extern "C" {

int lbm_params_default(lbm_params *out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    memset(out, 0, sizeof *out);
    out->W = 4.0;
    out->M = 0.1;
    out->alpha = 1.0;
    out->sigma = 1e-3;
    out->phi_l = 1.0;
    out->phi_v = 0.0;
    out->rho_l = 10.0;
    out->rho_v = 1.0;
    out->nu_l = 0.1;
    out->nu_v = 0.1;
    out->tau_f = 0.0;
    out->precision = LBM_FP32;
    out->diag_every = 0;
    return LBM_OK;
}

}  // extern "C"

namespace {

// bytes of one f buffer, one g buffer and S_prev of a valid problem
void state_sizes(const lbm_grid *grid, int lattice, const lbm_params *params, size_t *fb,
                 size_t *gb, size_t *sb)
{
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    const int Q = lattice == LBM_D3Q19 ? 19 : 9, D = lattice == LBM_D3Q19 ? 3 : 2;
    if (params->precision == LBM_FP32_F16OFF || params->precision == LBM_FP32_BF16OFF) {
        const OffsetLayout L = offset_layout(N, Q, D);
        *fb = L.fbytes;
        *gb = L.gbytes;
        *sb = (size_t)N * 4;
        return;
    }
    const size_t esz = params->precision == LBM_FP64 ? 8 : 4;
    const int nf = Q + (params->precision == LBM_FP32 ? 1 : 0);
    *fb = (size_t)nf * N * esz;
    *gb = (size_t)Q * N * esz;
    *sb = (size_t)N * esz;
}

int create_impl(const lbm_grid *grid, int lattice, const lbm_params *params, void *cuda_stream,
                void *const *bufs, lbm_ctx **out);

}  // namespace

extern "C" {

int lbm_create(const lbm_grid *grid, int lattice, const lbm_params *params, void *cuda_stream,
               lbm_ctx **out)
{
    return create_impl(grid, lattice, params, cuda_stream, nullptr, out);
}

int lbm_state_bytes(const lbm_grid *grid, int lattice, const lbm_params *params, size_t out[3])
{
    if (!out) return LBM_ERR_INVALID_ARG;
    int rc = validate(grid, lattice, params);
    if (rc != LBM_OK) return rc;
    state_sizes(grid, lattice, params, &out[0], &out[1], &out[2]);
    return LBM_OK;
}

int lbm_create_with_buffers(const lbm_grid *grid, int lattice, const lbm_params *params,
                            void *cuda_stream, void *const buffers[5], lbm_ctx **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!buffers) return LBM_ERR_INVALID_ARG;
    for (int k = 0; k < 5; ++k)
        if (!buffers[k] || ((uintptr_t)buffers[k] & 255u)) return LBM_ERR_INVALID_ARG;
    return create_impl(grid, lattice, params, cuda_stream, buffers, out);
}

}  // extern "C"

namespace {

int create_impl(const lbm_grid *grid, int lattice, const lbm_params *params, void *cuda_stream,
                void *const *bufs, lbm_ctx **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate(grid, lattice, params);
    if (rc != LBM_OK) return rc;

    lbm_ctx *ctx = (lbm_ctx *)calloc(1, sizeof(lbm_ctx));
    if (!ctx) return LBM_ERR_OOM;
    ctx->grid = *grid;
    ctx->lattice = lattice;
    ctx->prm = *params;
    ctx->Q = lattice == LBM_D3Q19 ? 19 : 9;
    ctx->D = lattice == LBM_D3Q19 ? 3 : 2;
    ctx->nf = ctx->Q + (params->precision == LBM_FP32 ? 1 : 0);
    ctx->N = (long long)grid->nx * grid->ny * grid->nz;
    ctx->esz = params->precision == LBM_FP64 ? 8 : 4;
    ctx->codec = params->precision == LBM_FP32_F16OFF    ? OFFSET_F16
                 : params->precision == LBM_FP32_BF16OFF ? OFFSET_BF16
                                                         : -1;
    if (ctx->codec >= 0) {
        const OffsetLayout L = offset_layout(ctx->N, ctx->Q, ctx->D);
        ctx->nf = ctx->Q;
        ctx->esz = 2;
        ctx->fbytes = L.fbytes;
        ctx->gbytes = L.gbytes;
    } else {
        ctx->fbytes = (size_t)ctx->nf * ctx->N * ctx->esz;
        ctx->gbytes = (size_t)ctx->Q * ctx->N * ctx->esz;
    }
    // S_prev and the D3Q19 phi work field: FP64 in the FP64 form, else FP32
    const size_t ssz = params->precision == LBM_FP64 ? 8 : 4;
    ctx->stream = (cudaStream_t)cuda_stream;

    const Derived dp = derive_params(*params);
    ctx->kappa = dp.kappa;
    ctx->beta = dp.beta;
    ctx->tau_f = dp.tau_f;
    ctx->alpha = dp.alpha;
    fill_params(ctx->pd, ctx);
    fill_params(ctx->pf, ctx);

    cudaError_t e = cudaGetDevice(&ctx->device);
    int nsm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        free(ctx);
        return LBM_ERR_CUDA;
    }
    ctx->nsm = nsm;
    if (lattice == LBM_D3Q19) {
        const int occ = ctx->codec >= 0 ? d3q19_off_ctas_per_sm(ctx->codec)
                                        : d3q19_ctas_per_sm(params->precision);
        ctx->shape = d3q19_shape(grid->nx, grid->ny, grid->nz, nsm, occ);
    } else {
        ctx->shape = d2q9_shape(grid->nx, grid->ny, nsm);
    }
    ctx->npart = ctx->shape.nblocks;
    const size_t N = (size_t)ctx->N, Q = (size_t)ctx->Q;
    bool oom = false;
    auto dalloc = [&](void **p, size_t bytes) {
        if (oom) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            *p = nullptr;
            oom = true;
        }
    };
    (void)Q;
    if (bufs) {  // the caller's memory, used in place
        ctx->f[0] = bufs[0];
        ctx->f[1] = bufs[1];
        ctx->g[0] = bufs[2];
        ctx->g[1] = bufs[3];
        ctx->S = bufs[4];
        ctx->own_state = 0;
    } else {
        ctx->own_state = 1;
        dalloc(&ctx->f[0], ctx->fbytes);
        dalloc(&ctx->f[1], ctx->fbytes);
        dalloc(&ctx->g[0], ctx->gbytes);
        dalloc(&ctx->g[1], ctx->gbytes);
        dalloc(&ctx->S, N * ssz);
    }
    dalloc((void **)&ctx->aux, N * sizeof(double));
    if (lattice == LBM_D3Q19) dalloc(&ctx->phiw, N * ssz);
    if (ctx->codec >= 0) dalloc((void **)&ctx->scw, 4 * sizeof(float));
    dalloc((void **)&ctx->eqs, 4 * sizeof(float));
    ctx->recentre = 1;
    dalloc((void **)&ctx->partials, (size_t)ctx->npart * sizeof(DiagPartial));
    dalloc((void **)&ctx->dres, 2 * sizeof(DiagPartial));
    if (!oom && cudaMallocHost((void **)&ctx->hres, 2 * sizeof(DiagPartial)) != cudaSuccess)
        oom = true;
    if (!oom && (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
                 cudaEventCreateWithFlags(&ctx->diag_ev, cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&ctx->up_ev, cudaEventDisableTiming) != cudaSuccess))
        oom = true;
    if (oom) {
        cudaGetLastError();  // clear the allocation error
        free_all(ctx);
        free(ctx);
        return LBM_ERR_OOM;
    }
    memset(ctx->hres, 0, 2 * sizeof(DiagPartial));
    if ((ctx->codec >= 0 && reset_scales(ctx) != LBM_OK) || set_eq_shift(ctx, 0.0f) != LBM_OK ||
        (lattice == LBM_D2Q9 && d2q9_prepare() != cudaSuccess) ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        free_all(ctx);
        free(ctx);
        return LBM_ERR_CUDA;
    }
    *out = ctx;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_init_phi(lbm_ctx *ctx, const double *phi, int on_device)
{
    if (!ctx || !phi) return LBM_ERR_INVALID_ARG;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->N;
    const double *src = phi;
    if (!on_device) {
        // staged through the other f buffer: the initial condition writes
        // buffer 0 only, and an f buffer holds at least N doubles (>= 9 N
        // 4-byte or 19 N 2-byte values, 256-byte aligned)
        double *stage = static_cast<double *>(ctx->f[1]);
        CK(cudaMemcpyAsync(stage, phi, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaEventRecord(ctx->up_ev, ctx->stream));
        src = stage;
    }
    if (int rc = set_eq_shift(ctx, 0.0f)) return rc;
    cudaError_t e = cudaSuccess;
    if (ctx->codec >= 0) {
        e = cudaMemcpyAsync(ctx->scw, OFFSET_INITIAL_SCALES, sizeof OFFSET_INITIAL_SCALES,
                            cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = d3q19_off_init(ctx->codec, &ctx->pd, &ctx->pf, src, ctx->aux, ctx->f[0],
                               ctx->g[0], ctx->S, OFFSET_INITIAL_SCALES, ctx->stream);
    } else if (ctx->lattice == LBM_D3Q19) {
        e = d3q19_init(ctx->prm.precision, &ctx->pd, src, ctx->aux, ctx->f[0], ctx->g[0],
                       ctx->S, ctx->stream);
    } else {
        e = d2q9_init(ctx->prm.precision, &ctx->pd, src, ctx->aux, ctx->f[0], ctx->g[0],
                      ctx->S, ctx->stream);
    }
    // a host array is read until the upload completes: return after it
    if (e == cudaSuccess && !on_device) e = cudaEventSynchronize(ctx->up_ev);
    CK(e);
    ctx->cur = 0;
    ctx->step = 0;
    ctx->initialized = 1;
    ctx->has_last_diag = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx *ctx, int n)
{
    if (!ctx || n < 0) return LBM_ERR_INVALID_ARG;
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (int rc = set_device(ctx)) return rc;
    poll_diag(ctx, false);
    if (ctx->err) return take_err(ctx);
    const int de = ctx->prm.diag_every;
    int left = n;
    while (left > 0) {
        if (de > 0 && ctx->step % de == 0) {
            // fused diagnostics step: reduce the partials, copy the record
            int rc = run_pass(ctx, PASS_STATE | PASS_DIAG, ctx->stream, nullptr, nullptr,
                              nullptr, nullptr);
            if (rc) return rc;
            CK(diag_reduce(ctx->partials, ctx->npart, ctx->dres + 1, ctx->stream));
            CK(cudaMemcpyAsync(ctx->hres + 1, ctx->dres + 1, sizeof(DiagPartial),
                               cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaEventRecord(ctx->diag_ev, ctx->stream));
            ctx->diag_pending = 1;
            ctx->has_last_diag = 1;
            ctx->last_diag_step = ctx->step;
            ctx->cur ^= 1;
            ctx->step += 1;
            left -= 1;
            if (int rc2 = refresh_scales(ctx, ctx->stream)) return rc2;
            continue;
        }
        // plain steps up to the next diagnostics step
        long long run = left;
        if (de > 0) {
            const long long to_diag = de - ctx->step % de;
            if (to_diag < run) run = to_diag;
        }
        if (run >= GRAPH_STEPS) {
            if (ctx->cur == 1) {
                int rc = run_pass(ctx, PASS_STATE, ctx->stream, nullptr, nullptr, nullptr, nullptr);
                if (rc) return rc;
                ctx->cur = 0;
                ctx->step += 1;
                left -= 1;
                run -= 1;
            }
            if (run >= GRAPH_STEPS) {
                if (int rc = ensure_graph(ctx)) return rc;
                const long long reps = run / GRAPH_STEPS;
                for (long long r = 0; r < reps; ++r) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
                ctx->step += reps * GRAPH_STEPS;
                left -= (int)(reps * GRAPH_STEPS);
                run -= reps * GRAPH_STEPS;
            }
        }
        for (long long k = 0; k < run; ++k) {
            int rc = run_pass(ctx, PASS_STATE, ctx->stream, nullptr, nullptr, nullptr, nullptr);
            if (rc) return rc;
            ctx->cur ^= 1;
            ctx->step += 1;
            left -= 1;
        }
    }
    return LBM_OK;
}

int lbm_moments(lbm_ctx *ctx, double *phi, double *p, double *u, double *mu, int on_device)
{
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->N;
    if (on_device) return run_pass(ctx, PASS_MACROS, ctx->stream, phi, p, u, mu);
    // Host arrays in pinned (page-locked, device-mapped) memory: the pass
    // writes them directly through their device addresses, with no staging
    // buffer and no separate copies; it returns once they are written.
    {
        double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
        double *const host[4] = {phi, p, u, mu};
        bool mapped = true;
        for (int k = 0; k < 4 && mapped; ++k) {
            if (!host[k]) continue;
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, host[k]) != cudaSuccess ||
                at.type != cudaMemoryTypeHost || !at.devicePointer) {
                cudaGetLastError();
                mapped = false;
            } else {
                dev[k] = static_cast<double *>(at.devicePointer);
            }
        }
        if (mapped) {
            int rc = run_pass(ctx, PASS_MACROS, ctx->stream, dev[0], dev[1], dev[2], dev[3]);
            if (rc) return rc;
            CK(cudaStreamSynchronize(ctx->stream));
            return LBM_OK;
        }
    }
    if (!ctx->stage) CK(cudaMalloc((void **)&ctx->stage, (3 + ctx->D) * N * sizeof(double)));
    double *s_phi = ctx->stage, *s_p = s_phi + N, *s_mu = s_p + N, *s_u = s_mu + N;
    int rc = run_pass(ctx, PASS_MACROS, ctx->stream, phi ? s_phi : nullptr, p ? s_p : nullptr,
                      u ? s_u : nullptr, mu ? s_mu : nullptr);
    if (rc) return rc;
    const size_t b = N * sizeof(double);
    if (phi) CK(cudaMemcpyAsync(phi, s_phi, b, cudaMemcpyDeviceToHost, ctx->stream));
    if (p) CK(cudaMemcpyAsync(p, s_p, b, cudaMemcpyDeviceToHost, ctx->stream));
    if (mu) CK(cudaMemcpyAsync(mu, s_mu, b, cudaMemcpyDeviceToHost, ctx->stream));
    if (u) CK(cudaMemcpyAsync(u, s_u, ctx->D * b, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_diagnostics(lbm_ctx *ctx, lbm_diag *out)
{
    if (!ctx || !out) return LBM_ERR_INVALID_ARG;
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    int rc = run_pass(ctx, PASS_DIAG, ctx->stream, nullptr, nullptr, nullptr, nullptr);
    if (rc) return rc;
    if ((rc = refresh_scales(ctx, ctx->stream))) return rc;
    CK(diag_reduce(ctx->partials, ctx->npart, ctx->dres, ctx->stream));
    if (ctx->prm.precision == LBM_FP32 && ctx->recentre)
        CK(eq_recentre(ctx->dres, ctx->alpha, ctx->eqs + 2, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hres, ctx->dres, sizeof(DiagPartial), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    fill_diag(ctx->hres[0], ctx->step, out);
    return LBM_OK;
}

int lbm_last_diagnostics(lbm_ctx *ctx, lbm_diag *out)
{
    if (!ctx || !out) return LBM_ERR_INVALID_ARG;
    if (!ctx->has_last_diag) return LBM_ERR_STATE;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    // a fresh device-to-host read of the record, ordered after all queued work
    CK(cudaMemcpyAsync(ctx->hres + 1, ctx->dres + 1, sizeof(DiagPartial), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->diag_pending = 0;
    if (ctx->hres[1].nonfinite != 0.0 && ctx->err == LBM_OK) ctx->err = LBM_ERR_NONFINITE;
    fill_diag(ctx->hres[1], ctx->last_diag_step, out);
    return LBM_OK;
}

int lbm_get_state(lbm_ctx *ctx, double *f, double *g, double *S_prev, int on_device)
{
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->N, QN = (size_t)ctx->Q * N;
    auto get = [&](double *fo, double *go, double *so) {
        if (ctx->codec >= 0)
            return d3q19_off_get_state(ctx->codec, &ctx->pf, ctx->f[ctx->cur], ctx->g[ctx->cur],
                                       ctx->S, fo, go, so, ctx->stream);
        return ctx->lattice == LBM_D3Q19
                   ? d3q19_get_state(ctx->prm.precision, &ctx->pd, ctx->f[ctx->cur],
                                     ctx->g[ctx->cur], ctx->S, ctx->eqs + ctx->cur, fo, go, so,
                                     ctx->stream)
                   : d2q9_get_state(ctx->prm.precision, ctx->grid.nx, ctx->grid.ny,
                                    ctx->f[ctx->cur], ctx->g[ctx->cur], ctx->S,
                                    ctx->eqs + ctx->cur, fo, go, so, ctx->stream);
    };
    if (on_device) {
        CK(get(f, g, S_prev));
        return LBM_OK;
    }
    double *tmp = nullptr;
    CK(cudaMalloc((void **)&tmp, (2 * QN + N) * sizeof(double)));
    cudaError_t e = get(tmp, tmp + QN, tmp + 2 * QN);
    if (e == cudaSuccess && f)
        e = cudaMemcpyAsync(f, tmp, QN * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && g)
        e = cudaMemcpyAsync(g, tmp + QN, QN * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && S_prev)
        e = cudaMemcpyAsync(S_prev, tmp + 2 * QN, N * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    CK(e);
    return LBM_OK;
}

int lbm_set_state(lbm_ctx *ctx, const double *f, const double *g, const double *S_prev,
                  long long step, int on_device)
{
    if (!ctx || !f || !g || !S_prev || step < 0) return LBM_ERR_INVALID_ARG;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    const size_t N = (size_t)ctx->N, QN = (size_t)ctx->Q * N;
    const double *fi = f, *gi = g, *si = S_prev;
    double *tmp = nullptr;
    if (!on_device) {
        CK(cudaMalloc((void **)&tmp, (2 * QN + N) * sizeof(double)));
        cudaError_t e = cudaMemcpyAsync(tmp, f, QN * sizeof(double), cudaMemcpyHostToDevice,
                                        ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp + QN, g, QN * sizeof(double), cudaMemcpyHostToDevice,
                                ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp + 2 * QN, S_prev, N * sizeof(double),
                                cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return fail_cuda(ctx, e);
        }
        fi = tmp;
        gi = tmp + QN;
        si = tmp + 2 * QN;
    }
    cudaError_t e = cudaSuccess;
    if (int rc = set_eq_shift(ctx, 0.0f)) {
        if (tmp) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(tmp);
        }
        return rc;
    }
    if (ctx->codec >= 0) {
        e = cudaMemcpyAsync(ctx->scw, OFFSET_INITIAL_SCALES, sizeof OFFSET_INITIAL_SCALES,
                            cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = d3q19_off_set_state(ctx->codec, &ctx->pf, ctx->f[0], ctx->g[0], ctx->S, fi, gi,
                                    si, OFFSET_INITIAL_SCALES, ctx->stream);
    } else if (ctx->lattice == LBM_D3Q19) {
        e = d3q19_set_state(ctx->prm.precision, &ctx->pd, ctx->f[0], ctx->g[0], ctx->S, fi, gi,
                            si, ctx->stream);
    } else {
        e = d2q9_set_state(ctx->prm.precision, ctx->grid.nx, ctx->grid.ny, ctx->f[0], ctx->g[0],
                           ctx->S, fi, gi, si, ctx->stream);
    }
    if (tmp) {
        cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
        cudaFree(tmp);
        if (e == cudaSuccess) e = e2;
    }
    CK(e);
    ctx->cur = 0;
    ctx->step = step;
    ctx->initialized = 1;
    ctx->has_last_diag = 0;
    return LBM_OK;
}

namespace {
// bytes of one S_prev value
size_t state_S_bytes(const lbm_ctx *ctx) { return ctx->prm.precision == LBM_FP64 ? 8 : 4; }

struct SaveHeader {
    char magic[8];
    int version, lattice, precision, Q;
    int nx, ny, nz;
    float eq_shift;  // FP32: equilibrium shift of the saved populations
    long long step;
};
}  // namespace

int lbm_save(lbm_ctx *ctx, void *buf, size_t *bytes)
{
    if (!ctx || !bytes) return LBM_ERR_INVALID_ARG;
    const size_t N = (size_t)ctx->N, popf = ctx->fbytes, pop = ctx->gbytes, ssz = state_S_bytes(ctx);
    const size_t need = sizeof(SaveHeader) + popf + pop + N * ssz;
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (*bytes < need) return LBM_ERR_INVALID_ARG;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    SaveHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "WBLBMCK", 8);
    h.version = 2;
    CK(cudaMemcpyAsync(&h.eq_shift, ctx->eqs + ctx->cur, sizeof(float), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    h.lattice = ctx->lattice;
    h.precision = ctx->prm.precision;
    h.Q = ctx->Q;
    h.nx = ctx->grid.nx;
    h.ny = ctx->grid.ny;
    h.nz = ctx->grid.nz;
    h.step = ctx->step;
    char *b = (char *)buf;
    memcpy(b, &h, sizeof h);
    b += sizeof h;
    CK(cudaMemcpyAsync(b, ctx->f[ctx->cur], popf, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b + popf, ctx->g[ctx->cur], pop, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b + popf + pop, ctx->S, N * ssz, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *bytes = need;
    return LBM_OK;
}

int lbm_load(lbm_ctx *ctx, const void *buf, size_t bytes)
{
    if (!ctx || !buf) return LBM_ERR_INVALID_ARG;
    const size_t N = (size_t)ctx->N, popf = ctx->fbytes, pop = ctx->gbytes, ssz = state_S_bytes(ctx);
    const size_t need = sizeof(SaveHeader) + popf + pop + N * ssz;
    if (bytes < need) return LBM_ERR_INVALID_ARG;
    SaveHeader h;
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "WBLBMCK", 8) != 0 || h.version != 2 || h.lattice != ctx->lattice ||
        h.precision != ctx->prm.precision || h.Q != ctx->Q || h.nx != ctx->grid.nx ||
        h.ny != ctx->grid.ny || h.nz != ctx->grid.nz || h.step < 0)
        return LBM_ERR_INVALID_ARG;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    const char *b = (const char *)buf + sizeof h;
    CK(cudaMemcpyAsync(ctx->f[0], b, popf, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->g[0], b + popf, pop, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->S, b + popf + pop, N * ssz, cudaMemcpyHostToDevice,
                       ctx->stream));
    if (int rc = set_eq_shift(ctx, h.eq_shift)) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->cur = 0;
    ctx->step = h.step;
    ctx->initialized = 1;
    ctx->has_last_diag = 0;
    return LBM_OK;
}

int lbm_sync(lbm_ctx *ctx)
{
    if (!ctx) return LBM_ERR_INVALID_ARG;
    if (int rc = set_device(ctx)) return rc;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    poll_diag(ctx, true);
    return take_err(ctx);
}

long long lbm_time(const lbm_ctx *ctx) { return ctx ? ctx->step : -1; }

int lbm_derived(const lbm_ctx *ctx, double out[4])
{
    if (!ctx || !out) return LBM_ERR_INVALID_ARG;
    out[0] = ctx->kappa;
    out[1] = ctx->beta;
    out[2] = ctx->tau_f;
    out[3] = ctx->alpha;
    return LBM_OK;
}

int lbm_debug_poke(lbm_ctx *ctx, int field, int i, long long n, double value)
{
    if (!ctx || field < 0 || field > 1 || i < 0 || i >= ctx->Q || n < 0 || n >= ctx->N)
        return LBM_ERR_INVALID_ARG;
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (int rc = set_device(ctx)) return rc;
    if (ctx->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    // the paper's f_i(x) is stored at x - c_i (pull layout)
    const int nx = ctx->grid.nx, ny = ctx->grid.ny, nz = ctx->grid.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    const int *c = ctx->lattice == LBM_D3Q19 ? HC3[i] : HC2[i];
    const int xs = ((x - c[0]) % nx + nx) % nx, ys = ((y - c[1]) % ny + ny) % ny,
              zs = ((z - c[2]) % nz + nz) % nz;
    const size_t node = ((size_t)zs * ny + ys) * nx + xs;
    if (ctx->codec >= 0) {
        CK(d3q19_off_poke(ctx->codec, &ctx->pf, ctx->f[ctx->cur], ctx->g[ctx->cur], field, i, node,
                          value, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return LBM_OK;
    }
    const size_t m = (size_t)i * ctx->N + node;
    char *base = (char *)(field == 0 ? ctx->f[ctx->cur] : ctx->g[ctx->cur]);
    if (ctx->esz == 8) {
        CK(cudaMemcpyAsync(base + m * 8, &value, 8, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        static const float zero = 0.0f;
        double shifted = value;
        if (field == 0) {  // stored f is shifted by the equilibrium shift of its buffer
            float a = 0.0f;
            CK(cudaMemcpyAsync(&a, ctx->eqs + ctx->cur, sizeof a, cudaMemcpyDeviceToHost,
                               ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            const double w0 = ctx->lattice == LBM_D3Q19 ? 1.0 / 3.0 : 4.0 / 9.0;
            const double wi = ctx->lattice == LBM_D3Q19 ? (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0)
                                                        : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
            shifted -= (i == 0 ? -(1.0 - w0) : wi) * (double)a;
        }
        float v = (float)shifted;
        CK(cudaMemcpyAsync(base + m * 4, &v, 4, cudaMemcpyHostToDevice, ctx->stream));
        if (field == 0 && i == 0)  // low word of the rest population pair
            CK(cudaMemcpyAsync(base + (m + (size_t)ctx->Q * ctx->N) * 4, &zero, 4,
                               cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    free(ctx);
}

const char *lbm_strerror(int code)
{
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_CUDA: return "CUDA error (context unusable)";
    case LBM_ERR_NONFINITE: return "non-finite value in the fields";
    case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
    case LBM_ERR_STATE: return "context not initialised";
    default: return "unknown error";
    }
}


}  // extern "C"

// ------------------------------------------------------------------ batches

// Status of a batch in mapped pinned host memory (written by the device):
// the timeout word, then one diagnostics record per grid.
struct BatchStatus {
    int err;  // a multi-step launch timed out
    int pad[15];
};
DiagPartial *status_rec(BatchStatus *s) { return reinterpret_cast<DiagPartial *>(s + 1); }

struct lbm_batch {
    int n;
    lbm_ctx **ctx;
    int precision;
    int device, nsm;
    cudaStream_t stream, cap;
    BatchCase *d_cases;       // S_out = S (real steps)
    BatchCase *d_cases_tune;  // S_out = scratch (tuning leaves the state unchanged)
    BatchTile *d_tiles;
    int *d_tile0;             // ncases + 1: first tile of each grid
    int tiles_cap, ntiles;
    int width, rows, tuned;
    cudaGraphExec_t gexec;
    int gexec_valid;
    int err;                  // sticky error of the batch (LBM_ERR_TIMEOUT until a reset)
    // multi-step launches (a queue of (step, tile) pairs per cooperative launch)
    int persist;     // requested
    int persist_ok;  // the current tiles have neighbour lists
    int seg;         // FP32 and every grid's rows a multiple of 4 nodes: the
                     // multi-step launches stage their pulls as row segments
    int *d_nbr;      // per tile: count, then up to PERSIST_NBMAX neighbour tiles
    int *d_ctr;      // two sets, used by alternate launches, each: 4 counters, per tile
                     // the steps completed, one spare (never set), per grid the
                     // tiles done with the diagnostics step, per step of the
                     // launch (up to PERSIST_STEP_CAP) the tiles done with it
    int ctr_sel;     // the set the next multi-step launch uses (the other is zero)
    int stall_tile;  // fault injection: the tile made to wait (else -1)
    int *d_err;      // set by a wait that timed out
    int persist_cap; // tiles d_nbr and d_ctr hold
    // fused diagnostics
    int diag_every;          // 0: none; else every step starting at a multiple of it
    DiagPartial *d_partials; // one per tile
    int partials_cap;
    BatchStatus *h_status;   // mapped pinned host memory: error word and per-grid records
    BatchStatus *d_status;   // its device address
    cudaEvent_t diag_ev;     // recorded after the launch that wrote the records
    int diag_pending, has_last_diag;
    long long last_diag_step;
};

namespace {

constexpr int BATCH_GRAPH_STEPS = 32;

void batch_free(lbm_batch *b)
{
    if (b->gexec_valid) cudaGraphExecDestroy(b->gexec);
    void *dev[] = {b->d_nbr, b->d_ctr, b->d_err, b->d_cases, b->d_cases_tune, b->d_tiles,
                   b->d_tile0, b->d_partials};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->diag_ev) cudaEventDestroy(b->diag_ev);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ctx) {
        for (int c = 0; c < b->n; ++c) lbm_destroy(b->ctx[c]);
        free(b->ctx);
    }
    free(b);
}

#define BK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            b->err = LBM_ERR_CUDA;                      \
            return LBM_ERR_CUDA;                        \
        }                                               \
    } while (0)

// device buffers of at least `count` ints / records, reallocated on growth
int grow(void **p, int *cap, int count, size_t elem)
{
    if (count <= *cap) return LBM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, (size_t)count * elem) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return LBM_ERR_OOM;
    }
    *cap = count;
    return LBM_OK;
}

// Neighbour lists of the tiles for multi-step launches: for every tile the
// other tiles of its grid whose region meets the tile's stencil reach (3
// nodes: phi at radius 2 is summed from populations pulled at radius 1),
// periodic.  Sets persist_ok unless a list is longer than PERSIST_NBMAX.
int batch_build_nbr(lbm_batch *b, const BatchTile *h, int count, int width, int rows)
{
    b->persist_ok = 0;
    if (rows < 1) return LBM_OK;
    constexpr int REACH = 3;
    const int stride = PERSIST_NBMAX + 1;
    int *nb = (int *)malloc((size_t)count * stride * sizeof(int));
    if (!nb) return LBM_ERR_OOM;
    int base = 0;  // index of the case's first tile
    bool ok = true;
    for (int k = 0; k < count && ok; ++k) {
        const BatchTile &t = h[k];
        if (k > 0 && t.c != h[k - 1].c) base = k;
        const lbm_grid &g = b->ctx[t.c]->grid;
        const int sx = (g.nx + width - 1) / width;
        const int xe = t.x0 + width < g.nx ? t.x0 + width : g.nx;
        // the distinct tile rows and strips the reach touches, then their product
        int rs[PERSIST_NBMAX + 1], ss[PERSIST_NBMAX + 1], nr = 0, ns = 0;
        for (int yy = t.y0 - REACH; yy < t.yend + REACH && ok; ++yy) {
            const int r = ((yy % g.ny) + g.ny) % g.ny / rows;
            bool seen = false;
            for (int j = 0; j < nr; ++j) seen = seen || rs[j] == r;
            if (!seen) {
                if (nr == PERSIST_NBMAX + 1) ok = false;
                else rs[nr++] = r;
            }
        }
        for (int xx = t.x0 - REACH; xx < xe + REACH && ok; ++xx) {
            const int sidx = ((xx % g.nx) + g.nx) % g.nx / width;
            bool seen = false;
            for (int j = 0; j < ns; ++j) seen = seen || ss[j] == sidx;
            if (!seen) {
                if (ns == PERSIST_NBMAX + 1) ok = false;
                else ss[ns++] = sidx;
            }
        }
        int *row = nb + (size_t)k * stride, n = 0;
        for (int i = 0; i < nr && ok; ++i)
            for (int j = 0; j < ns && ok; ++j) {
                const int u = base + rs[i] * sx + ss[j];
                if (u == k) continue;
                if (n == PERSIST_NBMAX) ok = false;
                else row[1 + n++] = u;
            }
        row[0] = n;
    }
    if (!ok) {
        free(nb);
        return LBM_OK;
    }
    if (count > b->persist_cap) {
        int cap_nbr = 0, cap_ctr = 0;
        if (b->d_nbr) cudaFree(b->d_nbr);
        if (b->d_ctr) cudaFree(b->d_ctr);
        b->d_nbr = nullptr;
        b->d_ctr = nullptr;
        b->persist_cap = 0;
        if (grow((void **)&b->d_nbr, &cap_nbr, count * stride, sizeof(int)) ||
            grow((void **)&b->d_ctr, &cap_ctr, 2 * (count + 5 + b->n + PERSIST_STEP_CAP),
                 sizeof(int))) {
            free(nb);
            return LBM_ERR_OOM;
        }
        b->persist_cap = count;
    }
    // both counter sets start at zero; each launch zeroes the other one
    cudaError_t e =
        cudaMemset(b->d_ctr, 0, 2 * ((size_t)count + 5 + b->n + PERSIST_STEP_CAP) * sizeof(int));
    b->ctr_sel = 0;
    b->stall_tile = -1;
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_nbr, nb, (size_t)count * stride * sizeof(int), cudaMemcpyHostToDevice);
    free(nb);
    if (e != cudaSuccess) {
        b->err = LBM_ERR_CUDA;
        return LBM_ERR_CUDA;
    }
    b->persist_ok = 1;
    return LBM_OK;
}

// tiles of every grid: strips of `width` columns, row tiles of `rows` rows,
// row-major per grid; odd row tiles march up
int batch_build_tiles(lbm_batch *b, int width, int rows)
{
    long long count = 0;
    for (int c = 0; c < b->n; ++c) {
        const lbm_grid &g = b->ctx[c]->grid;
        count += (long long)((g.nx + width - 1) / width) * ((g.ny + rows - 1) / rows);
    }
    if (count > (1LL << 30)) return LBM_ERR_INVALID_ARG;
    BatchTile *h = (BatchTile *)malloc((size_t)count * sizeof(BatchTile));
    int *t0 = (int *)malloc(((size_t)b->n + 1) * sizeof(int));
    if (!h || !t0) {
        free(h);
        free(t0);
        return LBM_ERR_OOM;
    }
    long long k = 0;
    for (int c = 0; c < b->n; ++c) {
        const lbm_grid &g = b->ctx[c]->grid;
        const int ty = (g.ny + rows - 1) / rows;
        t0[c] = (int)k;
        for (int r = 0; r < ty; ++r)
            for (int x0 = 0; x0 < g.nx; x0 += width) {
                BatchTile t;
                t.c = c;
                t.x0 = x0;
                t.y0 = r * rows;
                t.yend = t.y0 + rows < g.ny ? t.y0 + rows : g.ny;
                t.dir = (r & 1) ? -1 : 1;
                h[k++] = t;
            }
    }
    t0[b->n] = (int)k;
    int rc = grow((void **)&b->d_tiles, &b->tiles_cap, (int)count, sizeof(BatchTile));
    if (rc == LBM_OK)
        rc = grow((void **)&b->d_partials, &b->partials_cap, (int)count, sizeof(DiagPartial));
    if (rc == LBM_OK &&
        (cudaMemcpy(b->d_tiles, h, (size_t)count * sizeof(BatchTile), cudaMemcpyHostToDevice) !=
             cudaSuccess ||
         cudaMemcpy(b->d_tile0, t0, ((size_t)b->n + 1) * sizeof(int), cudaMemcpyHostToDevice) !=
             cudaSuccess)) {
        b->err = LBM_ERR_CUDA;
        rc = LBM_ERR_CUDA;
    }
    if (rc == LBM_OK) rc = batch_build_nbr(b, h, (int)count, width, rows);
    free(h);
    free(t0);
    if (rc) return rc;
    b->ntiles = (int)count;
    b->width = width;
    b->rows = rows;
    if (b->gexec_valid) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec_valid = 0;
    }
    return LBM_OK;
}

int batch_ready(lbm_batch *b)
{
    for (int c = 0; c < b->n; ++c) {
        const lbm_ctx *x = b->ctx[c];
        if (!x->initialized || x->cur != b->ctx[0]->cur || x->step != b->ctx[0]->step)
            return LBM_ERR_STATE;
        if (x->err == LBM_ERR_CUDA) return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int batch_launch(lbm_batch *b, const BatchCase *cases, int parity, cudaStream_t st,
                 DiagPartial *partials = nullptr)
{
    BK(d2q9_batch_step(b->precision, b->width, cases, b->d_tiles, b->ntiles, parity, partials,
                       st));
    return LBM_OK;
}

// tiles of every grid at strip width w and r rows per tile
long long count_tiles(const lbm_batch *b, int w, int r)
{
    long long n = 0;
    for (int c = 0; c < b->n; ++c) {
        const lbm_grid &g = b->ctx[c]->grid;
        n += (long long)((g.nx + w - 1) / w) * ((g.ny + r - 1) / r);
    }
    return n;
}

int batch_tune(lbm_batch *b)
{
    const int parity = b->ctx[0]->cur;
    const int widths[2] = {128, 64};
    constexpr int NR = 15;
    const int rowsc[NR] = {8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 64, 80, 96, 128};
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    float best = 3.4e38f;
    int bw = 128, br = 16;
    int rc = LBM_OK;
    for (int wi = 0; wi < 2 && rc == LBM_OK; ++wi) {
        // the listed row counts, and the shortest even one whose tiles fill
        // one wave of resident CTAs (every SM then holds the same number)
        int cand[NR + 1], nc = 0;
        for (int ri = 0; ri < NR; ++ri) cand[nc++] = rowsc[ri];
        const int per_sm = d2q9_batch_persist_ctas_per_sm(b->precision == LBM_FP64 ? 0 : 1,
                                                          widths[wi], b->seg != 0);
        const long long slots = (long long)(per_sm > 0 ? per_sm : 4) * b->nsm;
        for (int r = 2; r <= 256; r += 2)
            if (count_tiles(b, widths[wi], r) <= slots) {
                bool listed = false;
                for (int ri = 0; ri < NR; ++ri) listed = listed || rowsc[ri] == r;
                if (!listed) cand[nc++] = r;
                break;
            }
        for (int ri = 0; ri < nc && rc == LBM_OK; ++ri) {
            rc = batch_build_tiles(b, widths[wi], cand[ri]);
            if (rc) break;
            for (int k = 0; k < 2 && rc == LBM_OK; ++k)
                rc = batch_launch(b, b->d_cases_tune, parity, b->stream);
            if (rc) break;
            cudaEventRecord(e0, b->stream);
            for (int k = 0; k < 5 && rc == LBM_OK; ++k)
                rc = batch_launch(b, b->d_cases_tune, parity, b->stream);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_ERR_CUDA;
            float ms = 0.0f;
            if (rc == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
                best = ms;
                bw = widths[wi];
                br = cand[ri];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = batch_build_tiles(b, bw, br);
    if (rc == LBM_OK) b->tuned = 1;
    return rc;
}

int batch_graph(lbm_batch *b)
{
    if (b->gexec_valid) return LBM_OK;
    cudaGraph_t graph = nullptr;
    BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    for (int k = 0; k < BATCH_GRAPH_STEPS && rc == LBM_OK; ++k)
        rc = batch_launch(b, b->d_cases, k & 1, b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc != LBM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        b->err = LBM_ERR_CUDA;
        return rc ? rc : LBM_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    BK(e);
    b->gexec_valid = 1;
    return LBM_OK;
}

void batch_advance(lbm_batch *b, int steps)
{
    for (int c = 0; c < b->n; ++c) {
        b->ctx[c]->cur ^= (steps & 1);
        b->ctx[c]->step += steps;
    }
}

// the records of the last diagnostics launch, once it has completed (or at
// once with wait): non-finite fields become the batch's pending error
void batch_poll(lbm_batch *b, bool wait)
{
    volatile int *herr = &b->h_status->err;  // written by the device
    if (*herr && b->err == LBM_OK) b->err = LBM_ERR_TIMEOUT;
    if (!b->diag_pending) return;
    const cudaError_t e = wait ? cudaEventSynchronize(b->diag_ev) : cudaEventQuery(b->diag_ev);
    if (e == cudaErrorNotReady) return;
    if (e != cudaSuccess) {
        b->err = LBM_ERR_CUDA;
        return;
    }
    b->diag_pending = 0;
    if (*herr && b->err == LBM_OK) b->err = LBM_ERR_TIMEOUT;
    for (int c = 0; c < b->n; ++c)
        if (status_rec(b->h_status)[c].nonfinite != 0.0 && b->err == LBM_OK) b->err = LBM_ERR_NONFINITE;
}

// the batch's error, once: a timeout stays until the tiles are rebuilt
int batch_take_err(lbm_batch *b)
{
    const int e = b->err;
    if (e == LBM_ERR_NONFINITE) b->err = LBM_OK;
    return e;
}

// first step >= t that carries diagnostics, or -1
long long next_diag(const lbm_batch *b, long long t)
{
    if (b->diag_every <= 0) return -1;
    const long long k = b->diag_every;
    return (t + k - 1) / k * k;
}

// n steps as multi-step launches, each holding at most one diagnostics step
int batch_run_persistent(lbm_batch *b, int n)
{
    const int prec = b->precision == LBM_FP64 ? 0 : 1;
    int cap = (int)((0x7fffffff - 1) / (b->ntiles > 0 ? b->ntiles : 1));
    if (cap > PERSIST_STEP_CAP) cap = PERSIST_STEP_CAP;
    int left = n;
    while (left > 0) {
        const long long t = b->ctx[0]->step;
        int m = left < cap ? left : cap;
        const long long d = next_diag(b, t);
        int diag_k = -1;
        if (d >= 0 && d < t + m) {
            diag_k = (int)(d - t);
            const long long d2 = d + b->diag_every;  // the next one starts a new launch
            if (d2 < t + m) m = (int)(d2 - t);
        }
        PersistArgs pa;
        pa.cases = b->d_cases;
        pa.tiles = b->d_tiles;
        pa.nbr = b->d_nbr;
        pa.tile0 = b->d_tile0;
        pa.ntiles = b->ntiles;
        pa.ncases = b->n;
        pa.parity0 = b->ctx[0]->cur;
        pa.nsteps = m;
        pa.diag_k = diag_k;
        const size_t nctr = (size_t)b->ntiles + 5 + b->n + PERSIST_STEP_CAP;  // per counter set
        pa.ctr = b->d_ctr + (size_t)b->ctr_sel * nctr;
        pa.ctr_next = b->d_ctr + (size_t)(b->ctr_sel ^ 1) * nctr;
        pa.nctr = (int)nctr;
        pa.flags = pa.ctr + 4;
        pa.case_ctr = pa.flags + b->ntiles + 1;
        pa.step_done = pa.case_ctr + b->n;
        pa.stall_tile = b->stall_tile;
        pa.err = b->d_err;
        pa.err_host = &b->d_status->err;
        pa.partials = b->d_partials;
        pa.records = status_rec(b->d_status);
        const int per_sm = d2q9_batch_persist_ctas_per_sm(prec, b->width, b->seg != 0);
        if (per_sm < 1) {
            b->err = LBM_ERR_CUDA;
            return LBM_ERR_CUDA;
        }
        // one CTA per tile when they all fit at once, else a queue over every slot
        const long long pairs = (long long)m * b->ntiles, slots = (long long)per_sm * b->nsm;
        const int nctas = b->ntiles <= slots ? b->ntiles : (int)(pairs < slots ? pairs : slots);
        BK(d2q9_batch_persist(prec, b->width, b->seg != 0, pa, nctas, b->stream));
        b->ctr_sel ^= 1;
        if (diag_k >= 0) {
            BK(cudaEventRecord(b->diag_ev, b->stream));
            b->diag_pending = 1;
            b->has_last_diag = 1;
            b->last_diag_step = t + diag_k;
        }
        batch_advance(b, m);
        left -= m;
    }
    return LBM_OK;
}

// one step with diagnostics of its source state (per-step launches)
int batch_diag_step(lbm_batch *b)
{
    const long long t = b->ctx[0]->step;
    if (int rc = batch_launch(b, b->d_cases, b->ctx[0]->cur, b->stream, b->d_partials)) return rc;
    BK(d2q9_batch_reduce(b->precision == LBM_FP64 ? 0 : 1, b->d_partials, b->d_tile0, b->d_cases,
                         b->n, status_rec(b->d_status), b->stream));
    BK(cudaEventRecord(b->diag_ev, b->stream));
    b->diag_pending = 1;
    b->has_last_diag = 1;
    b->last_diag_step = t;
    batch_advance(b, 1);
    return LBM_OK;
}

// n plain steps as per-step launches (CUDA-graph replay of 32-step blocks)
int batch_run_plain(lbm_batch *b, int n)
{
    int left = n;
    if (left >= BATCH_GRAPH_STEPS) {
        if (b->ctx[0]->cur == 1) {
            if (int rc = batch_launch(b, b->d_cases, 1, b->stream)) return rc;
            batch_advance(b, 1);
            --left;
        }
        if (left >= BATCH_GRAPH_STEPS) {
            if (int rc = batch_graph(b)) return rc;
            const int reps = left / BATCH_GRAPH_STEPS;
            for (int r = 0; r < reps; ++r) BK(cudaGraphLaunch(b->gexec, b->stream));
            batch_advance(b, reps * BATCH_GRAPH_STEPS);
            left -= reps * BATCH_GRAPH_STEPS;
        }
    }
    for (; left > 0; --left) {
        if (int rc = batch_launch(b, b->d_cases, b->ctx[0]->cur, b->stream)) return rc;
        batch_advance(b, 1);
    }
    return LBM_OK;
}

// a rebuild of the tiles clears a timeout: the error words and the sticky error
// Tile shape for multi-step launches: each candidate (the per-step
// tuner's list, plus for each width the shortest tiles that fit one wave
// and two waves of resident CTAs) is timed as multi-step launches on the
// grids' own state, with diagnostics off.  The state the steps change (the
// current population buffers, S, the FP32 equilibrium shifts, the step
// count and parity) is saved first and put back after, so tuning leaves it
// as it was.  Candidates whose neighbour lists overflow are skipped.
int batch_tune_persist(lbm_batch *b)
{
    const int widths[2] = {128, 64};
    constexpr int NR = 15;
    const int rowsc[NR] = {8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 64, 80, 96, 128};
    constexpr int WARM = 2, TIMED = 8;
    const int prec = b->precision == LBM_FP64 ? 0 : 1;
    // save the state
    size_t total = 0;
    for (int c = 0; c < b->n; ++c) {
        const lbm_ctx *x = b->ctx[c];
        total += x->fbytes + x->gbytes + (size_t)x->N * x->esz + 4 * sizeof(float);
    }
    char *save = nullptr;
    if (cudaMalloc((void **)&save, total) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    const int cur0 = b->ctx[0]->cur;
    const long long step0 = b->ctx[0]->step;
    const int diag_every0 = b->diag_every;
    auto copy_state = [&](bool restore) {
        size_t o = 0;
        for (int c = 0; c < b->n; ++c) {
            const lbm_ctx *x = b->ctx[c];
            const size_t sb = (size_t)x->N * x->esz;
            void *live[4] = {x->f[cur0], x->g[cur0], x->S, x->eqs};
            const size_t len[4] = {x->fbytes, x->gbytes, sb, 4 * sizeof(float)};
            for (int k = 0; k < 4; ++k) {
                void *dst = restore ? live[k] : (void *)(save + o);
                const void *src = restore ? (const void *)(save + o) : live[k];
                if (cudaMemcpyAsync(dst, src, len[k], cudaMemcpyDeviceToDevice, b->stream) !=
                    cudaSuccess)
                    return false;
                o += len[k];
            }
        }
        return true;
    };
    int rc = copy_state(false) ? LBM_OK : LBM_ERR_CUDA;
    b->diag_every = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = LBM_ERR_CUDA;
    float best = 3.4e38f;
    int bw = 0, br = 0;
    for (int wi = 0; wi < 2 && rc == LBM_OK; ++wi) {
        int cand[NR + 2], nc = 0;
        for (int ri = 0; ri < NR; ++ri) cand[nc++] = rowsc[ri];
        const int per_sm = d2q9_batch_persist_ctas_per_sm(prec, widths[wi], b->seg != 0);
        const long long slots = (long long)(per_sm > 0 ? per_sm : 4) * b->nsm;
        for (long long waves = 1; waves <= 2; ++waves)
            for (int r = 2; r <= 256; r += 2)
                if (count_tiles(b, widths[wi], r) <= waves * slots) {
                    bool listed = false;
                    for (int ri = 0; ri < nc; ++ri) listed = listed || cand[ri] == r;
                    if (!listed) cand[nc++] = r;
                    break;
                }
        for (int ri = 0; ri < nc && rc == LBM_OK; ++ri) {
            rc = batch_build_tiles(b, widths[wi], cand[ri]);
            if (rc || !b->persist_ok) continue;
            rc = batch_run_persistent(b, WARM);
            if (rc) break;
            cudaEventRecord(e0, b->stream);
            rc = batch_run_persistent(b, TIMED);
            cudaEventRecord(e1, b->stream);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = LBM_ERR_CUDA;
                break;
            }
            if (*(volatile int *)&b->h_status->err) {  // a wait timed out
                b->err = LBM_ERR_TIMEOUT;
                rc = LBM_ERR_TIMEOUT;
                break;
            }
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
                best = ms;
                bw = widths[wi];
                br = cand[ri];
            }
        }
    }
    // put the state back (also after a failure: the steps taken are undone)
    if (!copy_state(true) && rc == LBM_OK) rc = LBM_ERR_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && rc == LBM_OK) rc = LBM_ERR_CUDA;
    for (int c = 0; c < b->n; ++c) {
        b->ctx[c]->cur = cur0;
        b->ctx[c]->step = step0;
    }
    b->diag_every = diag_every0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (rc) return rc;
    if (bw == 0) return LBM_ERR_INVALID_ARG;  // no shape has usable neighbour lists
    rc = batch_build_tiles(b, bw, br);
    if (rc == LBM_OK) b->tuned = 1;
    return rc;
}

int batch_reset_timeout(lbm_batch *b)
{
    if (b->err != LBM_ERR_TIMEOUT && !*(volatile int *)&b->h_status->err) return LBM_OK;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess) {
        b->err = LBM_ERR_CUDA;
        return LBM_ERR_CUDA;
    }
    b->h_status->err = 0;
    if (b->err == LBM_ERR_TIMEOUT) b->err = LBM_OK;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int ncases, const lbm_grid *grids, const lbm_params *params,
                     void *cuda_stream, lbm_batch **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (ncases < 1 || !grids || !params) return LBM_ERR_INVALID_ARG;
    for (int c = 0; c < ncases; ++c) {
        if (int rc = validate(&grids[c], LBM_D2Q9, &params[c])) return rc;
        if (params[c].precision != params[0].precision) return LBM_ERR_INVALID_ARG;
    }
    lbm_batch *b = (lbm_batch *)calloc(1, sizeof(lbm_batch));
    if (!b) return LBM_ERR_OOM;
    b->n = ncases;
    b->precision = params[0].precision;
    b->stream = (cudaStream_t)cuda_stream;
    b->ctx = (lbm_ctx **)calloc((size_t)ncases, sizeof(lbm_ctx *));
    if (!b->ctx) {
        free(b);
        return LBM_ERR_OOM;
    }
    for (int c = 0; c < ncases; ++c) {
        int rc = lbm_create(&grids[c], LBM_D2Q9, &params[c], cuda_stream, &b->ctx[c]);
        if (rc) {
            batch_free(b);
            return rc;
        }
    }
    b->device = b->ctx[0]->device;
    b->seg = b->precision != LBM_FP64;
    for (int c = 0; c < ncases; ++c)
        if (grids[c].nx % 4 != 0) b->seg = 0;
    BatchCase *h = (BatchCase *)calloc((size_t)ncases, sizeof(BatchCase));
    if (!h) {
        batch_free(b);
        return LBM_ERR_OOM;
    }
    for (int c = 0; c < ncases; ++c) {
        lbm_ctx *x = b->ctx[c];
        h[c].pd = x->pd;
        h[c].pf = x->pf;
        h[c].f[0] = x->f[0];
        h[c].f[1] = x->f[1];
        h[c].g[0] = x->g[0];
        h[c].g[1] = x->g[1];
        h[c].S = x->S;
        h[c].S_out = x->S;
        h[c].eqs = x->eqs;
        h[c].recentre = x->recentre;
    }
    const size_t bytes = (size_t)ncases * sizeof(BatchCase);
    const size_t sbytes = sizeof(BatchStatus) + (size_t)ncases * sizeof(DiagPartial);
    bool ok = cudaMalloc((void **)&b->d_cases, bytes) == cudaSuccess &&
              cudaMalloc((void **)&b->d_cases_tune, bytes) == cudaSuccess &&
              cudaMemcpy(b->d_cases, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMalloc((void **)&b->d_tile0, ((size_t)ncases + 1) * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_err, sizeof(int)) == cudaSuccess &&
              cudaMemset(b->d_err, 0, sizeof(int)) == cudaSuccess &&
              cudaHostAlloc((void **)&b->h_status, sbytes, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&b->d_status, b->h_status, 0) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->diag_ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) memset(b->h_status, 0, sbytes);
    for (int c = 0; c < ncases && ok; ++c) h[c].S_out = b->ctx[c]->aux;  // scratch for tuning
    ok = ok && cudaMemcpy(b->d_cases_tune, h, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
         cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess;
    free(h);
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        return LBM_ERR_OOM;
    }
    // untuned default: 128-column strips, about one wave of 4 CTAs per SM
    long long strip_rows = 0;
    for (int c = 0; c < ncases; ++c)
        strip_rows += (long long)((grids[c].nx + 127) / 128) * grids[c].ny;
    long long rows = (strip_rows + 4LL * b->nsm - 1) / (4LL * b->nsm);
    rows = rows < 8 ? 8 : (rows > 128 ? 128 : rows);
    if (int rc = batch_build_tiles(b, 128, (int)(rows + (rows & 1)))) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_case(lbm_batch *b, int c, lbm_ctx **ctx)
{
    if (!b || !ctx || c < 0 || c >= b->n) return LBM_ERR_INVALID_ARG;
    *ctx = b->ctx[c];
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int n)
{
    if (!b || n < 0) return LBM_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    batch_poll(b, false);
    if (b->err) return batch_take_err(b);
    if (int rc = batch_ready(b)) return rc;
    if (!b->tuned && n > 0)
        if (int rc = b->persist ? batch_tune_persist(b) : batch_tune(b)) return rc;
    if (b->persist && b->persist_ok && n >= 2) return batch_run_persistent(b, n);
    int left = n;
    while (left > 0) {
        const long long t = b->ctx[0]->step;
        const long long d = next_diag(b, t);
        if (d == t) {
            if (int rc = batch_diag_step(b)) return rc;
            --left;
            continue;
        }
        const int run = (d >= 0 && d - t < left) ? (int)(d - t) : left;
        if (int rc = batch_run_plain(b, run)) return rc;
        left -= run;
    }
    return LBM_OK;
}

int lbm_batch_set_diag_every(lbm_batch *b, int k)
{
    if (!b || k < 0) return LBM_ERR_INVALID_ARG;
    b->diag_every = k;
    return LBM_OK;
}

int lbm_batch_last_diagnostics(lbm_batch *b, lbm_diag *out)
{
    if (!b || !out) return LBM_ERR_INVALID_ARG;
    if (!b->has_last_diag) return LBM_ERR_STATE;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    if (b->diag_pending) {
        if (cudaEventSynchronize(b->diag_ev) != cudaSuccess) {
            b->err = LBM_ERR_CUDA;
            return LBM_ERR_CUDA;
        }
    }
    batch_poll(b, true);
    for (int c = 0; c < b->n; ++c) fill_diag(status_rec(b->h_status)[c], b->last_diag_step, &out[c]);
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch *b)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        b->err = LBM_ERR_CUDA;
        return LBM_ERR_CUDA;
    }
    batch_poll(b, true);
    return batch_take_err(b);
}

int lbm_batch_shape(const lbm_batch *b, int *width, int *rows, int *ntiles)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (width) *width = b->width;
    if (rows) *rows = b->rows;
    if (ntiles) *ntiles = b->ntiles;
    return LBM_OK;
}


int lbm_batch_tune(lbm_batch *b, int *width, int *rows)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    if (int rc = batch_ready(b)) return rc;
    if (int rc = batch_reset_timeout(b)) return rc;
    if (int rc = b->persist ? batch_tune_persist(b) : batch_tune(b)) return rc;
    if (width) *width = b->width;
    if (rows) *rows = b->rows;
    return LBM_OK;
}

int lbm_batch_set_shape(lbm_batch *b, int width, int rows)
{
    if (!b || (width != 64 && width != 128) || rows < 2) return LBM_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    if (int rc = batch_reset_timeout(b)) return rc;
    if (int rc = batch_build_tiles(b, width, rows)) return rc;
    b->tuned = 1;
    return LBM_OK;
}

int lbm_batch_set_persistent(lbm_batch *b, int on)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    if (on && !b->tuned) {
        // timed on the state when there is one, else with per-step launches
        if (batch_ready(b) == LBM_OK) {
            if (int rc = batch_reset_timeout(b)) return rc;
            if (int rc = batch_tune_persist(b)) return rc;
        } else if (int rc = batch_tune(b)) {
            return rc;
        }
    }
    if (on && !b->persist_ok) return LBM_ERR_INVALID_ARG;
    b->persist = on ? 1 : 0;
    return LBM_OK;
}

int lbm_batch_persistent(const lbm_batch *b, int *on, int *timed_out)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (on) *on = b->persist && b->persist_ok;
    if (timed_out) {
        int v = 0;
        if (cudaSetDevice(b->device) != cudaSuccess ||
            cudaMemcpy(&v, b->d_err, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess)
            return LBM_ERR_CUDA;
        *timed_out = v;
    }
    return LBM_OK;
}

int lbm_batch_debug_stall(lbm_batch *b, int tile)
{
    if (!b || tile < 0 || tile >= b->ntiles || !b->persist || !b->persist_ok)
        return LBM_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ERR_CUDA;
    // one neighbour: the spare counter after the tiles' own (index ntiles);
    // the tile always waits (no step-completion shortcut)
    const int rec[2] = {1, b->ntiles};
    if (cudaMemcpy(b->d_nbr + (size_t)tile * (PERSIST_NBMAX + 1), rec, sizeof rec,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return LBM_ERR_CUDA;
    b->stall_tile = tile;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint

struct lbm_adjoint {
    lbm_ctx *ctx;
    int K, max_steps, nsteps, recorded;
    size_t snap;        // bytes of one state snapshot (f, g, S at the context's precision)
    size_t slot;        // bytes of one segment slot: a snapshot, then its moments
    char *ckpt;         // (max_steps / K + 1) snapshots
    char *seg;          // K slots of the segment being reversed
    int real;           // adjoint arithmetic: 0 FP64, 1 FP32 (the context's precision)
    size_t rsz;         // bytes per adjoint value
    double *phi0;       // N
    void *lf[2], *lg[2], *lS[2];  // adjoint fields at the adjoint precision
    void *lpt;                    // the adjoint of f common to all directions [N]
    double *macro;      // N doubles: device staging of dL/dphi0 for a host destination
    void *work;         // 6N adjoint values (at least N doubles)
    double *dpar;       // 3
};

namespace {

int snapshot(lbm_ctx *ctx, char *dst, size_t snap)
{
    const size_t N = (size_t)ctx->N, fb = ctx->fbytes, gb = ctx->gbytes;
    (void)snap;
    CK(cudaMemcpyAsync(dst, ctx->f[ctx->cur], fb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dst + fb, ctx->g[ctx->cur], gb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dst + fb + gb, ctx->S, N * ctx->esz, cudaMemcpyDeviceToDevice, ctx->stream));
    return LBM_OK;
}

int restore(lbm_ctx *ctx, const char *src, long long step)
{
    const size_t N = (size_t)ctx->N, fb = ctx->fbytes, gb = ctx->gbytes;
    CK(cudaMemcpyAsync(ctx->f[0], src, fb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->g[0], src + fb, gb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->S, src + fb + gb, N * ctx->esz, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->cur = 0;
    ctx->step = step;
    ctx->initialized = 1;
    return LBM_OK;
}

void adjoint_free(lbm_adjoint *a)
{
    void *p[] = {a->ckpt, a->seg, a->phi0, a->lf[0], a->lf[1], a->lg[0], a->lg[1],
                 a->lS[0], a->lS[1], a->lpt, a->macro, a->work, a->dpar};
    for (void *q : p)
        if (q) cudaFree(q);
    free(a);
}

}  // namespace

extern "C" {

int lbm_adjoint_create(lbm_ctx *ctx, int checkpoint_every, int max_steps, lbm_adjoint **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx || ctx->lattice != LBM_D2Q9 || checkpoint_every < 1 || max_steps < 1)
        return LBM_ERR_INVALID_ARG;
    if (int rc = set_device(ctx)) return rc;
    lbm_adjoint *a = (lbm_adjoint *)calloc(1, sizeof(lbm_adjoint));
    if (!a) return LBM_ERR_OOM;
    a->ctx = ctx;
    a->K = checkpoint_every;
    a->max_steps = max_steps;
    const size_t N = (size_t)ctx->N, Q = (size_t)ctx->Q;
    a->snap = ((size_t)ctx->nf * N + Q * N + N) * ctx->esz;
    a->snap = (a->snap + 255) / 256 * 256;
    // phi, mu, p and u (5N values) of each segment state sit after its snapshot
    a->slot = a->snap + (5 * N * ctx->esz + 255) / 256 * 256;
    const size_t nck = (size_t)(max_steps / checkpoint_every + 1);
    a->real = ctx->prm.precision == LBM_FP64 ? 0 : 1;
    a->rsz = a->real == 0 ? sizeof(double) : sizeof(float);
    bool ok = cudaMalloc((void **)&a->ckpt, nck * a->snap) == cudaSuccess &&
              cudaMalloc((void **)&a->seg, (size_t)checkpoint_every * a->slot) == cudaSuccess &&
              cudaMalloc((void **)&a->phi0, N * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&a->macro, N * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&a->work, 6 * N * a->rsz) == cudaSuccess &&
              cudaMalloc(&a->lpt, N * a->rsz) == cudaSuccess &&
              cudaMalloc((void **)&a->dpar, 3 * sizeof(double)) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaMalloc(&a->lf[b], Q * N * a->rsz) == cudaSuccess &&
             cudaMalloc(&a->lg[b], Q * N * a->rsz) == cudaSuccess &&
             cudaMalloc(&a->lS[b], N * a->rsz) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        adjoint_free(a);
        return LBM_ERR_OOM;
    }
    ctx->recentre = 0;  // the recorded states keep one equilibrium shift
    *out = a;
    return LBM_OK;
}

int lbm_adjoint_forward(lbm_adjoint *a, const double *phi0, int on_device, int nsteps)
{
    if (!a || !phi0 || nsteps < 0 || nsteps > a->max_steps) return LBM_ERR_INVALID_ARG;
    lbm_ctx *ctx = a->ctx;
    if (int rc = set_device(ctx)) return rc;
    const size_t N = (size_t)ctx->N;
    CK(cudaMemcpyAsync(a->phi0, phi0, N * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    if (int rc = lbm_init_phi(ctx, a->phi0, 1)) return rc;
    for (int done = 0, k = 0; done <= nsteps; done += a->K, ++k) {
        if (int rc = snapshot(ctx, a->ckpt + (size_t)k * a->snap, a->snap)) return rc;
        const int m = nsteps - done < a->K ? nsteps - done : a->K;
        if (m > 0)
            if (int rc = lbm_step(ctx, m)) return rc;
        if (m < a->K) break;
    }
    a->nsteps = nsteps;
    a->recorded = 1;
    return LBM_OK;
}

int lbm_adjoint_backward(lbm_adjoint *a, const double *dL_dphi, int on_device, double *dL_dphi0,
                         double grads[4])
{
    if (!a || !dL_dphi || !dL_dphi0 || !grads) return LBM_ERR_INVALID_ARG;
    if (!a->recorded) return LBM_ERR_STATE;
    lbm_ctx *ctx = a->ctx;
    if (int rc = set_device(ctx)) return rc;
    const size_t N = (size_t)ctx->N;
    const int nx = ctx->grid.nx, ny = ctx->grid.ny;
    // the seed: dL/dphi of the final state into the adjoint of every f_i
    double *seed = (double *)a->work;  // 6 N adjoint values hold N doubles
    CK(cudaMemcpyAsync(seed, dL_dphi, N * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    int cb = 0;
    CK(adj_d2q9_seed(a->real, (int)N, seed, a->lf[cb], a->lpt, a->lg[cb], a->lS[cb], ctx->stream));
    CK(cudaMemsetAsync(a->dpar, 0, 3 * sizeof(double), ctx->stream));
    const int nseg = (a->nsteps + a->K - 1) / a->K;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int t0 = sgi * a->K;
        const int len = a->nsteps - t0 < a->K ? a->nsteps - t0 : a->K;
        // recompute the segment forward from its checkpoint, each step writing
        // straight into the next state slot of the segment and the moments of
        // the state it steps from beside that state (the last state's moments
        // come from a moments-only pass)
        CK(cudaMemcpyAsync(a->seg, a->ckpt + (size_t)sgi * a->snap, a->snap,
                           cudaMemcpyDeviceToDevice, ctx->stream));
        for (int j = 0; j < len; ++j) {
            char *sj = a->seg + (size_t)j * a->slot;
            const bool last = j + 1 == len;
            if (int rc = run_pass_snap(ctx, last ? PASS_MACROS_T : PASS_STATE | PASS_MACROS_T, sj,
                                       last ? nullptr : sj + a->slot, sj + a->snap))
                return rc;
        }
        // reverse through it, reading each state and its moments where they lie
        for (int j = len - 1; j >= 0; --j) {
            const char *sj = a->seg + (size_t)j * a->slot;
            CK(adj_d2q9_step(a->real, params_ptr(ctx), nx, ny, sj, sj + ctx->fbytes, sj + a->snap,
                             a->lf[cb], a->lpt, a->lg[cb], a->lS[cb], a->lf[cb ^ 1],
                             a->lg[cb ^ 1], a->lS[cb ^ 1], a->work, a->dpar, ctx->stream));
            cb ^= 1;
        }
    }
    // initial condition f = f^eq(phi0, mu(phi0))
    double *lphi0 = on_device ? dL_dphi0 : a->macro;
    CK(adj_d2q9_init(a->real, params_ptr(ctx), nx, ny, a->phi0, a->lf[cb], a->lpt, a->work, lphi0,
                     a->dpar, ctx->stream));
    double dp[3];
    CK(cudaMemcpyAsync(dp, a->dpar, sizeof dp, cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device)
        CK(cudaMemcpyAsync(dL_dphi0, lphi0, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    // leave the context at the final state
    if (int rc = restore(ctx, a->ckpt + (size_t)(a->nsteps / a->K) * a->snap,
                         (long long)(a->nsteps / a->K) * a->K))
        return rc;
    if (a->nsteps % a->K)
        if (int rc = lbm_step(ctx, a->nsteps % a->K)) return rc;
    const lbm_params &pr = ctx->prm;
    const double d2 = (pr.phi_l - pr.phi_v) * (pr.phi_l - pr.phi_v);
    grads[2] = dp[0];
    grads[3] = dp[1];
    grads[0] = dp[0] * 3.0 * pr.W / (2.0 * d2) + dp[1] * 12.0 / (pr.W * d2 * d2);
    // 1/tau_f with tau_f = 1/2 + M/(cs2 alpha): d(1/tau_f)/dM = -1/(tau_f^2 cs2 alpha)
    grads[1] = dp[2] * (-1.0 / (ctx->tau_f * ctx->tau_f * CS2 * ctx->alpha));
    return LBM_OK;
}

void lbm_adjoint_destroy(lbm_adjoint *a)
{
    if (!a) return;
    cudaSetDevice(a->ctx->device);
    cudaStreamSynchronize(a->ctx->stream);
    a->ctx->recentre = 1;
    adjoint_free(a);
}

}  // extern "C"
