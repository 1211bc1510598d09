// Internal declarations shared by the library's translation units.
// Not part of the public ABI (see include/lbm.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

namespace wblbm {

// Scalars of one run in the compute type T (derived on the host from the
// paper's parameters; see lbm_create).
template <typename T>
struct StepParams {
    int nx, ny, nz;
    long long N;         // nodes
    T kappa, beta;       // Eqs. beta, suiface_tension
    T phil, phiv, phibar;
    T alpha, inv_tauf;   // Eq. H_i, Eq. mobility
    T rhov, drho;        // rho = rhov + (phi - phiv) * drho
    T nuv, dnu;          // nu  = nuv  + (phi - phiv) * dnu  (Eq. vis)
    T G[3];              // body force
};

// ------------------------------------------------ parameters (host only)

// The checks every entry point taking (grid, lattice, params) applies.
inline int validate_problem(const lbm_grid *g, int lattice, const lbm_params *p)
{
    auto finite_pos = [](double v) { return isfinite(v) && v > 0.0; };
    if (!g || !p) return LBM_ERR_INVALID_ARG;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return LBM_ERR_INVALID_ARG;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) return LBM_ERR_INVALID_ARG;
    if (lattice == LBM_D2Q9 && g->nz != 1) return LBM_ERR_INVALID_ARG;
    // population offsets are 32-bit in the kernels (up to 20 arrays: the 19
    // D3Q19 populations and the FP32 rest population's low word)
    if ((long long)g->nx * g->ny * g->nz * 20 >= (1LL << 32)) return LBM_ERR_INVALID_ARG;
    if (!finite_pos(p->W) || !isfinite(p->sigma) || p->sigma < 0.0) return LBM_ERR_INVALID_ARG;
    if (!finite_pos(p->M)) return LBM_ERR_INVALID_ARG;
    if (p->tau_f == 0.0) {
        if (!finite_pos(p->alpha)) return LBM_ERR_INVALID_ARG;
    } else if (!isfinite(p->tau_f) || p->tau_f <= 0.5) {
        return LBM_ERR_INVALID_ARG;
    }
    if (!isfinite(p->phi_l) || !isfinite(p->phi_v) || p->phi_l == p->phi_v)
        return LBM_ERR_INVALID_ARG;
    if (!finite_pos(p->rho_l) || !finite_pos(p->rho_v)) return LBM_ERR_INVALID_ARG;
    if (!finite_pos(p->nu_l) || !finite_pos(p->nu_v)) return LBM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(p->body_force[a])) return LBM_ERR_INVALID_ARG;
    if (p->precision != LBM_FP64 && p->precision != LBM_FP32 &&
        p->precision != LBM_FP32_F16OFF && p->precision != LBM_FP32_BF16OFF)
        return LBM_ERR_INVALID_ARG;
    // 16-bit offset storage is built for the D3Q19 path
    if ((p->precision == LBM_FP32_F16OFF || p->precision == LBM_FP32_BF16OFF) &&
        lattice != LBM_D3Q19)
        return LBM_ERR_INVALID_ARG;
    if (p->diag_every < 0) return LBM_ERR_INVALID_ARG;
    return LBM_OK;
}

// Eqs. beta and suiface_tension solved for kappa and beta; Eq. mobility
// (tau_f from M and alpha, or alpha from M and a given tau_f).
struct Derived {
    double kappa, beta, tau_f, alpha;
};
inline Derived derive_params(const lbm_params &p)
{
    const double cs2 = 1.0 / 3.0;
    const double d2 = (p.phi_l - p.phi_v) * (p.phi_l - p.phi_v);
    Derived d;
    d.kappa = 3.0 * p.W * p.sigma / (2.0 * d2);
    d.beta = 12.0 * p.sigma / (p.W * d2 * d2);
    if (p.tau_f == 0.0) {
        d.alpha = p.alpha;
        d.tau_f = 0.5 + p.M / (cs2 * p.alpha);
    } else {
        d.tau_f = p.tau_f;
        d.alpha = p.M / (cs2 * (p.tau_f - 0.5));
    }
    return d;
}

// One CTA's partial diagnostics (8 doubles, FP64 whatever the precision).
struct DiagPartial {
    double sum_phi, E, u2max, mu_min, mu_max, budget, nonfinite, pad;
};

// What a pass over the grid does (bit set).
enum : int {
    PASS_STATE = 1,   // write post-collision f*, g* and S (a time step)
    PASS_MACROS = 2,  // write phi, p, u, mu (FP64)
    PASS_DIAG = 4,    // per-CTA diagnostics partials
    PASS_MACROS_T = 8,  // write phi, p, u, mu in the storage type (D2Q9 only;
                        // alone or with PASS_STATE: the moments of the source state)
};

struct PassArgs {
    const void *f_src;
    void *f_dst;
    const void *g_src;
    void *g_dst;
    void *S;              // S_prev in
    void *S_out;          // S out (same node; may equal S: in place)
    double *out_phi, *out_p, *out_u, *out_mu;
    void *mt_phi, *mt_p, *mt_u, *mt_mu;  // PASS_MACROS_T: all four, storage type
    DiagPartial *partials;
    // FP32 equilibrium shift a (see below): of the source buffer, of the
    // destination buffer (written by the step) and the target for new writes
    const float *eqs_src;
    float *eqs_dst;
    const float *eqs_target;
    int flip;  // step parity: D2Q9 row tiles reverse their march direction on odd steps
};

// The kernels' scalars of a problem in the compute type T.
template <typename T>
void fill_step_params(StepParams<T> &P, const lbm_grid &g, const lbm_params &p, const Derived &d)
{
    const double dphi = p.phi_l - p.phi_v;
    P.nx = g.nx;
    P.ny = g.ny;
    P.nz = g.nz;
    P.N = (long long)g.nx * g.ny * g.nz;
    P.kappa = (T)d.kappa;
    P.beta = (T)d.beta;
    P.phil = (T)p.phi_l;
    P.phiv = (T)p.phi_v;
    P.phibar = (T)(0.5 * (p.phi_l + p.phi_v));
    P.alpha = (T)d.alpha;
    P.inv_tauf = (T)(1.0 / d.tau_f);
    P.rhov = (T)p.rho_v;
    P.drho = (T)((p.rho_l - p.rho_v) / dphi);
    P.nuv = (T)p.nu_v;
    P.dnu = (T)((p.nu_l - p.nu_v) / dphi);
    for (int a = 0; a < 3; ++a) P.G[a] = (T)p.body_force[a];
}

// FP32 storage holds the f populations shifted by a uniform equilibrium
// a = alpha mu_ref: f~_i = f_i - w_i a (i != 0), f~_0 = f_0 + (1 - w_0) a.  A
// uniform shift of mu in f^eq is an exact symmetry of the discrete step (it
// streams unchanged, relaxes unchanged, and leaves phi = sum_i f_i and every
// other moment the step uses unchanged), so it is free to choose; with mu_ref
// near the equilibrium chemical potential the stored moving populations are
// small and their per-step changes are not lost to FP32 rounding.  Each
// context keeps {a of buffer 0, a of buffer 1, target} on the device.

struct LaunchShape {
    int rows;      // rows per CTA (2D march length)
    int grid_x, grid_y;
    int nblocks;
    int variant;   // kernel variant (strip width) where several exist
};

// One grid of a batch (device-resident table): parameters in both
// precisions, the two population buffers of f and g, S_prev and the S output.
struct BatchCase {
    StepParams<double> pd;
    StepParams<float> pf;
    void *f[2], *g[2];
    void *S, *S_out;
    float *eqs;    // the grid's equilibrium shifts {buffer 0, buffer 1, target, next target}
    int recentre;  // FP32: batch diagnostics move the target to the middle of the mu range
};
// One CTA's tile of a batch: case, strip x0, rows [y0, yend), march direction.
struct BatchTile {
    int c, x0, y0, yend, dir;
};

// D2Q9 (kernels_d2q9.cu)
LaunchShape d2q9_shape(int nx, int ny, int num_sms);
// Shared-memory attributes of the staging multi-step D2Q9 kernels on the
// current device (dynamic size and carveout).
cudaError_t d2q9_prepare();
cudaError_t d2q9_pass(int precision, int pass, const void *params, const PassArgs &a,
                      const LaunchShape &s, cudaStream_t st);
// one time step of every grid of a batch (strip width 128 or 64); with
// partials (one record per tile) the step also writes the FP64 diagnostics
// partials of its source state
cudaError_t d2q9_batch_step(int precision, int width, const BatchCase *cases,
                            const BatchTile *tiles, int ntiles, int parity, DiagPartial *partials,
                            cudaStream_t st);
// per-grid records from the tiles' partials (tile0[c] .. tile0[c + 1] are
// grid c's tiles); FP32: also moves each grid's shift target
cudaError_t d2q9_batch_reduce(int precision, const DiagPartial *partials, const int *tile0,
                              const BatchCase *cases, int ncases, DiagPartial *records,
                              cudaStream_t st);

// Several time steps of a batch in one cooperative launch (a queue of
// (step, tile) pairs; see d2q9_batch_persist_kernel).
constexpr int PERSIST_STEP_CAP = 1024;  // steps per multi-step launch (longer runs split)
constexpr int PERSIST_NBMAX = 16;
struct PersistArgs {
    const BatchCase *cases;
    const BatchTile *tiles;
    const int *nbr;    // per tile PERSIST_NBMAX + 1 ints: the count of the tiles its
                       // stencil reaches, then their indices (index ntiles: the spare
                       // counter nothing sets; fault-injection tests)
    const int *tile0;  // ncases + 1: first tile of each grid
    int ntiles, ncases, parity0, nsteps;  // nsteps * ntiles < 2^31
    int diag_k;        // step of the launch that carries the diagnostics, or -1
    int *ctr;          // 4 counters, then flags (= ctr + 4): ntiles + 1 step
                       // counters, then case_ctr (= flags + ntiles + 1):
                       // ncases counters, then step_done (= case_ctr + ncases):
                       // PERSIST_STEP_CAP counters; nctr ints, all zero at the launch
    int *ctr_next;     // the next launch's set of nctr ints, zeroed by this one
    int nctr;
    int *flags;
    int *case_ctr;     // per grid: tiles done with the diagnostics step
    int *step_done;    // per step of the launch: tiles done with it
    int stall_tile;    // fault injection: this tile always waits (else -1)
    int *err;          // device word set by a wait that timed out (never cleared here)
    int *err_host;     // mapped host word set with it (may be null)
    DiagPartial *partials;  // ntiles
    DiagPartial *records;   // ncases (device-visible; mapped host memory allowed)
};
// seg (FP32): the variant that stages the pulls as row segments, for
// batches whose grids all have rows of a multiple of 4 nodes.
cudaError_t d2q9_batch_persist(int precision, int width, bool seg, const PersistArgs &pa,
                               int nctas, cudaStream_t st);
int d2q9_batch_persist_ctas_per_sm(int precision, int width, bool seg);
cudaError_t d2q9_init(int precision, const void *params, const double *phi0, double *mu_tmp,
                      void *f, void *g, void *S, cudaStream_t st);
cudaError_t d2q9_get_state(int precision, int nx, int ny, const void *f, const void *g,
                           const void *S, const float *eqs, double *fo, double *go, double *So,
                           cudaStream_t st);
cudaError_t d2q9_set_state(int precision, int nx, int ny, void *f, void *g, void *S,
                           const double *fi, const double *gi, const double *Si,
                           cudaStream_t st);

// D3Q19 (kernels_d3q19.cu); a pass first writes phi into phi_work (N values
// at the context's precision)
LaunchShape d3q19_shape(int nx, int ny, int nz, int num_sms, int ctas_per_sm);
// resident CTAs per SM of the time-step kernel (occupancy query)
int d3q19_ctas_per_sm(int precision);
int d3q19_off_ctas_per_sm(int codec);
cudaError_t d3q19_pass(int precision, int pass, const void *params, const PassArgs &a,
                       const LaunchShape &s, void *phi_work, cudaStream_t st);
cudaError_t d3q19_init(int precision, const void *params, const double *phi0, double *mu_tmp,
                       void *f, void *g, void *S, cudaStream_t st);
cudaError_t d3q19_get_state(int precision, const void *params, const void *f, const void *g,
                            const void *S, const float *eqs, double *fo, double *go, double *So,
                            cudaStream_t st);
cudaError_t d3q19_set_state(int precision, const void *params, void *f, void *g, void *S,
                            const double *fi, const double *gi, const double *Si, cudaStream_t st);

// FP64 chemical potential of an initial phi field (Eq. chemical_potencial)
cudaError_t d3q19_init_mu_fp64(const void *params, const double *phi0, double *mu, cudaStream_t st);

// Populations stored as 16-bit offsets from their equilibria
// (kernels_d3q19_off.cu).  One parity of the state: the f buffer holds the
// Q offset arrays (u16), then D + 4 FP32 arrays (phi, mu, p, u, and the
// part of the next step's phi that does not depend on the offsets), then
// the two FP32 scales (s_f, s_g); the g buffer holds the Q offset arrays.
enum : int { OFFSET_F16 = 0, OFFSET_BF16 = 1 };
constexpr float OFFSET_SCALE_FLOOR = 1.0f / 65536.0f;  // 2^-16
constexpr float OFFSET_HEADROOM = 4096.0f;             // max |stored| after a refresh
struct OffsetLayout {
    size_t mac_off, sc_off, fbytes, gbytes;
};
__host__ __device__ inline OffsetLayout offset_layout(long long N, int Q, int D)
{
    const size_t n = (size_t)N, a = 256;
    OffsetLayout L;
    L.mac_off = ((size_t)Q * n * 2 + a - 1) / a * a;
    L.sc_off = L.mac_off + (((size_t)(D + 4) * n * 4 + a - 1) / a * a);
    L.fbytes = L.sc_off + a;
    L.gbytes = (size_t)Q * n * 2;
    return L;
}
cudaError_t d3q19_off_pass(int codec, int pass, const void *params32, const PassArgs &a,
                           const LaunchShape &s, void *phi_work, const float *target,
                           cudaStream_t st);
cudaError_t d3q19_off_init(int codec, const void *params64, const void *params32,
                           const double *phi0, double *mu_tmp, void *f, void *g, void *S,
                           const float *target_host, cudaStream_t st);
cudaError_t d3q19_off_get_state(int codec, const void *params32, const void *f, const void *g,
                                const void *S, double *fo, double *go, double *So, cudaStream_t st);
cudaError_t d3q19_off_set_state(int codec, const void *params32, void *f, void *g, void *S,
                                const double *fi, const double *gi, const double *Si,
                                const float *target_host, cudaStream_t st);
cudaError_t d3q19_off_poke(int codec, const void *params32, void *f, void *g, int field, int i,
                           size_t m, double value, cudaStream_t st);
// new target scales from the largest stored offsets of the state (f, g);
// maxbits: 2 device words of scratch; target: the 2 device target scales
cudaError_t offset_refresh(int codec, long long N, int Q, const void *f, const void *g,
                           unsigned *maxbits, float *target, int num_sms, cudaStream_t st);

// D2Q9 discrete adjoint (kernels_adjoint.cu) in the paper's convention.
// Adjoint fields (lf, lg [Q][N], lS [N], work 7 N) are FP64 when real == 0
// (the FP64 form) and FP32 when real == 1 (the FP32 form); the forward
// moments (phi, mu, p, u) are FP64; dpar accumulates in FP64
// {dL/dkappa, dL/dbeta, dL/d(1/tau_f)}.
// The adjoint of f is lf[i] + lpt (lpt [N]: the part common to every
// direction, the adjoint of phi = sum_i f_i); a step reads and rewrites lpt.
cudaError_t adj_d2q9_seed(int real, int N, const double *dphi, void *lf, void *lpt, void *lg,
                          void *lS, cudaStream_t st);
// real: 0 FP64, 1 FP32 (the context's storage type R); params: StepParams<R>;
// moments: phi, mu, p (N each) and u (2N) of the forward state, in R, as
// the PASS_MACROS_T pass writes them.
cudaError_t adj_d2q9_step(int real, const void *params, int nx, int ny, const void *f,
                          const void *g, const void *moments, const void *lf_in, void *lpt,
                          const void *lg_in, const void *lS_in, void *lf_out, void *lg_out,
                          void *lS_out, void *work, double *dpar, cudaStream_t st);
cudaError_t adj_d2q9_init(int real, const void *params, int nx, int ny, const double *phi0,
                          const void *lf, const void *lpt, void *work, double *lphi0, double *dpar,
                          cudaStream_t st);

// diagnostics reduction (kernels_diag.cu): partials[n] -> out (one record)
cudaError_t diag_reduce(const DiagPartial *partials, int n, DiagPartial *out, cudaStream_t st);
// new equilibrium-shift target alpha (mu_min + mu_max) / 2 from a reduced
// diagnostics record (kept if the record is not finite)
cudaError_t eq_recentre(const DiagPartial *rec, double alpha, float *target, cudaStream_t st);

}  // namespace wblbm
