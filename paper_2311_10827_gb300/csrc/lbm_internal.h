// Internal declarations shared by the library's translation units.
// Not part of the public ABI (see include/lbm.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

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

// One CTA's partial diagnostics (8 doubles, FP64 whatever the precision).
struct DiagPartial {
    double sum_phi, E, u2max, mu_min, mu_max, budget, nonfinite, pad;
};

// What a pass over the grid does (bit set).
enum : int {
    PASS_STATE = 1,   // write post-collision f*, g* and S (a time step)
    PASS_MACROS = 2,  // write phi, p, u, mu (FP64)
    PASS_DIAG = 4,    // per-CTA diagnostics partials
};

struct PassArgs {
    const void *f_src;
    void *f_dst;
    const void *g_src;
    void *g_dst;
    void *S;              // S_prev in
    void *S_out;          // S out (same node; may equal S: in place)
    double *out_phi, *out_p, *out_u, *out_mu;
    DiagPartial *partials;
};

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
};
// One CTA's tile of a batch: case, strip x0, rows [y0, yend), march direction.
struct BatchTile {
    int c, x0, y0, yend, dir;
};

// D2Q9 (kernels_d2q9.cu)
LaunchShape d2q9_shape(int nx, int ny, int num_sms);
cudaError_t d2q9_pass(int precision, int pass, const void *params, const PassArgs &a,
                      const LaunchShape &s, cudaStream_t st);
// one time step of every grid of a batch (strip width 128 or 64)
cudaError_t d2q9_batch_step(int precision, int width, const BatchCase *cases,
                            const BatchTile *tiles, int ntiles, int parity, cudaStream_t st);
cudaError_t d2q9_init(int precision, const void *params, const double *phi0, double *mu_tmp,
                      void *f, void *g, void *S, cudaStream_t st);
cudaError_t d2q9_get_state(int precision, int nx, int ny, const void *f, const void *g,
                           const void *S, double *fo, double *go, double *So, cudaStream_t st);
cudaError_t d2q9_set_state(int precision, int nx, int ny, void *f, void *g, void *S,
                           const double *fi, const double *gi, const double *Si,
                           cudaStream_t st);

// D3Q19 (kernels_d3q19.cu); a pass first writes phi into phi_work (N values
// at the context's precision)
LaunchShape d3q19_shape(int nx, int ny, int nz, int num_sms);
cudaError_t d3q19_pass(int precision, int pass, const void *params, const PassArgs &a,
                       const LaunchShape &s, void *phi_work, cudaStream_t st);
cudaError_t d3q19_init(int precision, const void *params, const double *phi0, double *mu_tmp,
                       void *f, void *g, void *S, cudaStream_t st);
cudaError_t d3q19_get_state(int precision, const void *params, const void *f, const void *g,
                            const void *S, double *fo, double *go, double *So, cudaStream_t st);
cudaError_t d3q19_set_state(int precision, const void *params, void *f, void *g, void *S,
                            const double *fi, const double *gi, const double *Si, cudaStream_t st);

// D2Q9 discrete adjoint (kernels_adjoint.cu); FP64 adjoint fields in the
// paper's convention; work holds 7 N doubles; dpar accumulates
// {dL/dkappa, dL/dbeta, dL/d(1/tau_f)}
cudaError_t adj_d2q9_seed(int N, const double *dphi, double *lf, double *lg, double *lS,
                          cudaStream_t st);
cudaError_t adj_d2q9_step(int precision, const void *params64, int nx, int ny, const void *f,
                          const void *g, const void *S, const double *phi, const double *mu,
                          const double *p, const double *u, const double *lf_in,
                          const double *lg_in, const double *lS_in, double *lf_out, double *lg_out,
                          double *lS_out, double *work, double *dpar, cudaStream_t st);
cudaError_t adj_d2q9_init(const void *params64, int nx, int ny, const double *phi0,
                          const double *lf, double *work, double *lphi0, double *dpar,
                          cudaStream_t st);

// diagnostics reduction (kernels_diag.cu): partials[n] -> out (one record)
cudaError_t diag_reduce(const DiagPartial *partials, int n, DiagPartial *out, cudaStream_t st);

}  // namespace wblbm
