// Discrete adjoint (reverse mode) of the D2Q9 time step, for gradients of a
// loss on the final order parameter with respect to the initial field phi0,
// the surface tension (through kappa and beta) and the mobility (through
// 1/tau_f).  Not in the paper: the derivative of the discrete map, stage by
// stage in reverse order.  Adjoint arithmetic is FP64; the forward state is
// read at its own precision.  Adjoint fields use the paper's convention
// (pre-collision populations f_i(x, t), [Q][N]).
//
// One reverse step (state at time n, adjoint of the state at n + 1):
//   1. the forward moments of time n (phi, mu, p, u) come from the ordinary
//      moments pass (FP64 fields);
//   2. adj_local: reverse streaming, then per node the reverse of both
//      collisions and of the moments, leaving the adjoint of g and S_prev,
//      the direct part of the adjoint of f, and the local adjoints of phi,
//      mu, grad(phi), grad(mu);
//   3. adj_mu: the transpose of the gradient stencil maps the grad(mu)
//      adjoint onto mu;
//   4. adj_phi: mu = psi'(phi) - kappa lap(phi) and phi = sum_i f_i are
//      reversed (the Laplacian is symmetric, the gradient antisymmetric).
#include <float.h>
#include <math.h>

#include "lbm_internal.h"

namespace wblbm {
namespace {

__host__ __device__ constexpr int cxa(int i)
{
    return (i == 2 || i == 5 || i == 8) ? 1 : ((i == 4 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cya(int i)
{
    return (i == 3 || i == 5 || i == 6) ? 1 : ((i == 1 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr double wa(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
__host__ __device__ constexpr double ba(int i) { return i == 0 ? -2.0 : (i <= 4 ? -0.5 : 1.0); }
constexpr double CS2A = 1.0 / 3.0;

__device__ __forceinline__ int wrapa(int c, int n)
{
    int r = c % n;
    return r < 0 ? r + n : r;
}

struct AdjGeom {
    int nx, ny;
    unsigned N;
};

__device__ __forceinline__ unsigned at(const AdjGeom &g, int x, int y, int dx, int dy)
{
    return (unsigned)wrapa(y + dy, g.ny) * g.nx + wrapa(x + dx, g.nx);
}

// isotropic gradient of an FP64 field at (x, y): (1/cs2) sum w_i c_i psi(x + c_i)
__device__ __forceinline__ void grad_at(const AdjGeom &g, const double *psi, int x, int y,
                                        double &gx, double &gy)
{
    gx = 0.0, gy = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const double v = psi[at(g, x, y, cxa(i), cya(i))];
        gx += wa(i) * cxa(i) * v;
        gy += wa(i) * cya(i) * v;
    }
    gx /= CS2A;
    gy /= CS2A;
}

// lambda_phi, lambda_mu, lambda_grad phi, lambda_grad mu and dL/d(1/tau_f)
template <typename T>
__global__ void adj_local(const StepParams<double> P, AdjGeom geo, const T *__restrict__ f,
                          const T *__restrict__ g, const T *__restrict__ S, int rest_pair,
                          const double *__restrict__ phi, const double *__restrict__ mu,
                          const double *__restrict__ pf, const double *__restrict__ uf,
                          const double *__restrict__ lf_in, const double *__restrict__ lg_in,
                          const double *__restrict__ lS_in, double *__restrict__ lf_out,
                          double *__restrict__ lg_out, double *__restrict__ lS_out,
                          double *__restrict__ lphi, double *__restrict__ lmu,
                          double *__restrict__ lgphi, double *__restrict__ lgmu, double *dpar)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned N = geo.N;
    double itf_part = 0.0;
    if (n < N) {
        const int x = n % geo.nx, y = n / geo.nx;
        const double ph = phi[n], m = mu[n], p = pf[n];
        const double u[2] = {uf[n], uf[N + n]};
        double gph[2], gmu[2];
        grad_at(geo, phi, x, y, gph[0], gph[1]);
        grad_at(geo, mu, x, y, gmu[0], gmu[1]);
        const double drho = P.drho, dnu = P.dnu;
        const double rho = P.rhov + (ph - P.phiv) * drho;
        const double nu = P.nuv + (ph - P.phiv) * dnu;
        const double itg = 1.0 / (0.5 + nu / CS2A);
        const double itf = P.inv_tauf, alpha = P.alpha;
        const double F[2] = {-ph * gmu[0] + P.G[0], -ph * gmu[1] + P.G[1]};
        const double gr[2] = {drho * gph[0], drho * gph[1]};
        const double ugr = u[0] * gr[0] + u[1] * gr[1], uu = u[0] * u[0] + u[1] * u[1];

        // forward populations of time n at x (pull layout: f_i(x) stored at x - c_i)
        double fv[9], gv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const unsigned src = at(geo, x, y, -cxa(i), -cya(i));
            fv[i] = (double)f[i * N + src];
            gv[i] = (double)g[i * N + src];
        }
        if (rest_pair) fv[0] += (double)f[9 * N + n];
        const double Sprev = (double)S[n];
        (void)Sprev;

        double lu[2] = {0, 0}, lF[2] = {0, 0}, lgr[2] = {0, 0}, lgp[2] = {0, 0};
        double lrho = 0, lp = 0, lSx = 0, litg = 0, lph = 0, lmux = 0, lsrc = 0;

        // CH collision: f* = (1 - 1/tau_f) f + f^eq/tau_f + w_i b_i (1.5 S - 0.5 S_prev)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double l = lf_in[i * N + at(geo, x, y, cxa(i), cya(i))];  // reverse streaming
            const double fe = i == 0 ? ph - (1.0 - wa(0)) * alpha * m : wa(i) * alpha * m;
            lf_out[i * N + n] = (1.0 - itf) * l;
            itf_part += l * (fe - fv[i]);
            lsrc += l * wa(i) * ba(i);
            const double lfe = l * itf;
            if (i == 0) {
                lph += lfe;
                lmux += -(1.0 - wa(0)) * alpha * lfe;
            } else {
                lmux += wa(i) * alpha * lfe;
            }
        }
        lSx += 1.5 * lsrc + lS_in[n];
        lS_out[n] = -0.5 * lsrc;

        // NS collision
        double lgn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) lgn[i] = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double l = lg_in[i * N + at(geo, x, y, cxa(i), cya(i))];
            const double cF = cxa(i) * F[0] + cya(i) * F[1];
            const double cu = cxa(i) * u[0] + cya(i) * u[1];
            const double cg = cxa(i) * gr[0] + cya(i) * gr[1];
            const double gam = wa(i) * (ugr + cF / CS2A + (cu * cg - CS2A * ugr) / CS2A);
            const double ge = p / CS2A * (wa(i) - (i == 0 ? 1.0 : 0.0)) +
                              rho * wa(i) * (cu / CS2A + cu * cu / (2 * CS2A * CS2A) - uu / (2 * CS2A));
            lgn[i] += (1.0 - itg) * l;
            litg += l * (ge - gv[i]) - 0.5 * l * gam;
            const double lge = l * itg, lgam = l * (1.0 - 0.5 * itg);
            lp += lge * (wa(i) - (i == 0 ? 1.0 : 0.0)) / CS2A;
            lrho += lge * wa(i) * (cu / CS2A + cu * cu / (2 * CS2A * CS2A) - uu / (2 * CS2A));
            const int c[2] = {cxa(i), cya(i)};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                lu[a] += lge * rho * wa(i) * (c[a] / CS2A + cu * c[a] / (CS2A * CS2A) - u[a] / CS2A);
                lF[a] += lgam * wa(i) * c[a] / CS2A;
                lu[a] += lgam * wa(i) * (gr[a] + (c[a] * cg - CS2A * gr[a]) / CS2A);
                lgr[a] += lgam * wa(i) * (u[a] + (cu * c[a] - CS2A * u[a]) / CS2A);
            }
        }
        lph += litg * (-(dnu / CS2A) * itg * itg);  // tau_g = 1/2 + nu(phi)/cs2
        // S = u.grad phi
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            lu[a] += lSx * gph[a];
            lgp[a] += lSx * u[a];
        }
        // p = cs2/(1-w0) [sum_{i!=0} g_i + u.grad rho/2 - rho w0 uu/(2 cs2)]
        {
            const double k = CS2A / (1.0 - wa(0));
#pragma unroll
            for (int i = 1; i < 9; ++i) lgn[i] += k * lp;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                lu[a] += k * lp * (0.5 * gr[a] - rho * wa(0) * u[a] / CS2A);
                lgr[a] += k * lp * 0.5 * u[a];
            }
            lrho += k * lp * (-wa(0) * uu / (2 * CS2A));
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) lgp[a] += drho * lgr[a];
        // u = (sum c g + F/2) / rho
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const double lj = lu[a] / rho;
#pragma unroll
            for (int i = 0; i < 9; ++i) lgn[i] += (a == 0 ? cxa(i) : cya(i)) * lj;
            lF[a] += 0.5 * lj;
            lrho += -lu[a] * u[a] / rho;
        }
        // F = -phi grad mu + G
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            lph += -lF[a] * gmu[a];
            lgmu[a * N + n] = -ph * lF[a];
            lgphi[a * N + n] = lgp[a];
        }
        lph += drho * lrho;
#pragma unroll
        for (int i = 0; i < 9; ++i) lg_out[i * N + n] = lgn[i];
        lphi[n] = lph;
        lmu[n] = lmux;
    }
    // dL/d(1/tau_f): warp sum, one FP64 atomic per warp
    for (int o = 16; o > 0; o >>= 1) itf_part += __shfl_xor_sync(0xffffffffu, itf_part, o);
    if ((threadIdx.x & 31) == 0 && itf_part != 0.0) atomicAdd(dpar + 2, itf_part);
}

// transpose of the gradient stencil: (G^T v)(y) = (1/cs2) sum_i w_i c_i . v(y - c_i)
__device__ __forceinline__ double gradT_at(const AdjGeom &g, const double *v, int x, int y)
{
    double s = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const unsigned m = at(g, x, y, -cxa(i), -cya(i));
        s += wa(i) * (cxa(i) * v[m] + cya(i) * v[g.N + m]);
    }
    return s / CS2A;
}

// symmetric Laplacian: (L v)(x) = (2/cs2) sum_i w_i (v(x + c_i) - v(x))
__device__ __forceinline__ double lap_at(const AdjGeom &g, const double *v, int x, int y)
{
    const double c = v[(unsigned)y * g.nx + x];
    double s = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) s += 2.0 * wa(i) * (v[at(g, x, y, cxa(i), cya(i))] - c);
    return s / CS2A;
}

__global__ void adj_mu(AdjGeom geo, const double *__restrict__ lmu, const double *__restrict__ lgmu,
                       double *__restrict__ lmu_tot)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= geo.N) return;
    const int x = n % geo.nx, y = n / geo.nx;
    lmu_tot[n] = lmu[n] + gradT_at(geo, lgmu, x, y);
}

// lambda_phi total; lambda_f += lambda_phi for every i; dL/dkappa, dL/dbeta
__global__ void adj_phi(const StepParams<double> P, AdjGeom geo, const double *__restrict__ phi,
                        const double *__restrict__ lphi, const double *__restrict__ lgphi,
                        const double *__restrict__ lmu_tot, double *__restrict__ lf_out,
                        double *lphi_out, double *dpar)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    double dk = 0.0, db = 0.0;
    if (n < geo.N) {
        const int x = n % geo.nx, y = n / geo.nx;
        const double ph = phi[n], lm = lmu_tot[n];
        const double a = ph - P.phil, b = ph - P.phiv, c = ph - P.phibar;
        const double d2psi = 4.0 * P.beta * (b * c + a * c + a * b);
        double l = lphi[n] + gradT_at(geo, lgphi, x, y) + d2psi * lm - P.kappa * lap_at(geo, lmu_tot, x, y);
        dk = lm * (-lap_at(geo, phi, x, y));
        db = lm * 4.0 * a * b * c;
        if (lf_out) {
#pragma unroll
            for (int i = 0; i < 9; ++i) lf_out[i * geo.N + n] += l;
        }
        if (lphi_out) lphi_out[n] = l;
    }
    for (int o = 16; o > 0; o >>= 1) {
        dk += __shfl_xor_sync(0xffffffffu, dk, o);
        db += __shfl_xor_sync(0xffffffffu, db, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (dk != 0.0) atomicAdd(dpar + 0, dk);
        if (db != 0.0) atomicAdd(dpar + 1, db);
    }
}

// initial condition f = f^eq(phi0, mu(phi0)): lambda_phi and lambda_mu from lambda_f
__global__ void adj_init_local(const StepParams<double> P, AdjGeom geo, const double *__restrict__ lf,
                               double *__restrict__ lphi, double *__restrict__ lmu,
                               double *__restrict__ lgphi)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= geo.N) return;
    double l = -(1.0 - wa(0)) * P.alpha * lf[n];
#pragma unroll
    for (int i = 1; i < 9; ++i) l += wa(i) * P.alpha * lf[i * geo.N + n];
    lmu[n] = l;
    lphi[n] = lf[n];
    lgphi[n] = 0.0;
    lgphi[geo.N + n] = 0.0;
}

// adjoint of the final state for L(phi^N): lambda_f_i = dL/dphi for every i
__global__ void adj_seed(unsigned N, const double *__restrict__ dphi, double *__restrict__ lf,
                         double *__restrict__ lg, double *__restrict__ lS)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double v = dphi[n];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        lf[i * N + n] = v;
        lg[i * N + n] = 0.0;
    }
    lS[n] = 0.0;
}

}  // namespace

cudaError_t adj_d2q9_seed(int N, const double *dphi, double *lf, double *lg, double *lS,
                          cudaStream_t st)
{
    adj_seed<<<(N + 255) / 256, 256, 0, st>>>((unsigned)N, dphi, lf, lg, lS);
    return cudaGetLastError();
}

cudaError_t adj_d2q9_step(int precision, const void *params64, int nx, int ny, const void *f,
                          const void *g, const void *S, const double *phi, const double *mu,
                          const double *p, const double *u, const double *lf_in,
                          const double *lg_in, const double *lS_in, double *lf_out, double *lg_out,
                          double *lS_out, double *work, double *dpar, cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params64);
    AdjGeom geo{nx, ny, (unsigned)((size_t)nx * ny)};
    const unsigned N = geo.N;
    double *lphi = work, *lmu = work + N, *lgphi = work + 2 * (size_t)N,
           *lgmu = work + 4 * (size_t)N, *lmu_tot = work + 6 * (size_t)N;
    const unsigned nb = (N + 255) / 256;
    if (precision == 0)
        adj_local<double><<<nb, 256, 0, st>>>(P, geo, (const double *)f, (const double *)g,
                                              (const double *)S, 0, phi, mu, p, u, lf_in, lg_in,
                                              lS_in, lf_out, lg_out, lS_out, lphi, lmu, lgphi,
                                              lgmu, dpar);
    else
        adj_local<float><<<nb, 256, 0, st>>>(P, geo, (const float *)f, (const float *)g,
                                             (const float *)S, 1, phi, mu, p, u, lf_in, lg_in,
                                             lS_in, lf_out, lg_out, lS_out, lphi, lmu, lgphi,
                                             lgmu, dpar);
    adj_mu<<<nb, 256, 0, st>>>(geo, lmu, lgmu, lmu_tot);
    adj_phi<<<nb, 256, 0, st>>>(P, geo, phi, lphi, lgphi, lmu_tot, lf_out, nullptr, dpar);
    return cudaGetLastError();
}

cudaError_t adj_d2q9_init(const void *params64, int nx, int ny, const double *phi0,
                          const double *lf, double *work, double *lphi0, double *dpar,
                          cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params64);
    AdjGeom geo{nx, ny, (unsigned)((size_t)nx * ny)};
    const unsigned N = geo.N;
    double *lphi = work, *lmu = work + N, *lgphi = work + 2 * (size_t)N;
    const unsigned nb = (N + 255) / 256;
    adj_init_local<<<nb, 256, 0, st>>>(P, geo, lf, lphi, lmu, lgphi);
    adj_phi<<<nb, 256, 0, st>>>(P, geo, phi0, lphi, lgphi, lmu, nullptr, lphi0, dpar);
    return cudaGetLastError();
}

}  // namespace wblbm
