// Discrete adjoint (reverse mode) of the D2Q9 time step, for gradients of a
// loss on the final order parameter with respect to the initial field phi0,
// the surface tension (through kappa and beta) and the mobility (through
// 1/tau_f).  Not in the paper: the derivative of the discrete map, stage by
// stage in reverse order.  Adjoint arithmetic, adjoint fields, the forward
// moments and the parameters are all in the context's precision R (FP64, or
// FP32 for the FP32 form: FP64 arithmetic runs at a small fraction of the
// FP32 rate on this GPU, so the FP32 adjoint does none per node); only the
// per-block sums of the parameter gradients are accumulated in FP64.
// Adjoint fields use the paper's convention
// (pre-collision populations f_i(x, t), [Q][N]).  The adjoint of f is kept
// as lf[i] + lpt: the adjoint of phi = sum_i f_i adds the same value to every
// direction of a node, so it is stored once per node (lpt) instead of being
// added into all Q arrays.
//
// One reverse step (state at time n, adjoint of the state at n + 1):
//   1. the forward moments of time n (phi, mu, p, u) come from the ordinary
//      moments pass (fields in the storage type);
//   2. adj_local: reverse streaming, then per node the reverse of both
//      collisions and of the moments, leaving the adjoint of g and S_prev,
//      the direct part of the adjoint of f, and the local adjoints of phi,
//      mu, grad(phi), grad(mu);
//   3. adj_mu_phi: the transpose of the gradient stencil maps the grad(mu)
//      adjoint onto mu (on a tile and its halo in shared memory), then
//      mu = psi'(phi) - kappa lap(phi) and phi = sum_i f_i are reversed
//      (the Laplacian is symmetric, the gradient antisymmetric).  adj_phi
//      does the last part alone for the initial condition.
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

// periodic wrap of a neighbour coordinate c in [-1, n] (every stencil here
// reaches one node at most)
__device__ __forceinline__ int wrapa(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

struct AdjGeom {
    int nx, ny;
    unsigned N;
};

__device__ __forceinline__ unsigned at(const AdjGeom &g, int x, int y, int dx, int dy)
{
    return (unsigned)wrapa(y + dy, g.ny) * g.nx + wrapa(x + dx, g.nx);
}

// isotropic gradient of a field at (x, y): (1/cs2) sum w_i c_i psi(x + c_i)
template <typename R>
__device__ __forceinline__ void grad_at(const AdjGeom &g, const R *psi, int x, int y, R &gx,
                                        R &gy)
{
    gx = R(0), gy = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R v = psi[at(g, x, y, cxa(i), cya(i))];
        gx += R(wa(i) * cxa(i) / CS2A) * v;
        gy += R(wa(i) * cya(i) / CS2A) * v;
    }
}

// one FP64 atomic per block for a per-thread partial: the block's sum is
// formed in R (warp shuffles, then the warps' sums through shared memory) and
// converted once; every thread of the block calls it
template <typename R>
__device__ __forceinline__ void block_add(R v, double *dst)
{
    __shared__ R part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();  // part[] may still be read by an earlier call
    if (lane == 0) part[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        R s = R(0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        if (s != R(0)) atomicAdd(dst, (double)s);
    }
}

// lambda_phi, lambda_mu, lambda_grad phi, lambda_grad mu and dL/d(1/tau_f);
// the FP32 form fits 80 registers (3 resident CTAs per SM instead of 2: the
// kernel waits on gathered loads, so more warps help)
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2)
    adj_local(const StepParams<R> P, AdjGeom geo, const R *__restrict__ f,
              const R *__restrict__ g, const R *__restrict__ phi, const R *__restrict__ mu,
              const R *__restrict__ pf, const R *__restrict__ uf, const R *__restrict__ lf_in,
                          const R *__restrict__ lpt_in, const R *__restrict__ lg_in,
                          const R *__restrict__ lS_in,
                          R *__restrict__ lf_out, R *__restrict__ lg_out, R *__restrict__ lS_out,
                          R *__restrict__ lphi, R *__restrict__ lmu, R *__restrict__ lgphi,
                          R *__restrict__ lgmu, double *dpar)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned N = geo.N;
    constexpr R IC = R(1.0 / CS2A);
    R itf_part = R(0);
    if (n < N) {
        const int x = n % geo.nx, y = n / geo.nx;
        const R ph = phi[n], m = mu[n], p = pf[n];
        const R u[2] = {uf[n], uf[N + n]};
        R gph[2], gmu[2];
        grad_at(geo, phi, x, y, gph[0], gph[1]);
        grad_at(geo, mu, x, y, gmu[0], gmu[1]);
        const R drho = P.drho, dnu = P.dnu;
        const R rho = P.rhov + (ph - P.phiv) * drho;
        const R nu = P.nuv + (ph - P.phiv) * dnu;
        const R itg = R(1) / (R(0.5) + nu * IC);
        const R itf = P.inv_tauf, alpha = P.alpha;
        const R F[2] = {-ph * gmu[0] + P.G[0], -ph * gmu[1] + P.G[1]};
        const R gr[2] = {drho * gph[0], drho * gph[1]};
        const R ugr = u[0] * gr[0] + u[1] * gr[1], uu = u[0] * u[0] + u[1] * u[1];

        // forward populations of time n at x (pull layout: f_i(x) stored at x - c_i)
        R fv[9], gv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const unsigned src = at(geo, x, y, -cxa(i), -cya(i));
            fv[i] = f[i * N + src];
            gv[i] = g[i * N + src];
        }
        if (sizeof(R) == 4) fv[0] += f[9 * N + n];  // FP32: the rest population's low word

        R lu[2] = {0, 0}, lF[2] = {0, 0}, lgr[2] = {0, 0}, lgp[2] = {0, 0};
        R lrho = 0, lp = 0, lSx = 0, litg = 0, lph = 0, lmux = 0, lsrc = 0;

        // CH collision: f* = (1 - 1/tau_f) f + f^eq/tau_f + w_i b_i (1.5 S - 0.5 S_prev)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const unsigned src = at(geo, x, y, cxa(i), cya(i));  // reverse streaming
            const R l = lf_in[i * N + src] + lpt_in[src];
            const R fe = i == 0 ? ph - R(1.0 - wa(0)) * alpha * m : R(wa(i)) * alpha * m;
            lf_out[i * N + n] = (R(1) - itf) * l;
            itf_part += l * (fe - fv[i]);
            lsrc += l * R(wa(i) * ba(i));
            const R lfe = l * itf;
            if (i == 0) {
                lph += lfe;
                lmux += -R(1.0 - wa(0)) * alpha * lfe;
            } else {
                lmux += R(wa(i)) * alpha * lfe;
            }
        }
        lSx += R(1.5) * lsrc + lS_in[n];
        lS_out[n] = R(-0.5) * lsrc;

        // NS collision
        R lgn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) lgn[i] = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const R l = lg_in[i * N + at(geo, x, y, cxa(i), cya(i))];
            const R w = R(wa(i));
            const R cF = R(cxa(i)) * F[0] + R(cya(i)) * F[1];
            const R cu = R(cxa(i)) * u[0] + R(cya(i)) * u[1];
            const R cg = R(cxa(i)) * gr[0] + R(cya(i)) * gr[1];
            const R gam = w * (ugr + cF * IC + (cu * cg - R(CS2A) * ugr) * IC);
            const R su = cu * IC + cu * cu * R(0.5 / (CS2A * CS2A)) - uu * R(0.5 / CS2A);
            const R ge = p * R((wa(i) - (i == 0 ? 1.0 : 0.0)) / CS2A) + rho * w * su;
            lgn[i] += (R(1) - itg) * l;
            litg += l * (ge - gv[i]) - R(0.5) * l * gam;
            const R lge = l * itg, lgam = l * (R(1) - R(0.5) * itg);
            lp += lge * R((wa(i) - (i == 0 ? 1.0 : 0.0)) / CS2A);
            lrho += lge * w * su;
            const int c[2] = {cxa(i), cya(i)};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                lu[a] += lge * rho * w * (R(c[a]) * IC + cu * R(c[a]) * IC * IC - u[a] * IC);
                lF[a] += lgam * w * R(c[a]) * IC;
                lu[a] += lgam * w * (gr[a] + (R(c[a]) * cg - R(CS2A) * gr[a]) * IC);
                lgr[a] += lgam * w * (u[a] + (cu * R(c[a]) - R(CS2A) * u[a]) * IC);
            }
        }
        lph += litg * (-(dnu * IC) * itg * itg);  // tau_g = 1/2 + nu(phi)/cs2
        // S = u.grad phi
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            lu[a] += lSx * gph[a];
            lgp[a] += lSx * u[a];
        }
        // p = cs2/(1-w0) [sum_{i!=0} g_i + u.grad rho/2 - rho w0 uu/(2 cs2)]
        {
            const R k = R(CS2A / (1.0 - wa(0)));
#pragma unroll
            for (int i = 1; i < 9; ++i) lgn[i] += k * lp;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                lu[a] += k * lp * (R(0.5) * gr[a] - rho * R(wa(0)) * u[a] * IC);
                lgr[a] += k * lp * R(0.5) * u[a];
            }
            lrho += k * lp * (-R(wa(0) / (2 * CS2A)) * uu);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) lgp[a] += drho * lgr[a];
        // u = (sum c g + F/2) / rho
        const R irho = R(1) / rho;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const R lj = lu[a] * irho;
#pragma unroll
            for (int i = 0; i < 9; ++i) lgn[i] += R(a == 0 ? cxa(i) : cya(i)) * lj;
            lF[a] += R(0.5) * lj;
            lrho += -lu[a] * u[a] * irho;
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
    // dL/d(1/tau_f): one FP64 atomic per block
    block_add(itf_part, dpar + 2);
}

// transpose of the gradient stencil: (G^T v)(y) = (1/cs2) sum_i w_i c_i . v(y - c_i)
template <typename R>
__device__ __forceinline__ R gradT_at(const AdjGeom &g, const R *v, int x, int y)
{
    R s = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const unsigned m = at(g, x, y, -cxa(i), -cya(i));
        s += R(wa(i) / CS2A) * (R(cxa(i)) * v[m] + R(cya(i)) * v[g.N + m]);
    }
    return s;
}

// symmetric Laplacian: (L v)(x) = (2/cs2) sum_i w_i (v(x + c_i) - v(x)), in R
template <typename R, typename V>
__device__ __forceinline__ R lap_at(const AdjGeom &g, const V *v, int x, int y)
{
    const R c = (R)v[(unsigned)y * g.nx + x];
    R s = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) s += R(2.0 * wa(i) / CS2A) * ((R)v[at(g, x, y, cxa(i), cya(i))] - c);
    return s;
}


// lambda_phi total (the part of lambda_f common to every direction, lpt_out);
// dL/dkappa, dL/dbeta
template <typename R, typename V>
__global__ void adj_phi(const StepParams<R> P, AdjGeom geo, const V *__restrict__ phi,
                        const R *__restrict__ lphi, const R *__restrict__ lgphi,
                        const R *__restrict__ lmu_tot, R *__restrict__ lpt_out, double *lphi_out,
                        double *dpar)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    R dk = R(0), db = R(0);
    if (n < geo.N) {
        const int x = n % geo.nx, y = n / geo.nx;
        const R ph = (R)phi[n], lm = lmu_tot[n];
        const R a = ph - P.phil, b = ph - P.phiv, c = ph - P.phibar;
        const R d2psi = R(4) * P.beta * (b * c + a * c + a * b);
        const R l = lphi[n] + gradT_at(geo, lgphi, x, y) + d2psi * lm -
                    P.kappa * lap_at<R>(geo, lmu_tot, x, y);
        dk = lm * (-lap_at<R>(geo, phi, x, y));
        db = lm * R(4) * a * b * c;
        if (lpt_out) lpt_out[n] = l;
        if (lphi_out) lphi_out[n] = (double)l;
    }
    block_add(dk, dpar + 0);
    block_add(db, dpar + 1);
}

// The mu and phi parts of a reverse step in one pass.  The block owns a 32 x 8
// tile (256 threads) and first forms lambda_mu_tot = lambda_mu + G^T
// lambda_grad_mu on the tile and a 1-node halo in shared memory (the halo
// recomputed by each block), then the phi adjoint of adj_phi from it.
constexpr int AMX = 32, AMY = 8, AHX = AMX + 2, AHY = AMY + 2;
template <typename R>
__global__ void __launch_bounds__(AMX *AMY)
    adj_mu_phi(const StepParams<R> P, AdjGeom geo, const R *__restrict__ phi,
               const R *__restrict__ lphi, const R *__restrict__ lgphi, const R *__restrict__ lmu,
               const R *__restrict__ lgmu, R *__restrict__ lpt_out, double *dpar)
{
    __shared__ R smu[AHX * AHY];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * AMX, y0 = blockIdx.y * AMY;
    for (int q = tid; q < AHX * AHY; q += AMX * AMY) {
        // any grid size: a full modulo for the (at most 2) halo coordinates
        int xx = (x0 - 1 + q % AHX) % geo.nx, yy = (y0 - 1 + q / AHX) % geo.ny;
        xx += xx < 0 ? geo.nx : 0;
        yy += yy < 0 ? geo.ny : 0;
        smu[q] = lmu[(unsigned)yy * geo.nx + xx] + gradT_at(geo, lgmu, xx, yy);
    }
    __syncthreads();
    const int x = x0 + tid % AMX, y = y0 + tid / AMX;
    R dk = R(0), db = R(0);
    if (x < geo.nx && y < geo.ny) {
        const unsigned n = (unsigned)y * geo.nx + x;
        const int c = (tid / AMX + 1) * AHX + tid % AMX + 1;
        const R ph = phi[n], lm = smu[c];
        const R a = ph - P.phil, b = ph - P.phiv, cc = ph - P.phibar;
        const R d2psi = R(4) * P.beta * (b * cc + a * cc + a * b);
        // symmetric Laplacian of lambda_mu_tot from the tile
        R lap = R(0);
#pragma unroll
        for (int i = 1; i < 9; ++i) lap += R(2.0 * wa(i) / CS2A) * (smu[c + cya(i) * AHX + cxa(i)] - lm);
        const R l = lphi[n] + gradT_at(geo, lgphi, x, y) + d2psi * lm - P.kappa * lap;
        dk = lm * (-lap_at<R>(geo, phi, x, y));
        db = lm * R(4) * a * b * cc;
        lpt_out[n] = l;
    }
    block_add(dk, dpar + 0);
    block_add(db, dpar + 1);
}

// initial condition f = f^eq(phi0, mu(phi0)): lambda_phi and lambda_mu from lambda_f
template <typename R>
__global__ void adj_init_local(const StepParams<R> P, AdjGeom geo, const R *__restrict__ lf,
                               const R *__restrict__ lpt, R *__restrict__ lphi,
                               R *__restrict__ lmu, R *__restrict__ lgphi)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= geo.N) return;
    const R alpha = P.alpha, lp = lpt[n];
    R l = -R(1.0 - wa(0)) * alpha * (lf[n] + lp);
#pragma unroll
    for (int i = 1; i < 9; ++i) l += R(wa(i)) * alpha * (lf[i * geo.N + n] + lp);
    lmu[n] = l;
    lphi[n] = lf[n] + lp;
    lgphi[n] = R(0);
    lgphi[geo.N + n] = R(0);
}

// adjoint of the final state for L(phi^N): lambda_f_i = dL/dphi for every i
// (all of it in the common part lpt)
template <typename R>
__global__ void adj_seed(unsigned N, const double *__restrict__ dphi, R *__restrict__ lf,
                         R *__restrict__ lpt, R *__restrict__ lg, R *__restrict__ lS)
{
    const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        lf[i * N + n] = R(0);
        lg[i * N + n] = R(0);
    }
    lpt[n] = (R)dphi[n];
    lS[n] = R(0);
}

template <typename R>
void adj_step_t(const StepParams<R> &P, AdjGeom geo, const R *f, const R *g, const R *phi,
                const R *mu, const R *p, const R *u, const R *lf_in, R *lpt, const R *lg_in,
                const R *lS_in, R *lf_out, R *lg_out, R *lS_out, R *work, double *dpar,
                cudaStream_t st)
{
    const unsigned N = geo.N;
    R *lphi = work, *lmu = work + N, *lgphi = work + 2 * (size_t)N, *lgmu = work + 4 * (size_t)N;
    const unsigned nb = (N + 255) / 256;
    adj_local<R><<<nb, 256, 0, st>>>(P, geo, f, g, phi, mu, p, u, lf_in, lpt, lg_in, lS_in,
                                     lf_out, lg_out, lS_out, lphi, lmu, lgphi, lgmu, dpar);
    // lpt is read (gathered) by adj_local above and rewritten here
    const dim3 tiles((geo.nx + AMX - 1) / AMX, (geo.ny + AMY - 1) / AMY);
    adj_mu_phi<R><<<tiles, AMX * AMY, 0, st>>>(P, geo, phi, lphi, lgphi, lmu, lgmu, lpt, dpar);
}

template <typename R>
void adj_init_t(const StepParams<R> &P, AdjGeom geo, const double *phi0, const R *lf,
                const R *lpt, R *work, double *lphi0, double *dpar, cudaStream_t st)
{
    const unsigned N = geo.N;
    R *lphi = work, *lmu = work + N, *lgphi = work + 2 * (size_t)N;
    const unsigned nb = (N + 255) / 256;
    adj_init_local<R><<<nb, 256, 0, st>>>(P, geo, lf, lpt, lphi, lmu, lgphi);
    adj_phi<R, double><<<nb, 256, 0, st>>>(P, geo, phi0, lphi, lgphi, lmu, nullptr, lphi0, dpar);
}

template <typename R>
void adj_step_r(const void *params, AdjGeom geo, const void *f, const void *g, const void *mom,
                const void *lf_in, void *lpt, const void *lg_in, const void *lS_in, void *lf_out,
                void *lg_out, void *lS_out, void *work, double *dpar, cudaStream_t st)
{
    const R *m = static_cast<const R *>(mom);
    const size_t N = geo.N;
    adj_step_t<R>(*static_cast<const StepParams<R> *>(params), geo, static_cast<const R *>(f),
                  static_cast<const R *>(g), m, m + N, m + 2 * N, m + 3 * N,
                  static_cast<const R *>(lf_in), static_cast<R *>(lpt),
                  static_cast<const R *>(lg_in), static_cast<const R *>(lS_in),
                  static_cast<R *>(lf_out), static_cast<R *>(lg_out), static_cast<R *>(lS_out),
                  static_cast<R *>(work), dpar, st);
}

}  // namespace

cudaError_t adj_d2q9_seed(int real, int N, const double *dphi, void *lf, void *lpt, void *lg,
                          void *lS, cudaStream_t st)
{
    if (real == 0)
        adj_seed<double><<<(N + 255) / 256, 256, 0, st>>>((unsigned)N, dphi, (double *)lf,
                                                          (double *)lpt, (double *)lg, (double *)lS);
    else
        adj_seed<float><<<(N + 255) / 256, 256, 0, st>>>((unsigned)N, dphi, (float *)lf,
                                                         (float *)lpt, (float *)lg, (float *)lS);
    return cudaGetLastError();
}

cudaError_t adj_d2q9_step(int real, const void *params, int nx, int ny, const void *f,
                          const void *g, const void *moments, const void *lf_in, void *lpt,
                          const void *lg_in, const void *lS_in, void *lf_out, void *lg_out,
                          void *lS_out, void *work, double *dpar, cudaStream_t st)
{
    const AdjGeom geo{nx, ny, (unsigned)((size_t)nx * ny)};
    if (real == 0)
        adj_step_r<double>(params, geo, f, g, moments, lf_in, lpt, lg_in, lS_in, lf_out, lg_out,
                           lS_out, work, dpar, st);
    else
        adj_step_r<float>(params, geo, f, g, moments, lf_in, lpt, lg_in, lS_in, lf_out, lg_out,
                          lS_out, work, dpar, st);
    return cudaGetLastError();
}

cudaError_t adj_d2q9_init(int real, const void *params, int nx, int ny, const double *phi0,
                          const void *lf, const void *lpt, void *work, double *lphi0, double *dpar,
                          cudaStream_t st)
{
    const AdjGeom geo{nx, ny, (unsigned)((size_t)nx * ny)};
    if (real == 0)
        adj_init_t<double>(*static_cast<const StepParams<double> *>(params), geo, phi0,
                           (const double *)lf, (const double *)lpt, (double *)work, lphi0, dpar,
                           st);
    else
        adj_init_t<float>(*static_cast<const StepParams<float> *>(params), geo, phi0,
                          (const float *)lf, (const float *)lpt, (float *)work, lphi0, dpar, st);
    return cudaGetLastError();
}

}  // namespace wblbm
