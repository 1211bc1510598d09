// D2Q9 kernels of the well-balanced phase-field LBM (arXiv:2311.10827,
// Section 2.3) for sm_103a: the fused pull stream-collide step, the same
// pass writing macroscopic fields or diagnostics, the initial condition and
// the state exchange in the paper's convention.
//
// Storage (pull scheme, double buffer): a population buffer holds the
// post-collision values f_i*(x) of the previous step at their source node, so
// the paper's f_i(x, t) is f_i*(x - c_i).  Layout is SoA, [i][y][x].  S (the
// previous step's u.grad(phi), needed by the backward-difference reading of
// the (1/2) dt^2 d_t F_i term of Eq. BGK) is read and rewritten at the same
// node, so it needs no second buffer.
//
// Stencil chain.  grad(mu) at x needs mu at radius 1, mu needs phi at
// radius 2, and phi(y) = sum_i f_i*(y - c_i) needs the stored populations at
// radius 3.  A CTA owns a strip of TX columns and marches down `rows` rows,
// two rows per iteration (thread row ty = 0, 1).  phi rows (TX + 4 columns)
// and mu rows (TX + 2 columns) live in small shared-memory rings, so each
// stored f value is read once per strip apart from the 4-column halo (served
// by L2).  A thread's own output row was summed into phi by the same thread
// one iteration earlier, so its nine pulled f values stay in registers.
#include <float.h>
#include <math.h>

#include "lbm_internal.h"

namespace wblbm {
namespace {

// Velocity order of Eq. eq:ci (diagonals of length sqrt 2):
//   0 (0,0)  1 (0,-1)  2 (1,0)  3 (0,1)  4 (-1,0)
//   5 (1,1)  6 (-1,1)  7 (-1,-1)  8 (1,-1)
// weights 4/9 (rest), 1/9 (axis), 1/36 (diagonal).
__host__ __device__ constexpr int cxv(int i)
{
    return (i == 2 || i == 5 || i == 8) ? 1 : ((i == 4 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cyv(int i)
{
    return (i == 3 || i == 5 || i == 6) ? 1 : ((i == 1 || i == 7 || i == 8) ? -1 : 0);
}

constexpr int TYB = 2;  // thread rows per CTA (fixed by the register reuse above)

__device__ __forceinline__ int wrapi(int c, int n)
{
    int r = c % n;
    return r < 0 ? r + n : r;
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p)
{
    return __ldg(p);
}

// The nine populations arriving at (x, y): v[i] = src_i(x - cx_i, y - cy_i).
// rm/r0/rp are the row offsets of y-1, y, y+1; xm/x/xp the wrapped columns.
template <typename T>
__device__ __forceinline__ void pull9(const T *__restrict__ s, size_t N, size_t rm, size_t r0,
                                      size_t rp, int xm, int x, int xp, T v[9])
{
    v[0] = ldg(s + r0 + x);
    v[1] = ldg(s + 1 * N + rp + x);   // c = (0,-1) comes from y + 1
    v[2] = ldg(s + 2 * N + r0 + xm);  // c = (1,0)  comes from x - 1
    v[3] = ldg(s + 3 * N + rm + x);   // c = (0,1)  comes from y - 1
    v[4] = ldg(s + 4 * N + r0 + xp);  // c = (-1,0) comes from x + 1
    v[5] = ldg(s + 5 * N + rm + xm);  // c = (1,1)
    v[6] = ldg(s + 6 * N + rm + xp);  // c = (-1,1)
    v[7] = ldg(s + 7 * N + rp + xp);  // c = (-1,-1)
    v[8] = ldg(s + 8 * N + rp + xm);  // c = (1,-1)
}

// sum of the eight moving populations, fixed pairing (the rest population is
// added last so that phi = f_0 + s keeps the small terms exact in FP32)
template <typename T>
__device__ __forceinline__ T sum_moving(const T v[9])
{
    return ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
}

__device__ __forceinline__ void warp_reduce(double &sum0, double &sum1, double &mx, double &mn,
                                            double &mxu, double &sum2, double &bad)
{
    for (int o = 16; o > 0; o >>= 1) {
        sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
        sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
        sum2 += __shfl_xor_sync(0xffffffffu, sum2, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mxu = fmax(mxu, __shfl_xor_sync(0xffffffffu, mxu, o));
        bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, o));
    }
}

template <typename T, int TX, int PASS>
__global__ void __launch_bounds__(TX *TYB) d2q9_pass_kernel(const StepParams<T> P, PassArgs a,
                                                            int rows)
{
    constexpr int R = 2 * TYB + 3;  // ring depth: writes never hit a row still read
    constexpr int WP = TX + 4;      // phi ring width (halo 2)
    constexpr int WM = TX + 2;      // mu ring width (halo 1)
    __shared__ T phs[R * WP];
    __shared__ T mus[R * WM];

    const int nx = P.nx, ny = P.ny;
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * TX;
    const int y0 = blockIdx.y * rows;
    const int yend = min(y0 + rows, ny);
    const T *__restrict__ fsrc = static_cast<const T *>(a.f_src);
    const T *__restrict__ gsrc = static_cast<const T *>(a.g_src);

    // own column (phi ring index tx + 2, mu ring index tx + 1)
    const int xo = x0 + tx;
    const bool col_ok = xo < nx;
    const int xO = wrapi(xo, nx), xOm = wrapi(xo - 1, nx), xOp = wrapi(xo + 1, nx);
    // phi halo column handled by threads 0..3: ring index 0, 1, TX+2, TX+3
    const int jH = tx < 2 ? tx : TX + tx;
    const int cH = x0 - 2 + jH;
    const int xH = wrapi(cH, nx), xHm = wrapi(cH - 1, nx), xHp = wrapi(cH + 1, nx);
    // mu halo column handled by threads 0, 1: ring index 0 and TX+1
    const int jM = tx == 0 ? 0 : TX + 1;

    auto slot = [&](int row) { return (row - y0 + 2) % R; };  // row >= y0 - 2

    // phi at row `row` for the own column (keeping the pulled values) and the
    // halo columns.
    auto phi_row = [&](int row, T v[9]) {
        const int y = wrapi(row, ny);
        const size_t rm = (size_t)wrapi(row - 1, ny) * nx, r0 = (size_t)y * nx,
                     rp = (size_t)wrapi(row + 1, ny) * nx;
        T *ph = phs + slot(row) * WP;
        pull9(fsrc, N, rm, r0, rp, xOm, xO, xOp, v);
        ph[tx + 2] = v[0] + sum_moving(v);
        if (tx < 4) {
            T h[9];
            pull9(fsrc, N, rm, r0, rp, xHm, xH, xHp, h);
            ph[jH] = h[0] + sum_moving(h);
        }
    };

    // Eq. chemical_potencial with the Laplacian of Eq. Laplace, written as a
    // sum of differences (cancellation-friendly in FP32):
    // lap = (2/3) sum_axis (phi_n - phi) + (1/6) sum_diag (phi_n - phi).
    auto mu_at = [&](const T *pm, const T *p0, const T *pp, int j) -> T {
        // j is the mu ring index; the phi ring index of the same column is j+1
        const T c = p0[j + 1];
        const T ax = (p0[j + 2] - c) + (p0[j] - c) + (pp[j + 1] - c) + (pm[j + 1] - c);
        const T dg = (pp[j + 2] - c) + (pp[j] - c) + (pm[j + 2] - c) + (pm[j] - c);
        const T lap = T(2.0 / 3.0) * ax + T(1.0 / 6.0) * dg;
        const T bulk = T(4) * P.beta * (c - P.phil) * (c - P.phiv) * (c - P.phibar);
        return bulk - P.kappa * lap;
    };
    auto mu_row = [&](int row) {
        const T *pm = phs + slot(row - 1) * WP;
        const T *p0 = phs + slot(row) * WP;
        const T *pp = phs + slot(row + 1) * WP;
        T *mr = mus + slot(row) * WM;
        mr[tx + 1] = mu_at(pm, p0, pp, tx + 1);
        if (tx < 2) mr[jM] = mu_at(pm, p0, pp, jM);
    };

    double d_phi = 0.0, d_E = 0.0, d_u2 = 0.0, d_mumin = DBL_MAX, d_mumax = -DBL_MAX,
           d_bud = 0.0, d_bad = 0.0;

    // prologue: phi rows y0-2 .. y0+1 (the own row y0+ty keeps its values),
    // mu rows y0-1 .. y0
    T fcur[9], fnext[9];
    phi_row(y0 - 2 + ty, fnext);
    phi_row(y0 + ty, fcur);
    __syncthreads();
    mu_row(y0 - 1 + ty);
    __syncthreads();

    for (int r = y0; r < yend; r += TYB) {
        const int row = r + ty;
        const bool out_ok = col_ok && row < yend;
        // issue the loads of the own node first so they overlap the stencil work
        T gv[9];
        T Sprev = T(0);
        const int yw = wrapi(row, ny);
        const size_t nrow = (size_t)yw * nx;
        {
            const size_t rm = (size_t)wrapi(row - 1, ny) * nx,
                         rp = (size_t)wrapi(row + 1, ny) * nx;
            pull9(gsrc, N, rm, nrow, rp, xOm, xO, xOp, gv);
            if ((PASS & (PASS_STATE | PASS_DIAG)) && out_ok)
                Sprev = static_cast<const T *>(a.S)[nrow + xo];
        }
        phi_row(r + 2 + ty, fnext);
        __syncthreads();
        mu_row(r + 1 + ty);
        __syncthreads();

        if (out_ok) {
            const T *pm = phs + slot(row - 1) * WP;
            const T *p0 = phs + slot(row) * WP;
            const T *pp = phs + slot(row + 1) * WP;
            const T *mm = mus + slot(row - 1) * WM;
            const T *m0 = mus + slot(row) * WM;
            const T *mp = mus + slot(row + 1) * WM;
            const int j = tx + 2;  // phi ring index of the own column
            const int k = tx + 1;  // mu ring index of the own column

            // phi from the pulled values (Eq. order-parameter)
            const T snz = sum_moving(fcur);
            const T phi = fcur[0] + snz;
            const T mu = m0[k];
            // Eq. gradient: grad = 3 sum_{i!=0} w_i c_i Psi(x + c_i)
            //   = (1/3)(axis differences) + (1/12)(diagonal differences)
            const T gpx = T(1.0 / 3.0) * (p0[j + 1] - p0[j - 1]) +
                          T(1.0 / 12.0) * ((pp[j + 1] - pp[j - 1]) + (pm[j + 1] - pm[j - 1]));
            const T gpy = T(1.0 / 3.0) * (pp[j] - pm[j]) +
                          T(1.0 / 12.0) * ((pp[j + 1] - pm[j + 1]) + (pp[j - 1] - pm[j - 1]));
            const T gmx = T(1.0 / 3.0) * (m0[k + 1] - m0[k - 1]) +
                          T(1.0 / 12.0) * ((mp[k + 1] - mp[k - 1]) + (mm[k + 1] - mm[k - 1]));
            const T gmy = T(1.0 / 3.0) * (mp[k] - mm[k]) +
                          T(1.0 / 12.0) * ((mp[k + 1] - mm[k + 1]) + (mp[k - 1] - mm[k - 1]));

            // F = -phi grad(mu) + G; rho, nu linear in phi (Eq. vis)
            const T Fx = -phi * gmx + P.G[0];
            const T Fy = -phi * gmy + P.G[1];
            const T dphi = phi - P.phiv;
            const T rho = P.rhov + dphi * P.drho;
            const T nu = P.nuv + dphi * P.dnu;
            const T inv_rho = T(1) / rho;
            const T inv_taug = T(1) / (T(0.5) + T(3) * nu);  // nu = cs2 (tau_g - 1/2)

            // rho u = sum_i c_i g_i + F/2
            const T jx = (gv[2] - gv[4]) + ((gv[5] - gv[6]) + (gv[8] - gv[7]));
            const T jy = (gv[3] - gv[1]) + ((gv[5] + gv[6]) - (gv[7] + gv[8]));
            const T ux = (jx + T(0.5) * Fx) * inv_rho;
            const T uy = (jy + T(0.5) * Fy) * inv_rho;
            const T grx = P.drho * gpx, gry = P.drho * gpy;  // grad rho (chain rule)
            const T ugr = ux * grx + uy * gry;
            const T uu = ux * ux + uy * uy;
            // p = cs2/(1-w0) [sum_{i!=0} g_i + u.grad(rho)/2 + rho s_0(u)],
            // rho s_0 = -(2/3) rho |u|^2 for D2Q9
            const T p = T(0.6) * (sum_moving(gv) + T(0.5) * ugr - T(2.0 / 3.0) * rho * uu);
            const T S = ux * gpx + uy * gpy;  // u.grad(phi)

            if (PASS & PASS_DIAG) {
                const double u2 = (double)uu;
                d_phi += (double)phi;
                d_E += 0.5 * (double)rho * u2;
                d_u2 = fmax(d_u2, u2);
                d_mumin = fmin(d_mumin, (double)mu);
                d_mumax = fmax(d_mumax, (double)mu);
                d_bud += 1.5 * (double)S - 0.5 * (double)Sprev;
                if (!isfinite((double)phi) || !isfinite((double)p) || !isfinite(u2) ||
                    !isfinite((double)mu))
                    d_bad = 1.0;
            }
            if (PASS & PASS_MACROS) {
                const size_t n = nrow + xo;
                if (a.out_phi) a.out_phi[n] = (double)phi;
                if (a.out_p) a.out_p[n] = (double)p;
                if (a.out_mu) a.out_mu[n] = (double)mu;
                if (a.out_u) {
                    a.out_u[n] = (double)ux;
                    a.out_u[N + n] = (double)uy;
                }
            }
            if (PASS & PASS_STATE) {
                const size_t n = nrow + xo;
                T *__restrict__ fd = static_cast<T *>(a.f_dst);
                T *__restrict__ gd = static_cast<T *>(a.g_dst);
                static_cast<T *>(a.S)[n] = S;

                // CH population, Eq. BGK with Eq. H_i and Eq. F_i; the source
                // w_i b_i (1.5 S - 0.5 S_prev), b = -2, -1/2, 1 (rest, axis, diagonal).
                const T Sh = T(1.5) * S - T(0.5) * Sprev;
                const T am = P.alpha * mu;
                const T itf = P.inv_tauf;
                // f_0 - f_0^eq = (5/9) alpha mu - sum_{i!=0} f_i (no cancellation)
                fd[n] = fcur[0] - (T(5.0 / 9.0) * am - snz) * itf + T(4.0 / 9.0) * T(-2) * Sh;
                const T feqa = T(1.0 / 9.0) * am, srca = T(1.0 / 9.0) * T(-0.5) * Sh;
                const T feqd = T(1.0 / 36.0) * am, srcd = T(1.0 / 36.0) * Sh;
#pragma unroll
                for (int i = 1; i <= 4; ++i)
                    fd[i * N + n] = fcur[i] - (fcur[i] - feqa) * itf + srca;
#pragma unroll
                for (int i = 5; i <= 8; ++i)
                    fd[i * N + n] = fcur[i] - (fcur[i] - feqd) * itf + srcd;

                // hydrodynamic population, Eq. BGK-NS with Eqs. G_i, Siu, GGi.
                // G_i = (1 - 1/(2 tau_g)) w_i [u.grad rho + c_i.F/cs2
                //        + ((c_i.u)(c_i.grad rho) - cs2 u.grad rho)/cs2]; the two
                // u.grad rho terms cancel, leaving 3 w_i (1 - 1/(2 tau_g)) [c_i.F + (c_i.u)(c_i.grad rho)].
                const T kg = T(1) - T(0.5) * inv_taug;
                const T p3 = T(3) * p;
                {
                    const T geq0 = p3 * (T(4.0 / 9.0) - T(1)) +
                                   rho * T(4.0 / 9.0) * (T(-1.5) * uu);
                    gd[n] = gv[0] - (gv[0] - geq0) * inv_taug;  // G_0 = 0 (c_0 = 0)
                }
#pragma unroll
                for (int i = 1; i <= 8; ++i) {
                    const T w = i <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0);
                    const T cu = T(cxv(i)) * ux + T(cyv(i)) * uy;
                    const T cF = T(cxv(i)) * Fx + T(cyv(i)) * Fy;
                    const T cg = T(cxv(i)) * grx + T(cyv(i)) * gry;
                    const T geq = w * (p3 + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
                    const T Gi = T(3) * w * kg * (cF + cu * cg);
                    gd[i * N + n] = gv[i] - (gv[i] - geq) * inv_taug + Gi;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) fcur[i] = fnext[i];
    }

    if (PASS & PASS_DIAG) {
        warp_reduce(d_phi, d_E, d_u2, d_mumin, d_mumax, d_bud, d_bad);
        constexpr int NW = TX * TYB / 32;
        __shared__ double red[7][NW];
        const int lane = (ty * TX + tx) & 31, wid = (ty * TX + tx) >> 5;
        if (lane == 0) {
            red[0][wid] = d_phi;
            red[1][wid] = d_E;
            red[2][wid] = d_u2;
            red[3][wid] = d_mumin;
            red[4][wid] = d_mumax;
            red[5][wid] = d_bud;
            red[6][wid] = d_bad;
        }
        __syncthreads();
        if (wid == 0 && lane == 0) {
            DiagPartial o;
            o.sum_phi = 0.0;
            o.E = 0.0;
            o.u2max = 0.0;
            o.mu_min = DBL_MAX;
            o.mu_max = -DBL_MAX;
            o.budget = 0.0;
            o.nonfinite = 0.0;
            o.pad = 0.0;
            for (int w = 0; w < NW; ++w) {
                o.sum_phi += red[0][w];
                o.E += red[1][w];
                o.u2max = fmax(o.u2max, red[2][w]);
                o.mu_min = fmin(o.mu_min, red[3][w]);
                o.mu_max = fmax(o.mu_max, red[4][w]);
                o.budget += red[5][w];
                o.nonfinite = fmax(o.nonfinite, red[6][w]);
            }
            a.partials[blockIdx.y * gridDim.x + blockIdx.x] = o;
        }
    }
}

// ------------------------------------------------------------ initial state

// mu0 = psi'(phi0) - kappa lap(phi0) in FP64 (Eq. chemical_potencial)
__global__ void d2q9_init_mu(const StepParams<double> P, const double *__restrict__ phi,
                             double *__restrict__ mu)
{
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)P.N) return;
    const int nx = P.nx, ny = P.ny;
    const int x = (int)(n % nx), y = (int)(n / nx);
    auto at = [&](int dx, int dy) {
        return phi[(size_t)wrapi(y + dy, ny) * nx + wrapi(x + dx, nx)];
    };
    const double c = phi[n];
    const double ax = (at(1, 0) - c) + (at(-1, 0) - c) + (at(0, 1) - c) + (at(0, -1) - c);
    const double dg = (at(1, 1) - c) + (at(-1, 1) - c) + (at(1, -1) - c) + (at(-1, -1) - c);
    const double lap = (2.0 / 3.0) * ax + (1.0 / 6.0) * dg;
    mu[n] = 4.0 * P.beta * (c - P.phil) * (c - P.phiv) * (c - P.phibar) - P.kappa * lap;
}

// f_i(x, 0) = f_i^eq(phi0(x), mu0(x)) stored pre-shifted for the pull scheme:
// buffer_i(y) = f_i^eq at y + c_i.  g = 0, S = 0 (initial condition, R9).
template <typename T>
__global__ void d2q9_init_pop(const StepParams<double> P, const double *__restrict__ phi,
                              const double *__restrict__ mu, T *__restrict__ f,
                              T *__restrict__ g, T *__restrict__ S)
{
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)P.N) return;
    const size_t N = (size_t)P.N;
    const int nx = P.nx, ny = P.ny;
    const int x = (int)(n % nx), y = (int)(n / nx);
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                         1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int i = 0; i < 9; ++i) {
        const size_t m = (size_t)wrapi(y + cyv(i), ny) * nx + wrapi(x + cxv(i), nx);
        const double am = P.alpha * mu[m];
        const double fe = i == 0 ? phi[m] - (1.0 - w[0]) * am : w[i] * am;
        f[i * N + n] = (T)fe;
        g[i * N + n] = T(0);
    }
    S[n] = T(0);
}

// paper convention <-> pull storage
template <typename T>
__global__ void d2q9_get_state_k(int nx, int ny, const T *__restrict__ f, const T *__restrict__ g,
                                 const T *__restrict__ S, double *fo, double *go, double *So)
{
    const size_t N = (size_t)nx * ny;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % nx), y = (int)(n / nx);
    for (int i = 0; i < 9; ++i) {
        const size_t m = (size_t)wrapi(y - cyv(i), ny) * nx + wrapi(x - cxv(i), nx);
        if (fo) fo[i * N + n] = (double)f[i * N + m];
        if (go) go[i * N + n] = (double)g[i * N + m];
    }
    if (So) So[n] = (double)S[n];
}

template <typename T>
__global__ void d2q9_set_state_k(int nx, int ny, T *__restrict__ f, T *__restrict__ g,
                                 T *__restrict__ S, const double *fi, const double *gi,
                                 const double *Si)
{
    const size_t N = (size_t)nx * ny;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % nx), y = (int)(n / nx);
    for (int i = 0; i < 9; ++i) {
        const size_t m = (size_t)wrapi(y + cyv(i), ny) * nx + wrapi(x + cxv(i), nx);
        f[i * N + n] = (T)fi[i * N + m];
        g[i * N + n] = (T)gi[i * N + m];
    }
    S[n] = (T)Si[n];
}

constexpr int TXW = 128;  // strip width (columns per CTA)

template <typename T, int PASS>
cudaError_t launch_pass(const void *params, const PassArgs &a, const LaunchShape &s,
                        cudaStream_t st)
{
    const StepParams<T> &P = *static_cast<const StepParams<T> *>(params);
    dim3 grid(s.grid_x, s.grid_y), block(TXW, TYB);
    d2q9_pass_kernel<T, TXW, PASS><<<grid, block, 0, st>>>(P, a, s.rows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pass_t(int pass, const void *params, const PassArgs &a, const LaunchShape &s,
                   cudaStream_t st)
{
    switch (pass) {
    case PASS_STATE: return launch_pass<T, PASS_STATE>(params, a, s, st);
    case PASS_STATE | PASS_DIAG: return launch_pass<T, PASS_STATE | PASS_DIAG>(params, a, s, st);
    case PASS_MACROS: return launch_pass<T, PASS_MACROS>(params, a, s, st);
    case PASS_DIAG: return launch_pass<T, PASS_DIAG>(params, a, s, st);
    case PASS_MACROS | PASS_DIAG: return launch_pass<T, PASS_MACROS | PASS_DIAG>(params, a, s, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

LaunchShape d2q9_shape(int nx, int ny, int num_sms)
{
    LaunchShape s;
    s.grid_x = (nx + TXW - 1) / TXW;
    // enough CTAs for several waves of resident blocks, marching >= 8 rows
    const long long target = 8LL * (num_sms > 0 ? num_sms : 152);
    int rows = (int)((long long)s.grid_x * ny / target);
    rows = rows < 8 ? 8 : (rows > 64 ? 64 : rows);
    rows += rows & 1;  // even: two rows per iteration
    s.rows = rows;
    s.grid_y = (ny + rows - 1) / rows;
    s.nblocks = s.grid_x * s.grid_y;
    return s;
}

cudaError_t d2q9_pass(int precision, int pass, const void *params, const PassArgs &a,
                      const LaunchShape &s, cudaStream_t st)
{
    return precision == 0 ? pass_t<double>(pass, params, a, s, st)
                          : pass_t<float>(pass, params, a, s, st);
}

cudaError_t d2q9_init(int precision, const void *params, const double *phi0, double *mu_tmp,
                      void *f, void *g, void *S, cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params);
    const int tb = 256;
    const unsigned nb = (unsigned)((P.N + tb - 1) / tb);
    d2q9_init_mu<<<nb, tb, 0, st>>>(P, phi0, mu_tmp);
    if (precision == 0)
        d2q9_init_pop<double><<<nb, tb, 0, st>>>(P, phi0, mu_tmp, (double *)f, (double *)g,
                                                 (double *)S);
    else
        d2q9_init_pop<float><<<nb, tb, 0, st>>>(P, phi0, mu_tmp, (float *)f, (float *)g,
                                                (float *)S);
    return cudaGetLastError();
}

cudaError_t d2q9_get_state(int precision, int nx, int ny, const void *f, const void *g,
                           const void *S, double *fo, double *go, double *So, cudaStream_t st)
{
    const size_t N = (size_t)nx * ny;
    const int tb = 256;
    const unsigned nb = (unsigned)((N + tb - 1) / tb);
    if (precision == 0)
        d2q9_get_state_k<double><<<nb, tb, 0, st>>>(nx, ny, (const double *)f, (const double *)g,
                                                    (const double *)S, fo, go, So);
    else
        d2q9_get_state_k<float><<<nb, tb, 0, st>>>(nx, ny, (const float *)f, (const float *)g,
                                                   (const float *)S, fo, go, So);
    return cudaGetLastError();
}

cudaError_t d2q9_set_state(int precision, int nx, int ny, void *f, void *g, void *S,
                           const double *fi, const double *gi, const double *Si, cudaStream_t st)
{
    const size_t N = (size_t)nx * ny;
    const int tb = 256;
    const unsigned nb = (unsigned)((N + tb - 1) / tb);
    if (precision == 0)
        d2q9_set_state_k<double><<<nb, tb, 0, st>>>(nx, ny, (double *)f, (double *)g,
                                                    (double *)S, fi, gi, Si);
    else
        d2q9_set_state_k<float><<<nb, tb, 0, st>>>(nx, ny, (float *)f, (float *)g, (float *)S,
                                                   fi, gi, Si);
    return cudaGetLastError();
}

}  // namespace wblbm
