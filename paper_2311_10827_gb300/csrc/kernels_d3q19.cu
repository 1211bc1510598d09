// D3Q19 kernels of the well-balanced phase-field LBM.  The paper works in 2D
// (D2Q9); the 3D form keeps its equilibria (Eqs. H_i, G_i, Siu), sources
// (Eqs. F_i, GGi), moments and isotropic stencils (Eqs. gradient, Laplace)
// on the standard 19-velocity lattice (weights 1/3, 1/18, 1/36; cs^2 = 1/3).
//
// Storage as in 2D: pull scheme, SoA [i][z][y][x], post-collision values at
// their source node.  A step is two passes:
//   1. d3q19_phi_kernel: phi = sum_i f_i pulled (one FP field);
//   2. d3q19_pass_kernel: a CTA owns a TX x TY column tile and marches down
//      z; phi planes (tile + 2 halo, read from the phi field, mostly L2) and
//      mu planes (tile + 1) live in shared-memory rings; each node pulls its
//      19 + 19 populations, recovers the moments and collides.
// HBM traffic per node (FP32): 84 B for pass 1, 324 B for pass 2.  As in 2D,
// FP32 storage keeps the rest population as a compensated pair hi + lo (lo in
// population slot 19) so that its small per-step changes are not lost.
#include <float.h>
#include <math.h>

#include "d3q19_lattice.cuh"
#include "lbm_internal.h"

namespace wblbm {
namespace {

using namespace d3;

// phi = sum_i f_i(x - c_i): rest population last, moving ones in fixed pairs
// grid (ceil(nx / PHI_TX), ny, nz): one thread per node of a row
constexpr int PHI_TX = 128;
template <typename T>
__global__ void __launch_bounds__(PHI_TX)
    d3q19_phi_kernel(const StepParams<T> P, const T *__restrict__ f, T *__restrict__ phi)
{
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = blockIdx.x * PHI_TX + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const unsigned N = (unsigned)P.N;
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    const unsigned n = b.at(0, 0, 0);
    T v[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) v[i] = __ldg(f + (i * N + b.at(-c3x(i), -c3y(i), -c3z(i))));
    T s = sizeof(T) == 4 ? __ldg(f + (19u * N + n)) : T(0);  // low word of the rest pair
#pragma unroll
    for (int i = 1; i < 19; i += 2) s += v[i] + v[i + 1];
    phi[n] = v[0] + s;
}

template <typename T, int PASS>
__global__ void __launch_bounds__(TX3 *TY3) d3q19_pass_kernel(const StepParams<T> P, PassArgs a,
                                                              const T *__restrict__ phif, int planes)
{
    constexpr int PX = TX3 + 4, PY = TY3 + 4, PA = PX * PY;  // phi plane (halo 2)
    constexpr int MX = TX3 + 2, MY = TY3 + 2, MA = MX * MY;  // mu plane (halo 1)
    constexpr int RP = 5, RM = 3;
    __shared__ T phs[RP * PA];
    __shared__ T mus[RM * MA];

    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const unsigned N = (unsigned)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX3 + tx;
    const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
    const int z0 = blockIdx.z * planes, zend = min(z0 + planes, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col_ok = x < nx && y < ny;
    const T *__restrict__ fsrc = static_cast<const T *>(a.f_src);
    const T *__restrict__ gsrc = static_cast<const T *>(a.g_src);
    const unsigned plane = (unsigned)nx * ny;

    auto pslot = [&](int zz) { return (zz - z0 + 2) % RP; };  // zz >= z0 - 2
    auto mslot = [&](int zz) { return (zz - z0 + 1) % RM; };  // zz >= z0 - 1

    // grids narrower than a tile plus halo wrap by division (uniform flags)
    const bool smx = nx < PX + 2, smy = ny < PY + 2, smz = nz < 8;
    auto load_phi_plane = [&](int zz) {
        T *dst = phs + pslot(zz) * PA;
        const unsigned zo = (unsigned)wrapc(zz, nz, smz) * plane;
        for (int q = tid; q < PA; q += TX3 * TY3) {
            const int lx = q % PX, ly = q / PX;
            const unsigned xx = wrapc(x0 - 2 + lx, nx, smx), yy = wrapc(y0 - 2 + ly, ny, smy);
            dst[q] = phif[zo + yy * nx + xx];
        }
    };
    // Eq. chemical_potencial with Eq. Laplace on D3Q19:
    // lap = (1/3) sum_faces (phi_n - phi) + (1/6) sum_edges (phi_n - phi)
    auto mu_plane = [&](int zz) {
        const T *pm = phs + pslot(zz - 1) * PA, *p0 = phs + pslot(zz) * PA,
                *pp = phs + pslot(zz + 1) * PA;
        T *dst = mus + mslot(zz) * MA;
        for (int q = tid; q < MA; q += TX3 * TY3) {
            const int lx = q % MX + 1, ly = q / MX + 1;  // phi plane coordinates
            const int c = ly * PX + lx;
            const T v = p0[c];
            const T fa = (p0[c + 1] - v) + (p0[c - 1] - v) + (p0[c + PX] - v) + (p0[c - PX] - v) +
                         (pp[c] - v) + (pm[c] - v);
            const T ed = ((p0[c + PX + 1] - v) + (p0[c + PX - 1] - v) + (p0[c - PX + 1] - v) +
                          (p0[c - PX - 1] - v)) +
                         ((pp[c + 1] - v) + (pp[c - 1] - v) + (pm[c + 1] - v) + (pm[c - 1] - v)) +
                         ((pp[c + PX] - v) + (pp[c - PX] - v) + (pm[c + PX] - v) + (pm[c - PX] - v));
            const T lap = T(1.0 / 3.0) * fa + T(1.0 / 6.0) * ed;
            dst[q] = T(4) * P.beta * (v - P.phil) * (v - P.phiv) * (v - P.phibar) - P.kappa * lap;
        }
    };
    // Eq. gradient on D3Q19: (1/6) face differences + (1/12) edge differences
    auto grad3 = [&](const T *m, const T *c0, const T *p, int c, int SX, T out[3]) {
        out[0] = T(1.0 / 6.0) * (c0[c + 1] - c0[c - 1]) +
                 T(1.0 / 12.0) * ((c0[c + SX + 1] - c0[c + SX - 1]) + (c0[c - SX + 1] - c0[c - SX - 1]) +
                                  (p[c + 1] - p[c - 1]) + (m[c + 1] - m[c - 1]));
        out[1] = T(1.0 / 6.0) * (c0[c + SX] - c0[c - SX]) +
                 T(1.0 / 12.0) * ((c0[c + SX + 1] - c0[c - SX + 1]) + (c0[c + SX - 1] - c0[c - SX - 1]) +
                                  (p[c + SX] - p[c - SX]) + (m[c + SX] - m[c - SX]));
        out[2] = T(1.0 / 6.0) * (p[c] - m[c]) +
                 T(1.0 / 12.0) * ((p[c + 1] - m[c + 1]) + (p[c - 1] - m[c - 1]) +
                                  (p[c + SX] - m[c + SX]) + (p[c - SX] - m[c - SX]));
    };

    double d_phi = 0.0, d_E = 0.0, d_u2 = 0.0, d_mumin = DBL_MAX, d_mumax = -DBL_MAX,
           d_bud = 0.0, d_bad = 0.0;

    // FP32: equilibrium shift of the source buffer and of the writes (only a
    // time step reads it)
    T a_src = T(0), a_dst = T(0);
    if (sizeof(T) == 4 && (PASS & PASS_STATE)) {
        a_src = *a.eqs_src;
        a_dst = *a.eqs_target;
        if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0) *a.eqs_dst = a_dst;
    }

    for (int q = 0; q < 5; ++q) load_phi_plane(z0 - 2 + q);
    __syncthreads();
    mu_plane(z0 - 1);
    mu_plane(z0);
    mu_plane(z0 + 1);
    __syncthreads();

    // Plane zz + 3 of phi travels through registers while plane zz is
    // updated, so its loads overlap the node's own pulls (one exposed memory
    // latency per plane).  Ring use during the update of plane zz: phi planes
    // zz-1..zz+1 (read), zz+3 (written: a fifth slot); mu planes zz-1..zz+1.
    constexpr int PPT = (PA + TX3 * TY3 - 1) / (TX3 * TY3);
    const unsigned xw = col_ok ? (unsigned)x : 0, yw = col_ok ? (unsigned)y : 0;
    Nb b = make_nb(xw, yw, z0, nx, ny, nz);
    for (int zz = z0; zz < zend; ++zz) {
        T pre[PPT];
        {
            const unsigned zo = (unsigned)wrapc(zz + 3, nz, smz) * plane;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int q = tid + k * TX3 * TY3;
                if (q < PA) {
                    const unsigned xx = wrapc(x0 - 2 + q % PX, nx, smx),
                                   yy = wrapc(y0 - 2 + q / PX, ny, smy);
                    pre[k] = phif[zo + yy * nx + xx];
                }
            }
        }
        if (col_ok) {
        nb_plane(b, zz, nx, ny, nz);
        const unsigned n = b.at(0, 0, 0);
        T fv[19], gv[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const unsigned src = b.at(-c3x(i), -c3y(i), -c3z(i));
            fv[i] = __ldg(fsrc + (i * N + src));
            gv[i] = __ldg(gsrc + (i * N + src));
        }
        T Sprev = T(0);
        if (PASS & (PASS_STATE | PASS_DIAG)) Sprev = __ldcs(static_cast<const T *>(a.S) + n);

        const T lo0 = sizeof(T) == 4 ? __ldg(fsrc + (19u * N + n)) : T(0);
        T snz = T(0), sg = T(0);
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            snz += fv[i] + fv[i + 1];
            sg += gv[i] + gv[i + 1];
        }
        const T phi = fv[0] + (lo0 + snz);
        const int cp = (ty + 2) * PX + (tx + 2), cm = (ty + 1) * MX + (tx + 1);
        const T *mz = mus + mslot(zz) * MA;
        const T mu = mz[cm];
        T gp[3], gm[3];
        grad3(phs + pslot(zz - 1) * PA, phs + pslot(zz) * PA, phs + pslot(zz + 1) * PA, cp, PX, gp);
        grad3(mus + mslot(zz - 1) * MA, mz, mus + mslot(zz + 1) * MA, cm, MX, gm);

        T F[3], gr[3], u[3];
        const T dphi = phi - P.phiv;
        const T rho = P.rhov + dphi * P.drho;
        const T nu = P.nuv + dphi * P.dnu;
        const T inv_rho = Arith3<T>::rcp(rho);
        const T itg = Arith3<T>::rcp(T(0.5) + T(3) * nu);
        T j3[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (c3x(i)) j3[0] += T(c3x(i)) * gv[i];
            if (c3y(i)) j3[1] += T(c3y(i)) * gv[i];
            if (c3z(i)) j3[2] += T(c3z(i)) * gv[i];
        }
        T ugr = T(0), uu = T(0), S = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            F[d] = -phi * gm[d] + P.G[d];
            gr[d] = P.drho * gp[d];
            u[d] = (j3[d] + T(0.5) * F[d]) * inv_rho;
            ugr += u[d] * gr[d];
            uu += u[d] * u[d];
            S += u[d] * gp[d];
        }
        // p = cs2/(1 - w0) [sum_{i!=0} g_i + u.grad(rho)/2 + rho s_0], cs2/(1-w0) = 1/2,
        // rho s_0 = -(1/2) rho |u|^2
        const T p = T(0.5) * (sg + T(0.5) * ugr - T(0.5) * rho * uu);

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
            if (a.out_phi) a.out_phi[n] = (double)phi;
            if (a.out_p) a.out_p[n] = (double)p;
            if (a.out_mu) a.out_mu[n] = (double)mu;
            if (a.out_u) {
                a.out_u[n] = (double)u[0];
                a.out_u[(size_t)N + n] = (double)u[1];
                a.out_u[2 * (size_t)N + n] = (double)u[2];
            }
        }
        if (PASS & PASS_STATE) {
            T *__restrict__ fd = static_cast<T *>(a.f_dst);
            T *__restrict__ gd = static_cast<T *>(a.g_dst);
            __stcs(static_cast<T *>(a.S) + n, S);
            // CH population: b = -5/2, -1, 1/2 (rest, face, edge) for D = 3
            const T Sh = T(1.5) * S - T(0.5) * Sprev;
            const T am = P.alpha * mu - a_src;  // in the source buffer's shifted variables
            const T dsh = a_src - a_dst;         // move the writes to the target shift
            const T itf = P.inv_tauf;
            {
                const T d0 = -(T(2.0 / 3.0) * am - snz) * itf - T(5.0 / 6.0) * Sh - T(2.0 / 3.0) * dsh;
                if (sizeof(T) == 4) {
                    const T sl = lo0 + d0;  // exact two-sum on the high word
                    const T hi = fv[0] + sl;
                    const T bp = hi - fv[0];
                    __stcs(fd + n, hi);
                    __stcs(fd + (19u * N + n), (fv[0] - (hi - bp)) + (sl - bp));
                } else {
                    __stcs(fd + n, fv[0] + d0);
                }
            }
            // each population moves by its own small increment (as in 2D: the
            // increments sum to sum_i F_i up to unbiased rounding)
            const T ea = T(1.0 / 18.0) * am, ee = T(1.0 / 36.0) * am;
            const T sa = T(-1.0 / 18.0) * Sh + T(1.0 / 18.0) * dsh;
            const T se = T(1.0 / 72.0) * Sh + T(1.0 / 36.0) * dsh;
#pragma unroll
            for (int i = 1; i < 19; ++i)
                __stcs(fd + (i * N + n), fv[i] + (((i <= 6 ? ea : ee) - fv[i]) * itf + (i <= 6 ? sa : se)));
            // hydrodynamic population, pairs of opposite directions (as in 2D)
            const T kg = T(1) - T(0.5) * itg;
            const T A = T(3) * p - T(1.5) * rho * uu;
            __stcs(gd + n, gv[0] + ((T(1.0 / 3.0) * A - T(3) * p) - gv[0]) * itg);
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const int o = (i <= 6) ? (i % 2 ? i + 1 : i - 1) : (i <= 10 ? 17 - i : (i <= 14 ? 25 - i : 33 - i));
                if (o < i) continue;  // each pair once, from its first member
                const T w = T(w3(i));
                const T cu = T(c3x(i)) * u[0] + T(c3y(i)) * u[1] + T(c3z(i)) * u[2];
                const T cF = T(c3x(i)) * F[0] + T(c3y(i)) * F[1] + T(c3z(i)) * F[2];
                const T cg = T(c3x(i)) * gr[0] + T(c3y(i)) * gr[1] + T(c3z(i)) * gr[2];
                const T eq_s = w * (A + T(4.5) * rho * cu * cu), eq_a = T(3) * w * rho * cu;
                const T G_s = T(3) * w * kg * cu * cg, G_a = T(3) * w * kg * cF;
                __stcs(gd + (i * N + n), gv[i] + ((eq_s + eq_a - gv[i]) * itg + (G_s + G_a)));
                __stcs(gd + (o * N + n), gv[o] + ((eq_s - eq_a - gv[o]) * itg + (G_s - G_a)));
            }
        }
        }  // col_ok
        {
            T *d = phs + pslot(zz + 3) * PA;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int q = tid + k * TX3 * TY3;
                if (q < PA) d[q] = pre[k];
            }
        }
        __syncthreads();
        mu_plane(zz + 2);
        __syncthreads();
    }

    if (PASS & PASS_DIAG) {
        for (int o = 16; o > 0; o >>= 1) {
            d_phi += __shfl_xor_sync(0xffffffffu, d_phi, o);
            d_E += __shfl_xor_sync(0xffffffffu, d_E, o);
            d_bud += __shfl_xor_sync(0xffffffffu, d_bud, o);
            d_u2 = fmax(d_u2, __shfl_xor_sync(0xffffffffu, d_u2, o));
            d_mumin = fmin(d_mumin, __shfl_xor_sync(0xffffffffu, d_mumin, o));
            d_mumax = fmax(d_mumax, __shfl_xor_sync(0xffffffffu, d_mumax, o));
            d_bad = fmax(d_bad, __shfl_xor_sync(0xffffffffu, d_bad, o));
        }
        constexpr int NW = TX3 * TY3 / 32;
        __shared__ double red[7][NW];
        const int lane = tid & 31, wid = tid >> 5;
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
        if (tid == 0) {
            DiagPartial o;
            o.sum_phi = 0.0, o.E = 0.0, o.u2max = 0.0, o.mu_min = DBL_MAX, o.mu_max = -DBL_MAX;
            o.budget = 0.0, o.nonfinite = 0.0, o.pad = 0.0;
            for (int w = 0; w < NW; ++w) {
                o.sum_phi += red[0][w];
                o.E += red[1][w];
                o.u2max = fmax(o.u2max, red[2][w]);
                o.mu_min = fmin(o.mu_min, red[3][w]);
                o.mu_max = fmax(o.mu_max, red[4][w]);
                o.budget += red[5][w];
                o.nonfinite = fmax(o.nonfinite, red[6][w]);
            }
            a.partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = o;
        }
    }
}

// ------------------------------------------------------------ initial state

// mu0 = psi'(phi0) - kappa lap(phi0) in FP64
__global__ void d3q19_init_mu(const StepParams<double> P, const double *__restrict__ phi,
                              double *__restrict__ mu)
{
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)P.N) return;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    const double c = phi[n];
    double fa = 0.0, ed = 0.0;
    for (int i = 1; i < 19; ++i) {
        const double d = phi[b.at(c3x(i), c3y(i), c3z(i))] - c;
        if (i <= 6) fa += d; else ed += d;
    }
    const double lap = (1.0 / 3.0) * fa + (1.0 / 6.0) * ed;
    mu[n] = 4.0 * P.beta * (c - P.phil) * (c - P.phiv) * (c - P.phibar) - P.kappa * lap;
}

template <typename T>
__global__ void d3q19_init_pop(const StepParams<double> P, const double *__restrict__ phi,
                               const double *__restrict__ mu, T *__restrict__ f, T *__restrict__ g,
                               T *__restrict__ S)
{
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)P.N) return;
    const size_t N = (size_t)P.N;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    for (int i = 0; i < 19; ++i) {
        const unsigned m = b.at(c3x(i), c3y(i), c3z(i));  // f_i(x,0) stored at x - c_i
        const double am = P.alpha * mu[m];
        const double fe = i == 0 ? phi[m] - (1.0 - w3(0)) * am : w3(i) * am;
        f[i * N + n] = (T)fe;
        g[i * N + n] = T(0);
        if (sizeof(T) == 4 && i == 0) f[19 * N + n] = (T)(fe - (double)(T)fe);
    }
    S[n] = T(0);
}

template <typename T>
__global__ void d3q19_get_state_k(StepParams<double> P, const T *__restrict__ f,
                                  const T *__restrict__ g, const T *__restrict__ S,
                                  const float *eqs, double *fo, double *go, double *So)
{
    const size_t N = (size_t)P.N;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    for (int i = 0; i < 19; ++i) {
        const unsigned m = b.at(-c3x(i), -c3y(i), -c3z(i));
        double fv = (double)f[i * N + m];
        if (sizeof(T) == 4 && i == 0) fv += (double)f[19 * N + m];
        if (sizeof(T) == 4) fv += (i == 0 ? -(2.0 / 3.0) : w3(i)) * (double)*eqs;  // equilibrium shift
        if (fo) fo[i * N + n] = fv;
        if (go) go[i * N + n] = (double)g[i * N + m];
    }
    if (So) So[n] = (double)S[n];
}

template <typename T>
__global__ void d3q19_set_state_k(StepParams<double> P, T *__restrict__ f, T *__restrict__ g,
                                  T *__restrict__ S, const double *fi, const double *gi,
                                  const double *Si)
{
    const size_t N = (size_t)P.N;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    for (int i = 0; i < 19; ++i) {
        const unsigned m = b.at(c3x(i), c3y(i), c3z(i));
        const double v = fi[i * N + m];
        f[i * N + n] = (T)v;
        if (sizeof(T) == 4 && i == 0) f[19 * N + n] = (T)(v - (double)(T)v);
        g[i * N + n] = (T)gi[i * N + m];
    }
    S[n] = (T)Si[n];
}

template <typename T, int PASS>
cudaError_t launch3(const void *params, const PassArgs &a, const LaunchShape &s, void *phi,
                    cudaStream_t st)
{
    const StepParams<T> &P = *static_cast<const StepParams<T> *>(params);
    const dim3 pg((P.nx + PHI_TX - 1) / PHI_TX, P.ny, P.nz);
    d3q19_phi_kernel<T><<<pg, PHI_TX, 0, st>>>(P, static_cast<const T *>(a.f_src), static_cast<T *>(phi));
    dim3 grid(s.grid_x, s.grid_y, s.nblocks / (s.grid_x * s.grid_y)), block(TX3, TY3);
    d3q19_pass_kernel<T, PASS><<<grid, block, 0, st>>>(P, a, static_cast<const T *>(phi), s.rows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pass3_t(int pass, const void *params, const PassArgs &a, const LaunchShape &s,
                    void *phi, cudaStream_t st)
{
    switch (pass) {
    case PASS_STATE: return launch3<T, PASS_STATE>(params, a, s, phi, st);
    case PASS_STATE | PASS_DIAG: return launch3<T, PASS_STATE | PASS_DIAG>(params, a, s, phi, st);
    case PASS_MACROS: return launch3<T, PASS_MACROS>(params, a, s, phi, st);
    case PASS_DIAG: return launch3<T, PASS_DIAG>(params, a, s, phi, st);
    case PASS_MACROS | PASS_DIAG: return launch3<T, PASS_MACROS | PASS_DIAG>(params, a, s, phi, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

LaunchShape d3q19_shape(int nx, int ny, int nz, int num_sms, int ctas_per_sm)
{
    LaunchShape s;
    s.variant = 0;
    s.grid_x = (nx + TX3 - 1) / TX3;
    s.grid_y = (ny + TY3 - 1) / TY3;
    // Split z into gz marches of `planes` planes.  Time ~ waves x (planes + 2)
    // (a march starts by filling its rings, about two planes of work), waves
    // = ceil(CTAs / resident CTAs): pick the split with the least of it, so a
    // partly filled last wave costs little.
    const long long cols = (long long)s.grid_x * s.grid_y;
    const long long slots = (long long)(ctas_per_sm > 0 ? ctas_per_sm : 2) * (num_sms > 0 ? num_sms : 152);
    long long best = -1, best_gz = 1;
    const int gz_max = nz / 4 > 1 ? nz / 4 : 1;
    for (int gz = 1; gz <= gz_max; ++gz) {
        const long long planes = (nz + gz - 1) / gz;
        const long long waves = (cols * gz + slots - 1) / slots;
        const long long cost = waves * (planes + 2);
        if (best < 0 || cost < best) {
            best = cost;
            best_gz = gz;
        }
    }
    const int planes = (nz + (int)best_gz - 1) / (int)best_gz;
    s.rows = planes;
    s.nblocks = (int)(cols * ((nz + planes - 1) / planes));
    return s;
}

int d3q19_ctas_per_sm(int precision)
{
    int n = 0;
    cudaError_t e = precision == 0
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &n, d3q19_pass_kernel<double, PASS_STATE>, TX3 * TY3, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                              &n, d3q19_pass_kernel<float, PASS_STATE>, TX3 * TY3, 0);
    return e == cudaSuccess && n > 0 ? n : 2;
}

cudaError_t d3q19_pass(int precision, int pass, const void *params, const PassArgs &a,
                       const LaunchShape &s, void *phi_work, cudaStream_t st)
{
    return precision == 0 ? pass3_t<double>(pass, params, a, s, phi_work, st)
                          : pass3_t<float>(pass, params, a, s, phi_work, st);
}

cudaError_t d3q19_init_mu_fp64(const void *params, const double *phi0, double *mu, cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    d3q19_init_mu<<<nb, 256, 0, st>>>(P, phi0, mu);
    return cudaGetLastError();
}

cudaError_t d3q19_init(int precision, const void *params, const double *phi0, double *mu_tmp,
                       void *f, void *g, void *S, cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    d3q19_init_mu<<<nb, 256, 0, st>>>(P, phi0, mu_tmp);
    if (precision == 0)
        d3q19_init_pop<double><<<nb, 256, 0, st>>>(P, phi0, mu_tmp, (double *)f, (double *)g, (double *)S);
    else
        d3q19_init_pop<float><<<nb, 256, 0, st>>>(P, phi0, mu_tmp, (float *)f, (float *)g, (float *)S);
    return cudaGetLastError();
}

cudaError_t d3q19_get_state(int precision, const void *params, const void *f, const void *g,
                            const void *S, const float *eqs, double *fo, double *go, double *So,
                            cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    if (precision == 0)
        d3q19_get_state_k<double><<<nb, 256, 0, st>>>(P, (const double *)f, (const double *)g,
                                                     (const double *)S, eqs, fo, go, So);
    else
        d3q19_get_state_k<float><<<nb, 256, 0, st>>>(P, (const float *)f, (const float *)g,
                                                    (const float *)S, eqs, fo, go, So);
    return cudaGetLastError();
}

cudaError_t d3q19_set_state(int precision, const void *params, void *f, void *g, void *S,
                            const double *fi, const double *gi, const double *Si, cudaStream_t st)
{
    const StepParams<double> &P = *static_cast<const StepParams<double> *>(params);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    if (precision == 0)
        d3q19_set_state_k<double><<<nb, 256, 0, st>>>(P, (double *)f, (double *)g, (double *)S, fi, gi, Si);
    else
        d3q19_set_state_k<float><<<nb, 256, 0, st>>>(P, (float *)f, (float *)g, (float *)S, fi, gi, Si);
    return cudaGetLastError();
}

}  // namespace wblbm
