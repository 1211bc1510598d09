// D3Q19 step with the populations stored as 16-bit offsets from their
// equilibria (FP16 or BF16), arithmetic in FP32.
//
// A post-collision value is stored as
//     f*_i(x) = f_i^eq(M(x)) + s_f h_i(x),   g*_i(x) = g_i^eq(M(x)) + s_g k_i(x),
// where M(x) = (phi, mu, p, u) are the FP32 macroscopic fields of node x from
// the same collision, f^eq is Eq. H_i, g^eq the equilibrium of Eq. G_i (with
// s_i(u)), h and k are 16-bit numbers and s_f, s_g are per-field scales
// (powers of two).  Only the non-equilibrium part and the source, which are
// small, pass through the 16-bit rounding.  Pull layout as in the other
// precisions: f*_i(x) is stored at x, the step at y reads it from y - c_i
// together with the macros of y - c_i.
//
// Storage of one parity of the double buffer (offset_layout):
//   f buffer: h[19][N] (u16) | M[7][N] (FP32: phi, mu, p, ux, uy, uz, B) | s_f, s_g
//   g buffer: k[19][N] (u16)
// B = phi + alpha sum_{i != 0} w_i (mu(x + c_i) - mu(x)) is the part of the
// next step's phi(x) that does not depend on the offsets; the step writes it
// from its mu ring, so the next phi pass streams B and the offsets only.
// The rest population keeps phi exactly the way the FP32 path's compensated
// pair does: phi (FP32) in M is its high word, and the rounding residual of
// phi is folded into the rest offset h_0.
//
// Scales: a step reads the scales stored with its source buffer and writes
// with the context's target scales, which it also stores with the
// destination buffer.  off_refresh (run with the diagnostics) sets the
// targets from the largest stored offsets: max |offset| / s near 2^12 (FP16
// range 65504), never below 2^-16 (so no offset up to about 1 can overflow
// between two refreshes).
//
// A step is two passes, as in the FP32 D3Q19 path: d3q19_off_phi_kernel
// writes phi from the pulled populations, then d3q19_off_pass_kernel marches
// down z with phi, mu and the macro planes of the source state in
// shared-memory rings.  HBM traffic per node: 38 + 4 + 4 B (pass 1) and
// 38 + 38 + 24 + 4 + 4 B read, 38 + 38 + 28 + 4 B written (pass 2).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>
#include <math.h>

#include "d3q19_lattice.cuh"
#include "lbm_internal.h"

namespace wblbm {
namespace {

using namespace d3;

struct CodecF16 {
    static constexpr unsigned short INF_BITS = 0x7c00;
    __device__ static float dec(unsigned short u) { return __half2float(__ushort_as_half(u)); }
    __device__ static unsigned short enc(float v) { return __half_as_ushort(__float2half_rn(v)); }
};
struct CodecBF16 {
    static constexpr unsigned short INF_BITS = 0x7f80;
    __device__ static float dec(unsigned short u)
    {
        return __bfloat162float(__ushort_as_bfloat16(u));
    }
    __device__ static unsigned short enc(float v)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};

// views of one parity of the offset storage
struct OffBuf {
    unsigned short *h, *k;  // f and g offsets [19][N]
    float *M;               // macros [7][N] (phi, mu, p, u, B)
    float *sc;              // s_f, s_g
};

__host__ __device__ inline OffBuf off_view(const void *fbuf, const void *gbuf, long long N)
{
    const OffsetLayout L = offset_layout(N, 19, 3);  // 3 + 4 FP32 arrays
    char *fb = (char *)fbuf;
    return OffBuf{(unsigned short *)fb, (unsigned short *)gbuf, (float *)(fb + L.mac_off),
                  (float *)(fb + L.sc_off)};
}

// ------------------------------------------------------------------ pass 1
// phi(x) = sum_i f_i(x): the rest value phi(x) - (1 - w0) alpha mu(x) + s_f h_0(x)
// and the moving values w_i alpha mu(x - c_i) + s_f h_i(x - c_i), i.e.
// B(x) + s_f sum_i h_i(x - c_i) with B = phi + alpha sum_{i != 0} w_i (mu(x - c_i) - mu(x)).
// grid (ceil(nx / PHI_TX), ny, nz): one thread per node of a row
constexpr int PHI_TX = 128;
template <class C>
__global__ void __launch_bounds__(PHI_TX)
    d3q19_off_phi_kernel(const StepParams<float> P, const OffBuf src, float *__restrict__ phi)
{
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = blockIdx.x * PHI_TX + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const unsigned N = (unsigned)P.N;
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    const unsigned n = b.at(0, 0, 0);
    float sh = C::dec(__ldg(src.h + n));
#pragma unroll
    for (int i = 1; i < 19; ++i) sh += C::dec(__ldg(src.h + (i * N + b.at(-c3x(i), -c3y(i), -c3z(i)))));
    phi[n] = __ldg(src.M + 6 * N + n) + __ldg(src.sc) * sh;
}

// B(x) from stored macros (after an initial condition or a state exchange)
__global__ void d3q19_off_prep_k(const StepParams<float> P, OffBuf o)
{
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = blockIdx.x * PHI_TX + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const unsigned N = (unsigned)P.N;
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    const unsigned n = b.at(0, 0, 0);
    const float *mu = o.M + N, mux = mu[n];
    float dfa = 0.0f, ded = 0.0f;
    for (int i = 1; i < 19; ++i) {
        const float d = mu[b.at(c3x(i), c3y(i), c3z(i))] - mux;
        if (i <= 6)
            dfa += d;
        else
            ded += d;
    }
    o.M[6 * N + n] = o.M[n] + P.alpha * (1.0f / 18.0f * dfa + 1.0f / 36.0f * ded);
}

// ------------------------------------------------------------------ pass 2

template <class C, int PASS>
__global__ void __launch_bounds__(TX3 *TY3) d3q19_off_pass_kernel(const StepParams<float> P,
                                                                  PassArgs a, const OffBuf src,
                                                                  const OffBuf dst,
                                                                  const float *__restrict__ target,
                                                                  const float *__restrict__ phif,
                                                                  int planes)
{
    constexpr int PX = TX3 + 4, PY = TY3 + 4, PA = PX * PY;  // phi plane (halo 2)
    constexpr int MX = TX3 + 2, MY = TY3 + 2, MA = MX * MY;  // mu / macro plane (halo 1)
    constexpr int RP = 5, RM = 3, RQ = 3;
    __shared__ float phs[RP * PA];
    __shared__ float mus[RM * MA];
    // the source macros of the plane two ahead, copied while a plane is updated
    __shared__ float mraw[6 * MA];
    // per source node: {alpha mu, A = 3p - 3/2 rho |u|^2, rho ux, rho uy} and
    // {rho uz, 9 / (2 rho)}: g^eq_i = w_i (A + 3 c.j + (9/2)(c.j)^2 / rho)
    __shared__ float4 qa[RQ * MA];
    __shared__ float2 qb[RQ * MA];

    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const unsigned N = (unsigned)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX3 + tx;
    const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
    const int z0 = blockIdx.z * planes, zend = min(z0 + planes, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col_ok = x < nx && y < ny;
    const unsigned plane = (unsigned)nx * ny;
    const float s_f = __ldg(src.sc), s_g = __ldg(src.sc + 1);
    const float t_f = __ldg(target), t_g = __ldg(target + 1);
    const float it_f = 1.0f / t_f, it_g = 1.0f / t_g;  // powers of two: exact
    if ((PASS & PASS_STATE) && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0) {
        dst.sc[0] = t_f;
        dst.sc[1] = t_g;
    }

    auto pslot = [&](int zz) { return (zz - z0 + 2) % RP; };
    auto mslot = [&](int zz) { return (zz - z0 + 1) % RM; };
    auto qslot = [&](int zz) { return (zz - z0 + 1) % RQ; };

    // grids narrower than a tile plus halo wrap by division (uniform flags)
    const bool smx = nx < PX + 2, smy = ny < PY + 2, smz = nz < 8;
    auto load_phi_plane = [&](int zz) {
        float *d = phs + pslot(zz) * PA;
        const unsigned zo = (unsigned)wrapc(zz, nz, smz) * plane;
        for (int q = tid; q < PA; q += TX3 * TY3) {
            const int lx = q % PX, ly = q / PX;
            const unsigned xx = wrapc(x0 - 2 + lx, nx, smx), yy = wrapc(y0 - 2 + ly, ny, smy);
            d[q] = phif[zo + yy * nx + xx];
        }
    };
    // Eq. chemical_potencial with Eq. Laplace on D3Q19
    auto mu_plane = [&](int zz) {
        const float *pm = phs + pslot(zz - 1) * PA, *p0 = phs + pslot(zz) * PA,
                    *pp = phs + pslot(zz + 1) * PA;
        float *d = mus + mslot(zz) * MA;
        for (int q = tid; q < MA; q += TX3 * TY3) {
            const int lx = q % MX + 1, ly = q / MX + 1;
            const int c = ly * PX + lx;
            const float v = p0[c];
            const float fa = (p0[c + 1] - v) + (p0[c - 1] - v) + (p0[c + PX] - v) +
                             (p0[c - PX] - v) + (pp[c] - v) + (pm[c] - v);
            const float ed = ((p0[c + PX + 1] - v) + (p0[c + PX - 1] - v) + (p0[c - PX + 1] - v) +
                              (p0[c - PX - 1] - v)) +
                             ((pp[c + 1] - v) + (pp[c - 1] - v) + (pm[c + 1] - v) + (pm[c - 1] - v)) +
                             ((pp[c + PX] - v) + (pp[c - PX] - v) + (pm[c + PX] - v) +
                              (pm[c - PX] - v));
            const float lap = (1.0f / 3.0f) * fa + (1.0f / 6.0f) * ed;
            d[q] = 4.0f * P.beta * (v - P.phil) * (v - P.phiv) * (v - P.phibar) - P.kappa * lap;
        }
    };
    // equilibrium data of the source state's macros (ph, mu, p, u) at item q
    // of a macro plane (tile + 1 halo)
    auto put_macros = [&](int slot, int q, const float m6[6]) {
        const float rho = P.rhov + (m6[0] - P.phiv) * P.drho;
        qa[slot * MA + q] = make_float4(P.alpha * m6[1],
                                        3.0f * m6[2] - 1.5f * rho * (m6[3] * m6[3] + m6[4] * m6[4] + m6[5] * m6[5]),
                                        rho * m6[3], rho * m6[4]);
        qb[slot * MA + q] = make_float2(rho * m6[5], 4.5f / rho);
    };
    auto macro_node = [&](int zz, int q) {
        const unsigned m = (unsigned)wrapc(zz, nz, smz) * plane +
                           (unsigned)wrapc(y0 - 1 + q / MX, ny, smy) * nx + wrapc(x0 - 1 + q % MX, nx, smx);
        return m;
    };
    auto macro_plane = [&](int zz) {
        for (int q = tid; q < MA; q += TX3 * TY3) {
            const unsigned m = macro_node(zz, q);
            float m6[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) m6[k] = __ldg(src.M + k * N + m);
            put_macros(qslot(zz), q, m6);
        }
    };
    auto grad3 = [&](const float *m, const float *c0, const float *p, int c, int SX, float out[3]) {
        out[0] = (1.0f / 6.0f) * (c0[c + 1] - c0[c - 1]) +
                 (1.0f / 12.0f) * ((c0[c + SX + 1] - c0[c + SX - 1]) + (c0[c - SX + 1] - c0[c - SX - 1]) +
                                   (p[c + 1] - p[c - 1]) + (m[c + 1] - m[c - 1]));
        out[1] = (1.0f / 6.0f) * (c0[c + SX] - c0[c - SX]) +
                 (1.0f / 12.0f) * ((c0[c + SX + 1] - c0[c - SX + 1]) + (c0[c + SX - 1] - c0[c - SX - 1]) +
                                   (p[c + SX] - p[c - SX]) + (m[c + SX] - m[c - SX]));
        out[2] = (1.0f / 6.0f) * (p[c] - m[c]) +
                 (1.0f / 12.0f) * ((p[c + 1] - m[c + 1]) + (p[c - 1] - m[c - 1]) +
                                   (p[c + SX] - m[c + SX]) + (p[c - SX] - m[c - SX]));
    };

    double d_phi = 0.0, d_E = 0.0, d_u2 = 0.0, d_mumin = DBL_MAX, d_mumax = -DBL_MAX,
           d_bud = 0.0, d_bad = 0.0;

    for (int q = 0; q < 5; ++q) load_phi_plane(z0 - 2 + q);
    macro_plane(z0 - 1);
    macro_plane(z0);
    macro_plane(z0 + 1);
    __syncthreads();
    mu_plane(z0 - 1);
    mu_plane(z0);
    mu_plane(z0 + 1);
    __syncthreads();

    // Plane zz + 3 of phi (into its ring slot) and the raw source macros of
    // plane zz + 2 (into mraw) are copied asynchronously while plane zz is
    // updated, so their loads overlap the node's own pulls and hold no
    // registers.  Ring use during the update of plane zz: phi zz-1..zz+1
    // (read) and zz+3 (being written); mu and macros zz-1..zz+1; once every
    // thread is past the update, macro plane zz+2 and mu plane zz+2 take the
    // slots of zz-1.
    const unsigned xw = col_ok ? (unsigned)x : 0, yw = col_ok ? (unsigned)y : 0;
    Nb b = make_nb(xw, yw, z0, nx, ny, nz);
    for (int zz = z0; zz < zend; ++zz) {
        {
            const unsigned zo = (unsigned)wrapc(zz + 3, nz, smz) * plane;
            float *d = phs + pslot(zz + 3) * PA;
            for (int q = tid; q < PA; q += TX3 * TY3) {
                const unsigned xx = wrapc(x0 - 2 + q % PX, nx, smx), yy = wrapc(y0 - 2 + q / PX, ny, smy);
                cp_async4(d + q, phif + (zo + yy * nx + xx));
            }
            for (int q = tid; q < MA; q += TX3 * TY3) {
                const unsigned m = macro_node(zz + 2, q);
#pragma unroll
                for (int c = 0; c < 6; ++c) cp_async4(mraw + c * MA + q, src.M + ((size_t)c * N + m));
            }
            cp_commit();
        }
        if (col_ok) {
        nb_plane(b, zz, nx, ny, nz);
        const unsigned n = b.at(0, 0, 0);
        // the two 16-bit offsets of direction i share one register
        unsigned hk[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const unsigned s = b.at(-c3x(i), -c3y(i), -c3z(i));
            hk[i] = (unsigned)__ldg(src.h + (i * N + s)) | ((unsigned)__ldg(src.k + (i * N + s)) << 16);
        }
        auto hr = [&](int i) { return (unsigned short)(hk[i] & 0xffffu); };
        auto kr = [&](int i) { return (unsigned short)(hk[i] >> 16); };
        float Sprev = 0.0f;
        if (PASS & (PASS_STATE | PASS_DIAG)) Sprev = __ldcs(static_cast<const float *>(a.S) + n);
        const float phi_hi = __ldg(src.M + n), p_own = __ldg(src.M + 2 * N + n);

        // populations after streaming, rebuilt from offsets and source macros
        const int cq = (ty + 1) * MX + (tx + 1);
        float fv[19], gv[19];
        float flo;  // rest population minus its high word phi_hi
        {
            const float4 A0 = qa[qslot(zz) * MA + cq];
            flo = -(2.0f / 3.0f) * A0.x + s_f * C::dec(hr(0));
            gv[0] = (1.0f / 3.0f) * A0.y - 3.0f * p_own + s_g * C::dec(kr(0));
            fv[0] = 0.0f;
        }
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int c = qslot(zz - c3z(i)) * MA + cq - c3y(i) * MX - c3x(i);
            const float4 A = qa[c];
            const float2 B = qb[c];
            const float w = (float)w3(i);
            fv[i] = w * A.x + s_f * C::dec(hr(i));
            float cj = 0.0f;
            if (c3x(i)) cj += (float)c3x(i) * A.z;
            if (c3y(i)) cj += (float)c3y(i) * A.w;
            if (c3z(i)) cj += (float)c3z(i) * B.x;
            gv[i] = w * (A.y + cj * (3.0f + B.y * cj)) + s_g * C::dec(kr(i));
        }

        float snz = 0.0f, sg = 0.0f;
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            snz += fv[i] + fv[i + 1];
            sg += gv[i] + gv[i + 1];
        }
        // phi = phi_hi + (flo + snz) as an exact two-sum: phi (FP32) + r
        const float lo_sum = flo + snz;
        const float phi = phi_hi + lo_sum;
        const float bp = phi - phi_hi;
        const float r = (phi_hi - (phi - bp)) + (lo_sum - bp);

        const int cp = (ty + 2) * PX + (tx + 2), cm = cq;
        const float *mz = mus + mslot(zz) * MA;
        const float mu = mz[cm];
        float gp[3], gm[3];
        grad3(phs + pslot(zz - 1) * PA, phs + pslot(zz) * PA, phs + pslot(zz + 1) * PA, cp, PX, gp);
        grad3(mus + mslot(zz - 1) * MA, mz, mus + mslot(zz + 1) * MA, cm, MX, gm);

        float F[3], gr[3], u[3];
        const float dphi = phi - P.phiv;
        const float rho = P.rhov + dphi * P.drho;
        const float nu = P.nuv + dphi * P.dnu;
        const float inv_rho = __fdividef(1.0f, rho);
        const float itg = __fdividef(1.0f, 0.5f + 3.0f * nu);
        float j3[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (c3x(i)) j3[0] += (float)c3x(i) * gv[i];
            if (c3y(i)) j3[1] += (float)c3y(i) * gv[i];
            if (c3z(i)) j3[2] += (float)c3z(i) * gv[i];
        }
        float ugr = 0.0f, uu = 0.0f, S = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            F[d] = -phi * gm[d] + P.G[d];
            gr[d] = P.drho * gp[d];
            u[d] = (j3[d] + 0.5f * F[d]) * inv_rho;
            ugr += u[d] * gr[d];
            uu += u[d] * u[d];
            S += u[d] * gp[d];
        }
        const float p = 0.5f * (sg + 0.5f * ugr - 0.5f * rho * uu);

        if (PASS & PASS_DIAG) {
            const double u2 = (double)uu;
            d_phi += (double)phi + (double)r;
            d_E += 0.5 * (double)rho * u2;
            d_u2 = fmax(d_u2, u2);
            d_mumin = fmin(d_mumin, (double)mu);
            d_mumax = fmax(d_mumax, (double)mu);
            d_bud += 1.5 * (double)S - 0.5 * (double)Sprev;
            if (!isfinite(phi) || !isfinite(p) || !isfinite(uu) || !isfinite(mu)) d_bad = 1.0;
        }
        if (PASS & PASS_MACROS) {
            if (a.out_phi) a.out_phi[n] = (double)phi + (double)r;
            if (a.out_p) a.out_p[n] = (double)p;
            if (a.out_mu) a.out_mu[n] = (double)mu;
            if (a.out_u) {
                a.out_u[n] = (double)u[0];
                a.out_u[(size_t)N + n] = (double)u[1];
                a.out_u[2 * (size_t)N + n] = (double)u[2];
            }
        }
        if (PASS & PASS_STATE) {
            __stcs(static_cast<float *>(a.S) + n, S);
            __stcs(dst.M + n, phi);
            __stcs(dst.M + N + n, mu);
            __stcs(dst.M + 2 * N + n, p);
            __stcs(dst.M + 3 * N + n, u[0]);
            __stcs(dst.M + 4 * N + n, u[1]);
            __stcs(dst.M + 5 * N + n, u[2]);
            {
                // B = phi + alpha sum_{i != 0} w_i (mu(x + c_i) - mu(x)) from the mu ring
                const float *m0 = mz, *mm = mus + mslot(zz - 1) * MA, *mp = mus + mslot(zz + 1) * MA;
                const float fa = (m0[cm + 1] - mu) + (m0[cm - 1] - mu) + (m0[cm + MX] - mu) +
                                 (m0[cm - MX] - mu) + (mp[cm] - mu) + (mm[cm] - mu);
                const float ed = ((m0[cm + MX + 1] - mu) + (m0[cm + MX - 1] - mu) +
                                  (m0[cm - MX + 1] - mu) + (m0[cm - MX - 1] - mu)) +
                                 ((mp[cm + 1] - mu) + (mp[cm - 1] - mu) + (mm[cm + 1] - mu) +
                                  (mm[cm - 1] - mu)) +
                                 ((mp[cm + MX] - mu) + (mp[cm - MX] - mu) + (mm[cm + MX] - mu) +
                                  (mm[cm - MX] - mu));
                __stcs(dst.M + 6 * N + n, phi + P.alpha * ((1.0f / 18.0f) * fa + (1.0f / 36.0f) * ed));
            }
            // CH population (Eqs. BGK, F_i): offset = (f - f^eq)(1 - 1/tau_f) + F_i,
            // b = -5/2, -1, 1/2; the rest offset also carries the residual r of phi
            const float Sh = 1.5f * S - 0.5f * Sprev;
            const float am = P.alpha * mu;
            const float omf = 1.0f - P.inv_tauf;
            const float d0 = ((2.0f / 3.0f) * am - snz) * omf + r - (5.0f / 6.0f) * Sh;
            __stcs(dst.h + n, C::enc(d0 * it_f));
            const float fa = -(1.0f / 18.0f) * Sh, fe = (1.0f / 72.0f) * Sh;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const float w = (float)w3(i);
                __stcs(dst.h + (i * N + n), C::enc(((fv[i] - w * am) * omf + (i <= 6 ? fa : fe)) * it_f));
            }
            // hydrodynamic population (Eqs. g_i, G_i): offset = (g - g^eq)(1 - 1/tau_g) + G_i
            const float kg = 1.0f - 0.5f * itg, omg = 1.0f - itg;
            const float A = 3.0f * p - 1.5f * rho * uu;
            __stcs(dst.k + n, C::enc((gv[0] - ((1.0f / 3.0f) * A - 3.0f * p)) * omg * it_g));
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const int o = (i <= 6) ? (i % 2 ? i + 1 : i - 1)
                                       : (i <= 10 ? 17 - i : (i <= 14 ? 25 - i : 33 - i));
                if (o < i) continue;  // each pair once, from its first member
                const float w = (float)w3(i);
                const float cu = (float)c3x(i) * u[0] + (float)c3y(i) * u[1] + (float)c3z(i) * u[2];
                const float cF = (float)c3x(i) * F[0] + (float)c3y(i) * F[1] + (float)c3z(i) * F[2];
                const float cg = (float)c3x(i) * gr[0] + (float)c3y(i) * gr[1] + (float)c3z(i) * gr[2];
                const float eq_s = w * (A + 4.5f * rho * cu * cu), eq_a = 3.0f * w * rho * cu;
                const float G_s = 3.0f * w * kg * cu * cg, G_a = 3.0f * w * kg * cF;
                __stcs(dst.k + (i * N + n), C::enc(((gv[i] - eq_s - eq_a) * omg + G_s + G_a) * it_g));
                __stcs(dst.k + (o * N + n), C::enc(((gv[o] - eq_s + eq_a) * omg + G_s - G_a) * it_g));
            }
        }
        }  // col_ok
        cp_wait_all();
        __syncthreads();
        for (int q = tid; q < MA; q += TX3 * TY3) {  // own copies: no barrier needed
            float m6[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) m6[c] = mraw[c * MA + q];
            put_macros(qslot(zz + 2), q, m6);
        }
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

// ------------------------------------------------- state in the paper's form

// equilibria of the stored macros of node m (the arithmetic of the pass kernel)
struct EqData {
    float q0, A, j[3], q5;
};
__device__ inline EqData eq_data(const StepParams<float> &P, const float *M, size_t N, size_t m)
{
    const float ph = M[m], mu = M[N + m], p = M[2 * N + m];
    const float u[3] = {M[3 * N + m], M[4 * N + m], M[5 * N + m]};
    const float rho = P.rhov + (ph - P.phiv) * P.drho;
    EqData e;
    e.q0 = P.alpha * mu;
    e.A = 3.0f * p - 1.5f * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int d = 0; d < 3; ++d) e.j[d] = rho * u[d];
    e.q5 = 4.5f / rho;
    return e;
}
__device__ inline double feq_of(const EqData &e, float phi_hi, int i)
{
    return i == 0 ? (double)phi_hi - (double)((2.0f / 3.0f) * e.q0) : (double)((float)w3(i) * e.q0);
}
__device__ inline double geq_of(const EqData &e, float p, int i)
{
    if (i == 0) return (double)((1.0f / 3.0f) * e.A - 3.0f * p);
    float cj = 0.0f;
    if (c3x(i)) cj += (float)c3x(i) * e.j[0];
    if (c3y(i)) cj += (float)c3y(i) * e.j[1];
    if (c3z(i)) cj += (float)c3z(i) * e.j[2];
    return (double)((float)w3(i) * (e.A + cj * (3.0f + e.q5 * cj)));
}

// initial state: macros (phi0, mu0, p = 0, u = 0) at every node, f_i(x, 0) =
// f^eq_i(phi0(x), mu0(x)) stored at x - c_i as an offset from the
// equilibrium of the storing node's macros; g = g^eq (offsets 0)
template <class C>
__global__ void d3q19_off_init_k(const StepParams<double> Pd, const StepParams<float> P,
                                 const double *__restrict__ phi0, const double *__restrict__ mu0,
                                 OffBuf o, float *__restrict__ S, float s_f, float s_g)
{
    const size_t N = (size_t)P.N;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) {
        o.sc[0] = s_f;
        o.sc[1] = s_g;
    }
    if (n >= N) return;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    const float phi_hi = (float)phi0[n], mu_f = (float)mu0[n];
    o.M[n] = phi_hi;
    o.M[N + n] = mu_f;
    for (int k = 2; k < 6; ++k) o.M[k * N + n] = 0.0f;
    S[n] = 0.0f;
    const float q0 = P.alpha * mu_f;
    for (int i = 0; i < 19; ++i) {
        const unsigned m = b.at(c3x(i), c3y(i), c3z(i));
        const double am = Pd.alpha * mu0[m];
        const double fe = i == 0 ? phi0[m] - (1.0 - w3(0)) * am : w3(i) * am;
        const double eq = i == 0 ? (double)phi_hi - (double)((2.0f / 3.0f) * q0)
                                 : (double)((float)w3(i) * q0);
        o.h[i * N + n] = C::enc((float)((fe - eq) / (double)s_f));
        o.k[i * N + n] = 0;  // +0 in both formats
    }
}

template <class C>
__global__ void d3q19_off_get_k(const StepParams<float> P, const OffBuf o,
                                const float *__restrict__ S, double *fo, double *go, double *So)
{
    const size_t N = (size_t)P.N;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    const double s_f = o.sc[0], s_g = o.sc[1];
    for (int i = 0; i < 19; ++i) {
        const unsigned m = b.at(-c3x(i), -c3y(i), -c3z(i));
        const EqData e = eq_data(P, o.M, N, m);
        if (fo) fo[i * N + n] = feq_of(e, o.M[m], i) + s_f * (double)C::dec(o.h[i * N + m]);
        if (go) go[i * N + n] = geq_of(e, o.M[2 * N + m], i) + s_g * (double)C::dec(o.k[i * N + m]);
    }
    if (So) So[n] = (double)S[n];
}

// macros of the storing node from its own stored values: phi = sum f*,
// mu from sum_{i != 0} f* = (1 - w0) alpha mu, u = sum c g* / rho,
// p = sum_{i != 0} g* / 2; the offsets carry the rest exactly (up to rounding)
template <class C>
__global__ void d3q19_off_set_k(const StepParams<float> P, OffBuf o, float *__restrict__ S,
                                const double *fi, const double *gi, const double *Si, float s_f,
                                float s_g)
{
    const size_t N = (size_t)P.N;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) {
        o.sc[0] = s_f;
        o.sc[1] = s_g;
    }
    if (n >= N) return;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((size_t)nx * ny));
    const Nb b = make_nb(x, y, z, nx, ny, nz);
    double fs[19], gs[19];
    double sphi = 0.0, snz = 0.0, sg = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        const unsigned m = b.at(c3x(i), c3y(i), c3z(i));
        fs[i] = fi[i * N + m];
        gs[i] = gi[i * N + m];
        sphi += fs[i];
        if (i) {
            snz += fs[i];
            sg += gs[i];
            j[0] += c3x(i) * gs[i];
            j[1] += c3y(i) * gs[i];
            j[2] += c3z(i) * gs[i];
        }
    }
    const float phi_hi = (float)sphi;
    const float rho = P.rhov + (phi_hi - P.phiv) * P.drho;
    o.M[n] = phi_hi;
    o.M[N + n] = (float)(snz / ((1.0 - w3(0)) * (double)P.alpha));
    o.M[2 * N + n] = (float)(0.5 * sg);
    for (int d = 0; d < 3; ++d) o.M[(3 + d) * N + n] = (float)(j[d] / (double)rho);
    S[n] = (float)Si[n];
    const EqData e = eq_data(P, o.M, N, n);
    for (int i = 0; i < 19; ++i) {
        o.h[i * N + n] = C::enc((float)((fs[i] - feq_of(e, phi_hi, i)) / (double)s_f));
        o.k[i * N + n] = C::enc((float)((gs[i] - geq_of(e, o.M[2 * N + n], i)) / (double)s_g));
    }
}

// one population value of the paper's form written into the storage
template <class C>
__global__ void d3q19_off_poke_k(const StepParams<float> P, OffBuf o, int field, int i,
                                 size_t m, double value)
{
    const size_t N = (size_t)P.N;
    const EqData e = eq_data(P, o.M, N, m);
    if (field == 0)
        o.h[i * N + m] = C::enc((float)((value - feq_of(e, o.M[m], i)) / (double)o.sc[0]));
    else
        o.k[i * N + m] = C::enc((float)((value - geq_of(e, o.M[2 * N + m], i)) / (double)o.sc[1]));
}

// ---------------------------------------------------------------- scales

// max over |stored value| bit patterns (monotonic in the magnitude for both
// formats); NaN patterns are larger than INF_BITS
__global__ void off_absmax_k(const unsigned short *__restrict__ v, size_t count,
                             unsigned *__restrict__ out)
{
    unsigned m = 0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (size_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned)(__ldg(v + q) & 0x7fffu));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <class C>
__global__ void off_target_k(const OffBuf cur, const unsigned *__restrict__ maxbits,
                             float *__restrict__ target)
{
    for (int k = 0; k < 2; ++k) {
        const unsigned bits = maxbits[k];
        if (bits >= C::INF_BITS) continue;  // overflowed or NaN: keep (diagnostics report it)
        const float m = C::dec((unsigned short)bits) * cur.sc[k];
        float t = OFFSET_SCALE_FLOOR;
        if (m > 0.0f) {
            int e;
            frexpf(m * (1.0f / OFFSET_HEADROOM), &e);
            t = fmaxf(t, ldexpf(1.0f, e));
        }
        target[k] = t;
    }
}

template <class C>
int off_ctas_per_sm_t()
{
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, d3q19_off_pass_kernel<C, PASS_STATE>, TX3 * TY3, 0);
    return e == cudaSuccess && n > 0 ? n : 2;
}

template <class C, int PASS>
cudaError_t launch_off(const StepParams<float> &P, const PassArgs &a, const LaunchShape &s,
                       float *phi, const float *target, cudaStream_t st)
{
    const OffBuf src = off_view(a.f_src, a.g_src, P.N), dst = off_view(a.f_dst, a.g_dst, P.N);
    const dim3 pg((P.nx + PHI_TX - 1) / PHI_TX, P.ny, P.nz);
    d3q19_off_phi_kernel<C><<<pg, PHI_TX, 0, st>>>(P, src, phi);
    dim3 grid(s.grid_x, s.grid_y, s.nblocks / (s.grid_x * s.grid_y)), block(TX3, TY3);
    d3q19_off_pass_kernel<C, PASS><<<grid, block, 0, st>>>(P, a, src, dst, target, phi, s.rows);
    return cudaGetLastError();
}

template <class C>
cudaError_t pass_off_t(int pass, const StepParams<float> &P, const PassArgs &a,
                       const LaunchShape &s, float *phi, const float *target, cudaStream_t st)
{
    switch (pass) {
    case PASS_STATE: return launch_off<C, PASS_STATE>(P, a, s, phi, target, st);
    case PASS_STATE | PASS_DIAG: return launch_off<C, PASS_STATE | PASS_DIAG>(P, a, s, phi, target, st);
    case PASS_MACROS: return launch_off<C, PASS_MACROS>(P, a, s, phi, target, st);
    case PASS_DIAG: return launch_off<C, PASS_DIAG>(P, a, s, phi, target, st);
    case PASS_MACROS | PASS_DIAG: return launch_off<C, PASS_MACROS | PASS_DIAG>(P, a, s, phi, target, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int d3q19_off_ctas_per_sm(int codec)
{
    return codec == OFFSET_F16 ? off_ctas_per_sm_t<CodecF16>() : off_ctas_per_sm_t<CodecBF16>();
}

cudaError_t d3q19_off_pass(int codec, int pass, const void *params32, const PassArgs &a,
                           const LaunchShape &s, void *phi_work, const float *target,
                           cudaStream_t st)
{
    const StepParams<float> &P = *static_cast<const StepParams<float> *>(params32);
    return codec == OFFSET_F16
               ? pass_off_t<CodecF16>(pass, P, a, s, (float *)phi_work, target, st)
               : pass_off_t<CodecBF16>(pass, P, a, s, (float *)phi_work, target, st);
}

cudaError_t d3q19_off_init(int codec, const void *params64, const void *params32,
                           const double *phi0, double *mu_tmp, void *f, void *g, void *S,
                           const float *target_host, cudaStream_t st)
{
    const StepParams<double> &Pd = *static_cast<const StepParams<double> *>(params64);
    const StepParams<float> &P = *static_cast<const StepParams<float> *>(params32);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    cudaError_t e = d3q19_init_mu_fp64(params64, phi0, mu_tmp, st);
    if (e != cudaSuccess) return e;
    const OffBuf o = off_view(f, g, P.N);
    if (codec == OFFSET_F16)
        d3q19_off_init_k<CodecF16><<<nb, 256, 0, st>>>(Pd, P, phi0, mu_tmp, o, (float *)S,
                                                       target_host[0], target_host[1]);
    else
        d3q19_off_init_k<CodecBF16><<<nb, 256, 0, st>>>(Pd, P, phi0, mu_tmp, o, (float *)S,
                                                        target_host[0], target_host[1]);
    d3q19_off_prep_k<<<dim3((P.nx + PHI_TX - 1) / PHI_TX, P.ny, P.nz), PHI_TX, 0, st>>>(P, o);
    return cudaGetLastError();
}

cudaError_t d3q19_off_get_state(int codec, const void *params32, const void *f, const void *g,
                                const void *S, double *fo, double *go, double *So, cudaStream_t st)
{
    const StepParams<float> &P = *static_cast<const StepParams<float> *>(params32);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    const OffBuf o = off_view(f, g, P.N);
    if (codec == OFFSET_F16)
        d3q19_off_get_k<CodecF16><<<nb, 256, 0, st>>>(P, o, (const float *)S, fo, go, So);
    else
        d3q19_off_get_k<CodecBF16><<<nb, 256, 0, st>>>(P, o, (const float *)S, fo, go, So);
    return cudaGetLastError();
}

cudaError_t d3q19_off_set_state(int codec, const void *params32, void *f, void *g, void *S,
                                const double *fi, const double *gi, const double *Si,
                                const float *target_host, cudaStream_t st)
{
    const StepParams<float> &P = *static_cast<const StepParams<float> *>(params32);
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    const OffBuf o = off_view(f, g, P.N);
    if (codec == OFFSET_F16)
        d3q19_off_set_k<CodecF16><<<nb, 256, 0, st>>>(P, o, (float *)S, fi, gi, Si,
                                                      target_host[0], target_host[1]);
    else
        d3q19_off_set_k<CodecBF16><<<nb, 256, 0, st>>>(P, o, (float *)S, fi, gi, Si,
                                                       target_host[0], target_host[1]);
    d3q19_off_prep_k<<<dim3((P.nx + PHI_TX - 1) / PHI_TX, P.ny, P.nz), PHI_TX, 0, st>>>(P, o);
    return cudaGetLastError();
}

cudaError_t d3q19_off_poke(int codec, const void *params32, void *f, void *g, int field, int i,
                           size_t m, double value, cudaStream_t st)
{
    const StepParams<float> &P = *static_cast<const StepParams<float> *>(params32);
    const OffBuf o = off_view(f, g, P.N);
    if (codec == OFFSET_F16)
        d3q19_off_poke_k<CodecF16><<<1, 1, 0, st>>>(P, o, field, i, m, value);
    else
        d3q19_off_poke_k<CodecBF16><<<1, 1, 0, st>>>(P, o, field, i, m, value);
    return cudaGetLastError();
}

cudaError_t offset_refresh(int codec, long long N, int Q, const void *f, const void *g,
                           unsigned *maxbits, float *target, int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(maxbits, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const size_t count = (size_t)Q * (size_t)N;
    const unsigned nb = (unsigned)(4 * (num_sms > 0 ? num_sms : 152));
    off_absmax_k<<<nb, 256, 0, st>>>((const unsigned short *)f, count, maxbits);
    off_absmax_k<<<nb, 256, 0, st>>>((const unsigned short *)g, count, maxbits + 1);
    const OffBuf cur = off_view(f, g, N);
    if (codec == OFFSET_F16)
        off_target_k<CodecF16><<<1, 1, 0, st>>>(cur, maxbits, target);
    else
        off_target_k<CodecBF16><<<1, 1, 0, st>>>(cur, maxbits, target);
    return cudaGetLastError();
}

}  // namespace wblbm
