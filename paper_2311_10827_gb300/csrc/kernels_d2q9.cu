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
// Row tiles march in alternating directions (even tiles down, odd tiles up),
// so two neighbouring tiles reach their shared boundary rows at the same
// time and the y-halo rows are served from L2 instead of being re-read from
// HBM; every other step reverses all directions, so a step starts on the
// rows the previous step wrote last (still in L2 when a step's data is
// comparable to the L2 size).
//
// FP32 storage keeps the rest population f_0 (~phi, O(1)) as a compensated
// pair hi + lo of FP32 words (lo in population slot 9): its per-step change
// near equilibrium (~1e-9) is below half an FP32 ulp of 1, so a plain FP32
// f_0 would stagnate and phi would drift.  The pair is updated with an exact
// two-sum; all arithmetic stays FP32.  FP64 storage has no lo slot.
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
struct Arith;
template <>
struct Arith<float> {
    // reciprocal to ~1 ulp (rho and tau_g are O(1); FP32 rounding elsewhere dominates)
    __device__ static float rcp(float x) { return __fdividef(1.0f, x); }
};
template <>
struct Arith<double> {
    __device__ static double rcp(double x) { return 1.0 / x; }
};

// row index wrap for rows in [-n, 2n) (n >= 4), any row otherwise
__device__ __forceinline__ int wrap_row(int r, int n, bool small)
{
    if (small) return wrapi(r, n);
    return r < 0 ? r + n : (r >= n ? r - n : r);
}

// Load of a population: through the read-only path (NC, data constant for
// the launch), or from L2 only (data that other CTAs write during the same
// launch: the multi-step kernel).
template <bool NC, typename T>
__device__ __forceinline__ T ldp(const T *p)
{
    return NC ? __ldg(p) : __ldcg(p);
}

// The nine populations arriving at (x, y): v[i] = src_i(x - cx_i, y - cy_i).
// rm/r0/rp are the offsets of rows y-1, y, y+1; xm/x/xp the wrapped columns.
// Offsets are 32-bit (Q N < 2^32 is checked at context creation).
template <bool NC, typename T>
__device__ __forceinline__ void pull9(const T *__restrict__ s, unsigned N, unsigned rm, unsigned r0,
                                      unsigned rp, unsigned xm, unsigned x, unsigned xp, T v[9])
{
    v[0] = ldp<NC>(s + (r0 + x));
    v[1] = ldp<NC>(s + (1u * N + rp + x));   // c = (0,-1) comes from y + 1
    v[2] = ldp<NC>(s + (2u * N + r0 + xm));  // c = (1,0)  comes from x - 1
    v[3] = ldp<NC>(s + (3u * N + rm + x));   // c = (0,1)  comes from y - 1
    v[4] = ldp<NC>(s + (4u * N + r0 + xp));  // c = (-1,0) comes from x + 1
    v[5] = ldp<NC>(s + (5u * N + rm + xm));  // c = (1,1)
    v[6] = ldp<NC>(s + (6u * N + rm + xp));  // c = (-1,1)
    v[7] = ldp<NC>(s + (7u * N + rp + xp));  // c = (-1,-1)
    v[8] = ldp<NC>(s + (8u * N + rp + xm));  // c = (1,-1)
}

// Per-thread asynchronous copy global -> shared (4 or 8 bytes) and its
// group fences: a thread's own copies are visible to it after wait_group.
template <typename T>
__device__ __forceinline__ void cp_async(T *dst, const T *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one()
{
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// the nine pull addresses of (x, y) (same order as pull9)
template <typename T>
__device__ __forceinline__ void stage9(T *dst, int stride, const T *__restrict__ s, unsigned N,
                                       unsigned rm, unsigned r0, unsigned rp, unsigned xm,
                                       unsigned x, unsigned xp)
{
    cp_async(dst + 0 * stride, s + (r0 + x));
    cp_async(dst + 1 * stride, s + (1u * N + rp + x));
    cp_async(dst + 2 * stride, s + (2u * N + r0 + xm));
    cp_async(dst + 3 * stride, s + (3u * N + rm + x));
    cp_async(dst + 4 * stride, s + (4u * N + r0 + xp));
    cp_async(dst + 5 * stride, s + (5u * N + rm + xm));
    cp_async(dst + 6 * stride, s + (6u * N + rm + xp));
    cp_async(dst + 7 * stride, s + (7u * N + rp + xp));
    cp_async(dst + 8 * stride, s + (8u * N + rp + xm));
}

// sum of the eight moving populations, fixed pairing (the rest population is
// added last so that phi = f_0 + s keeps the small terms exact in FP32)
template <typename T>
__device__ __forceinline__ T sum_moving(const T v[9])
{
    return ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
}

// Stores of the step's outputs are ordinary write-back stores: the next step
// reads them, and with the march reversed every step the rows a tile wrote
// last -- the ones most likely still in L2 -- are read first.
template <typename T>
__device__ __forceinline__ void st_stream(T *p, T v)
{
    *p = v;
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

// resident CTAs per SM targeted by the register budget of each precision
// resident CTAs per SM targeted by the register budget: the FP32 time step
// fits 64 registers (1024 threads per SM); variants carrying the FP64
// diagnostics accumulators get 80 (768 threads), FP64 512 threads
template <typename T, int PASS, int TX>
struct Occ {
    static constexpr int threads = sizeof(T) == 4 ? ((PASS & PASS_DIAG) ? 768 : 1024) : 512;
    static constexpr int ctas = threads / (TX * TYB) > 0 ? threads / (TX * TYB) : 1;
};

// One tile: columns [x0, x0 + TX), rows [y0, yend), marching in direction
// dir (+1 down from y0, -1 up from yend - 1); diagnostics partial record
// `part` (PASS_DIAG).  Shared by the single-grid and the batched kernels.
template <typename T, int TX, int PASS, bool NC = true>
__device__ __forceinline__ void d2q9_tile(const StepParams<T> &P, const PassArgs &a, int x0, int y0,
                                          int yend, int dir, int part)
{
    constexpr int R = 2 * TYB + 3;  // ring depth: writes never hit a row still read
    constexpr bool REST_PAIR = sizeof(T) == 4;
    constexpr int WP = TX + 4;      // phi ring width (halo 2)
    constexpr int WM = TX + 2;      // mu ring width (halo 1)
    __shared__ T phs[R * WP];
    __shared__ T mus[R * WM];
    // FP32: the f pulls of the next iteration's phi row are staged here by
    // per-thread asynchronous copies (two stages) while this iteration runs
    constexpr bool STAGE = sizeof(T) == 4;
    constexpr int NT = TX * TYB, NFS = REST_PAIR ? 10 : 9;
    __shared__ T fst[STAGE ? 2 * NFS * NT : 1];
    __shared__ T fsh[STAGE ? 2 * NFS * 4 * TYB : 1];
    const int lin = threadIdx.y * TX + threadIdx.x;

    const int nx = P.nx, ny = P.ny;
    const unsigned N = (unsigned)P.N;
    const bool small = ny < 4;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const T *__restrict__ fsrc = static_cast<const T *>(a.f_src);
    const T *__restrict__ gsrc = static_cast<const T *>(a.g_src);

    // own column (phi ring index tx + 2, mu ring index tx + 1)
    const int xo = x0 + tx;
    const bool col_ok = xo < nx;
    const unsigned xO = wrapi(xo, nx), xOm = wrapi(xo - 1, nx), xOp = wrapi(xo + 1, nx);
    // phi halo column handled by threads 0..3: ring index 0, 1, TX+2, TX+3
    const int jH = tx < 2 ? tx : TX + tx;
    const int cH = x0 - 2 + jH;
    const unsigned xH = wrapi(cH, nx), xHm = wrapi(cH - 1, nx), xHp = wrapi(cH + 1, nx);
    // mu halo column handled by threads 0, 1: ring index 0 and TX+1
    const int jM = tx == 0 ? 0 : TX + 1;

    // FP32: equilibrium shift of the source buffer and of the writes (a uniform
    // shift of mu in f^eq; phi, the moments and the stencils do not see it, so
    // only a time step reads it)
    T a_src = T(0), a_dst = T(0);
    if (REST_PAIR && (PASS & PASS_STATE)) {
        a_src = *a.eqs_src;
        a_dst = *a.eqs_target;
        if (a.eqs_dst && x0 == 0 && y0 == 0 && lin == 0) *a.eqs_dst = a_dst;
    }

    // m(row) = dir (row - first) is the march coordinate, >= -2 for every row used
    const int first = dir > 0 ? y0 : yend - 1;
    const int nout = yend - y0;
    auto slot = [&](int row) { return (dir * (row - first) + 2) % R; };

    // phi = f_0 + rest into ring slot sl, column j
    auto put_phi = [&](int sl, int j, T f0, T rest) { phs[sl * WP + j] = f0 + rest; };
    // phi at row `row` for the own column (keeping the pulled values) and the
    // halo columns.
    auto phi_row = [&](int row, int sl, T v[9], T &lo) {
        const unsigned rm = (unsigned)wrap_row(row - 1, ny, small) * nx;
        const unsigned r0 = (unsigned)wrap_row(row, ny, small) * nx;
        const unsigned rp = (unsigned)wrap_row(row + 1, ny, small) * nx;
        pull9<NC>(fsrc, N, rm, r0, rp, xOm, xO, xOp, v);
        lo = REST_PAIR ? ldp<NC>(fsrc + (9u * N + r0 + xO)) : T(0);
        put_phi(sl, tx + 2, v[0], lo + sum_moving(v));
        if (tx < 4) {
            T h[9];
            pull9<NC>(fsrc, N, rm, r0, rp, xHm, xH, xHp, h);
            const T hlo = REST_PAIR ? ldp<NC>(fsrc + (9u * N + r0 + xH)) : T(0);
            put_phi(sl, jH, h[0], hlo + sum_moving(h));
        }
    };

    // issue the copies of phi row `row`'s pulls into stage st (FP32 only)
    auto issue_phi_row = [&](int row, int st) {
        const unsigned rm = (unsigned)wrap_row(row - 1, ny, small) * nx;
        const unsigned r0 = (unsigned)wrap_row(row, ny, small) * nx;
        const unsigned rp = (unsigned)wrap_row(row + 1, ny, small) * nx;
        T *d = fst + (size_t)st * NFS * NT + lin;
        stage9(d, NT, fsrc, N, rm, r0, rp, xOm, xO, xOp);
        if (REST_PAIR) cp_async(d + 9 * NT, fsrc + (9u * N + r0 + xO));
        if (tx < 4) {
            T *h = fsh + (size_t)st * NFS * 4 * TYB + ty * 4 + tx;
            stage9(h, 4 * TYB, fsrc, N, rm, r0, rp, xHm, xH, xHp);
            if (REST_PAIR) cp_async(h + 9 * 4 * TYB, fsrc + (9u * N + r0 + xH));
        }
    };
    // phi row from stage st (the copies have landed)
    auto phi_row_staged = [&](int sl, int st, T v[9], T &lo) {
        const T *d = fst + (size_t)st * NFS * NT + lin;
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = d[i * NT];
        lo = REST_PAIR ? d[9 * NT] : T(0);
        put_phi(sl, tx + 2, v[0], lo + sum_moving(v));
        if (tx < 4) {
            const T *h = fsh + (size_t)st * NFS * 4 * TYB + ty * 4 + tx;
            T hv[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) hv[i] = h[i * 4 * TYB];
            const T hlo = REST_PAIR ? h[9 * 4 * TYB] : T(0);
            put_phi(sl, jH, hv[0], hlo + sum_moving(hv));
        }
    };

    // Eq. chemical_potencial with the Laplacian of Eq. Laplace, written as a
    // sum of differences (cancellation-friendly in FP32):
    // lap = (2/3) sum_axis (phi_n - phi) + (1/6) sum_diag (phi_n - phi).
    auto mu_at = [&](int sm, int s0, int sp, int j) -> T {
        // j is the mu ring index; the phi ring index of the same column is j+1
        const T *pm = phs + sm * WP, *p0 = phs + s0 * WP, *pp = phs + sp * WP;
        const T c = p0[j + 1];
        const T ax = (p0[j + 2] - c) + (p0[j] - c) + (pp[j + 1] - c) + (pm[j + 1] - c);
        const T dg = (pp[j + 2] - c) + (pp[j] - c) + (pm[j + 2] - c) + (pm[j] - c);
        const T lap = T(2.0 / 3.0) * ax + T(1.0 / 6.0) * dg;
        const T bulk = T(4) * P.beta * (c - P.phil) * (c - P.phiv) * (c - P.phibar);
        return bulk - P.kappa * lap;
    };
    // mu at the row with ring slot s0; sm / sp are the slots of rows y-1 / y+1
    auto mu_row = [&](int sm, int s0, int sp) {
        T *mr = mus + s0 * WM;
        mr[tx + 1] = mu_at(sm, s0, sp, tx + 1);
        if (tx < 2) mr[jM] = mu_at(sm, s0, sp, jM);
    };

    double d_phi = 0.0, d_E = 0.0, d_u2 = 0.0, d_mumin = DBL_MAX, d_mumax = -DBL_MAX,
           d_bud = 0.0, d_bad = 0.0;

    // prologue: phi rows y0-2 .. y0+1 (the own row y0+ty keeps its values),
    // mu rows y0-1 .. y0
    T fcur[9], fnext[9], locur, lonext;
    phi_row(first + dir * (ty - 2), slot(first + dir * (ty - 2)), fnext, lonext);
    phi_row(first + dir * ty, slot(first + dir * ty), fcur, locur);
    __syncthreads();
    {
        const int r = first + dir * (ty - 1);
        mu_row(slot(r - 1), slot(r), slot(r + 1));
    }
    __syncthreads();
    if (STAGE) {
        issue_phi_row(first + dir * (2 + ty), 0);
        cp_commit();
    }

    // ring slot of march coordinate t + k is (rb + k) mod R with rb = (t + 2) mod R
    int rb = 2 % R;
    for (int t = 0; t < nout; t += TYB) {
        auto ring = [&](int k) {
            int v = rb + k;
            v = v >= R ? v - R : v;
            return v < 0 ? v + R : v;
        };
        const int row = first + dir * (t + ty);
        const bool out_ok = col_ok && t + ty < nout;
        // issue the loads of the own node first so they overlap the stencil work
        T gv[9];
        T Sprev = T(0);
        const unsigned nrow = (unsigned)wrap_row(row, ny, small) * nx;
        {
            const unsigned rm = (unsigned)wrap_row(row - 1, ny, small) * nx;
            const unsigned rp = (unsigned)wrap_row(row + 1, ny, small) * nx;
            pull9<NC>(gsrc, N, rm, nrow, rp, xOm, xO, xOp, gv);
            if ((PASS & (PASS_STATE | PASS_DIAG)) && out_ok)
                Sprev = __ldcs(static_cast<const T *>(a.S) + (nrow + xo));
        }
        if (STAGE) {
            const int st = (t / TYB) & 1;
            if (t + TYB < nout) issue_phi_row(first + dir * (t + TYB + 2 + ty), st ^ 1);
            cp_commit();  // possibly empty: one group per iteration
            cp_wait_all_but_one();
            phi_row_staged(ring(2 + ty), st, fnext, lonext);
        } else {
            phi_row(first + dir * (t + 2 + ty), ring(2 + ty), fnext, lonext);
        }
        __syncthreads();
        mu_row(ring(1 + ty - dir), ring(1 + ty), ring(1 + ty + dir));
        __syncthreads();

        const int sm = ring(ty - dir), s0 = ring(ty), sp = ring(ty + dir);
        rb += TYB;
        rb = rb >= R ? rb - R : rb;
        if (out_ok) {
            const T *pm = phs + sm * WP;
            const T *p0 = phs + s0 * WP;
            const T *pp = phs + sp * WP;
            const T *mm = mus + sm * WM;
            const T *m0 = mus + s0 * WM;
            const T *mp = mus + sp * WM;
            const int j = tx + 2;  // phi ring index of the own column
            const int k = tx + 1;  // mu ring index of the own column

            // phi from the pulled values (Eq. order-parameter)
            const T snz = sum_moving(fcur);
            const T phi = fcur[0] + (locur + snz);
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
            const T inv_rho = Arith<T>::rcp(rho);
            const T itg = Arith<T>::rcp(T(0.5) + T(3) * nu);  // nu = cs2 (tau_g - 1/2)

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
                const size_t n = (size_t)nrow + xo;
                if (a.out_phi) a.out_phi[n] = (double)phi;
                if (a.out_p) a.out_p[n] = (double)p;
                if (a.out_mu) a.out_mu[n] = (double)mu;
                if (a.out_u) {
                    a.out_u[n] = (double)ux;
                    a.out_u[(size_t)N + n] = (double)uy;
                }
            }
            if (PASS & PASS_MACROS_T) {
                const size_t n = (size_t)nrow + xo;
                static_cast<T *>(a.mt_phi)[n] = phi;
                static_cast<T *>(a.mt_p)[n] = p;
                static_cast<T *>(a.mt_mu)[n] = mu;
                static_cast<T *>(a.mt_u)[n] = ux;
                static_cast<T *>(a.mt_u)[(size_t)N + n] = uy;
            }
            if (PASS & PASS_STATE) {
                const unsigned n = nrow + xo;
                T *__restrict__ fd = static_cast<T *>(a.f_dst);
                T *__restrict__ gd = static_cast<T *>(a.g_dst);
                st_stream(static_cast<T *>(a.S_out) + n, S);

                // CH population, Eq. BGK with Eq. H_i and Eq. F_i:
                // f* = f - (f - f^eq)/tau_f + w_i b_i (1.5 S - 0.5 S_prev),
                // b = -2, -1/2, 1 (rest, axis, diagonal); f_0 - f_0^eq is formed
                // as (5/9) alpha mu - sum_{i!=0} f_i (no cancellation against phi).
                // Every population is updated by its own small increment, so
                // the increments sum to sum_i F_i up to unbiased rounding (the
                // form f (1 - 1/tau) + f^eq/tau would add (1 - 1/tau + 1/tau - 1)
                // sum_{i!=0} f_i, a systematic FP32 drift of the phi mass).
                const T Sh = T(1.5) * S - T(0.5) * Sprev;
                // alpha mu in the source buffer's shifted variables; dsh moves
                // the written values to the target shift (0 unless it changed)
                const T am = P.alpha * mu - a_src;
                const T dsh = a_src - a_dst;
                const T itf = P.inv_tauf;
                {
                    // f_0* = f_0 - (f_0 - f_0^eq)/tau_f - (8/9) Sh with
                    // f_0 - f_0^eq = (5/9) alpha mu - sum_{i!=0} f_i
                    const T d0 = -(T(5.0 / 9.0) * am - snz) * itf - T(8.0 / 9.0) * Sh -
                                 T(5.0 / 9.0) * dsh;
                    if (REST_PAIR) {
                        // (hi, lo) + d0 with an exact two-sum on the high word
                        const T sl = locur + d0;
                        const T hi = fcur[0] + sl;
                        const T bp = hi - fcur[0];
                        const T lo = (fcur[0] - (hi - bp)) + (sl - bp);
                        st_stream(fd + n, hi);
                        st_stream(fd + (9u * N + n), lo);
                    } else {
                        st_stream(fd + n, fcur[0] + d0);
                    }
                }
                const T ea = T(1.0 / 9.0) * am, ed = T(1.0 / 36.0) * am;
                const T sa = T(-1.0 / 18.0) * Sh + T(1.0 / 9.0) * dsh;
                const T sd = T(1.0 / 36.0) * Sh + T(1.0 / 36.0) * dsh;
#pragma unroll
                for (int i = 1; i <= 4; ++i)
                    st_stream(fd + (i * N + n), fcur[i] + ((ea - fcur[i]) * itf + sa));
#pragma unroll
                for (int i = 5; i <= 8; ++i)
                    st_stream(fd + (i * N + n), fcur[i] + ((ed - fcur[i]) * itf + sd));

                // Hydrodynamic population, Eq. BGK-NS with Eqs. G_i, Siu, GGi:
                // g* = g + (g^eq - g)/tau_g + G_i.  With A = 3p - 1.5 rho |u|^2,
                // g^eq_i = w_i [A + 4.5 rho (c.u)^2] + 3 w_i rho (c.u) (i != 0), and
                // G_i = (1 - 1/(2 tau_g)) w_i [u.grad rho + c.F/cs2
                //       + ((c.u)(c.grad rho) - cs2 u.grad rho)/cs2]
                //     = 3 w_i k [c.F + (c.u)(c.grad rho)], k = 1 - 1/(2 tau_g)
                // (the two u.grad rho terms cancel).  Opposite directions share
                // the even part and flip the odd part.
                const T kg = T(1) - T(0.5) * itg;
                const T A = T(3) * p - T(1.5) * rho * uu;
                st_stream(gd + n, gv[0] + ((T(4.0 / 9.0) * A - T(3) * p) - gv[0]) * itg);  // G_0 = 0
                const T cu_[4] = {ux, uy, ux + uy, uy - ux};
                const T cF_[4] = {Fx, Fy, Fx + Fy, Fy - Fx};
                const T cg_[4] = {grx, gry, grx + gry, gry - grx};
                constexpr int ip[4] = {2, 3, 5, 6}, im[4] = {4, 1, 7, 8};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T w = q < 2 ? T(1.0 / 9.0) : T(1.0 / 36.0);
                    const T cu = cu_[q];
                    const T eq_s = w * (A + T(4.5) * rho * cu * cu), eq_a = T(3) * w * rho * cu;
                    const T G_s = T(3) * w * kg * cu * cg_[q], G_a = T(3) * w * kg * cF_[q];
                    const T gp = gv[ip[q]], gm = gv[im[q]];
                    st_stream(gd + (ip[q] * N + n), gp + ((eq_s + eq_a - gp) * itg + (G_s + G_a)));
                    st_stream(gd + (im[q] * N + n), gm + ((eq_s - eq_a - gm) * itg + (G_s - G_a)));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) fcur[i] = fnext[i];
        locur = lonext;
    }
    if (!NC) cp_wait_all();  // the next step of a multi-step launch reuses the stages

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
            a.partials[part] = o;
        }
    }
}

// Single grid: CTA (bx, by) owns strip bx and row tile by; even row tiles
// march down, odd ones up, so neighbouring tiles meet at their shared rows.
template <typename T, int TX, int PASS>
__global__ void __launch_bounds__(TX *TYB, (Occ<T, PASS, TX>::ctas))
    d2q9_pass_kernel(const StepParams<T> P, PassArgs a, int rows)
{
    const int y0 = blockIdx.y * rows;
    // march direction: alternating between neighbouring row tiles, and
    // reversed on every other step
    const int dir = ((blockIdx.y & 1) ? -1 : 1) * (a.flip ? -1 : 1);
    d2q9_tile<T, TX, PASS>(P, a, blockIdx.x * TX, y0, min(y0 + rows, P.ny), dir,
                           blockIdx.y * gridDim.x + blockIdx.x);
}

// Batched: CTA k runs tile k of a flat tile table over many independent grids
// (each with its own size and parameters); buffers are picked by the step
// parity shared by all cases.  S is read from S and written to S_out.
template <typename T, int TX, int PASS>
__global__ void __launch_bounds__(TX *TYB, (Occ<T, PASS, TX>::ctas))
    d2q9_batch_kernel(const BatchCase *__restrict__ cases, const BatchTile *__restrict__ tiles,
                      int parity, DiagPartial *partials)
{
    const BatchTile t = tiles[blockIdx.x];
    const BatchCase &c = cases[t.c];
    const StepParams<T> P = *reinterpret_cast<const StepParams<T> *>(
        sizeof(T) == 4 ? (const void *)&c.pf : (const void *)&c.pd);
    PassArgs a;
    a.f_src = c.f[parity];
    a.f_dst = c.f[parity ^ 1];
    a.g_src = c.g[parity];
    a.g_dst = c.g[parity ^ 1];
    a.S = c.S;
    a.S_out = c.S_out;
    a.out_phi = a.out_p = a.out_u = a.out_mu = nullptr;
    a.partials = partials;
    a.eqs_src = c.eqs + parity;
    a.eqs_dst = c.eqs + (parity ^ 1);
    a.eqs_target = c.eqs + 2;
    d2q9_tile<T, TX, PASS>(P, a, t.x0, t.y0, t.yend, parity ? -t.dir : t.dir, blockIdx.x);
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Longest wait of a tile for its neighbours, in SM clock cycles (about 2 s):
// a correct launch never comes near it (neighbours are at most one step
// apart and all CTAs are resident: cooperative launch).
constexpr long long PERSIST_WAIT_CYCLES = 4000000000LL;

// Several time steps of a batch in one cooperative launch, one CTA per tile
// for the whole launch (every tile resident at once).  After step k a tile
// publishes flags[tile] = k + 1 (release); before step k + 1 it waits until
// every tile whose region its stencil reaches (nbr: count, then indices) has
// published k + 1 (acquire).  Neighbours are then at most one step apart, so
// a tile never reads a buffer a neighbour is still writing or writes one a
// neighbour is still reading, and no grid-wide barrier is needed.  Populations
// other tiles write in this launch are read through L2 (no read-only path).
// The FP32 shift of the source buffer is the stored one at step 0 and the
// target after it (what step 0 wrote with); the caller records the final
// buffer's shift.  A wait that runs past PERSIST_WAIT_CYCLES sets *err,
// fills the tile's rest population (both buffers) and S with NaN (so the
// diagnostics report non-finite fields) and ends the CTA; tiles waiting on
// it see *err and end too.
template <typename T, int TX>
__global__ void __launch_bounds__(TX *TYB, (Occ<T, PASS_STATE, TX>::ctas))
    d2q9_batch_persist_kernel(const BatchCase *__restrict__ cases, const BatchTile *__restrict__ tiles,
                              const int *__restrict__ nbr, int parity0, int nsteps, int *flags,
                              int *err)
{
    const BatchTile t = tiles[blockIdx.x];
    const BatchCase &c = cases[t.c];
    const StepParams<T> P = *reinterpret_cast<const StepParams<T> *>(
        sizeof(T) == 4 ? (const void *)&c.pf : (const void *)&c.pd);
    const int lin = threadIdx.y * TX + threadIdx.x;
    const int *nb = nbr + (size_t)blockIdx.x * (PERSIST_NBMAX + 1);
    __shared__ int s_abort;
    for (int k = 0; k < nsteps; ++k) {
        if (k > 0) {
            if (lin < 32) {
                bool bad = false;
                if (lin < nb[0]) {
                    const int *fl = flags + nb[1 + lin];
                    const long long t0 = clock64();
                    while (ld_acquire_gpu(fl) < k) {
                        if (clock64() - t0 > PERSIST_WAIT_CYCLES || ld_acquire_gpu(err) != 0) {
                            bad = true;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                bad = __any_sync(0xffffffffu, bad);
                if (lin == 0) {
                    if (bad) atomicExch(err, 1);
                    s_abort = bad ? 1 : 0;
                }
                __threadfence();  // the polling warp's acquires reach the CTA through the barrier
            }
            __syncthreads();
            if (s_abort) {
                // the tile's state is invalid: NaN in its rest population of
                // both buffers (so phi, whichever buffer is current) and in S
                T *S = static_cast<T *>(c.S);
                T *f0 = static_cast<T *>(c.f[0]), *f1 = static_cast<T *>(c.f[1]);
                const int x = t.x0 + threadIdx.x;
                if (x < P.nx)
                    for (int y = t.y0 + (int)threadIdx.y; y < t.yend; y += TYB) {
                        const size_t n = (size_t)y * P.nx + x;
                        S[n] = T(NAN);
                        f0[n] = T(NAN);
                        f1[n] = T(NAN);
                    }
                return;
            }
        }
        const int parity = parity0 ^ (k & 1);
        PassArgs a;
        a.f_src = c.f[parity];
        a.f_dst = c.f[parity ^ 1];
        a.g_src = c.g[parity];
        a.g_dst = c.g[parity ^ 1];
        a.S = c.S;
        a.S_out = c.S;
        a.out_phi = a.out_p = a.out_u = a.out_mu = nullptr;
        a.mt_phi = a.mt_p = a.mt_u = a.mt_mu = nullptr;
        a.partials = nullptr;
        a.eqs_src = k == 0 ? c.eqs + parity0 : c.eqs + 2;
        a.eqs_dst = nullptr;
        a.eqs_target = c.eqs + 2;
        a.flip = 0;
        d2q9_tile<T, TX, PASS_STATE, false>(P, a, t.x0, t.y0, t.yend, parity ? -t.dir : t.dir,
                                            blockIdx.x);
        __syncthreads();  // every output of the step is stored
        if (lin == 0) {
            __threadfence();
            st_release_gpu(flags + blockIdx.x, k + 1);
        }
    }
}

// the final buffer's FP32 shift after a multi-step launch: the target
__global__ void d2q9_batch_eqs_final(const BatchCase *__restrict__ cases, int ncases, int parity)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ncases) cases[i].eqs[parity] = cases[i].eqs[2];
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
        if (sizeof(T) == 4 && i == 0) f[9 * N + n] = (T)(fe - (double)(T)fe);  // low word
    }
    S[n] = T(0);
}

// paper convention <-> pull storage
template <typename T>
__global__ void d2q9_get_state_k(int nx, int ny, const T *__restrict__ f, const T *__restrict__ g,
                                 const T *__restrict__ S, const float *eqs, double *fo,
                                 double *go, double *So)
{
    const size_t N = (size_t)nx * ny;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = (int)(n % nx), y = (int)(n / nx);
    const double a = sizeof(T) == 4 ? (double)*eqs : 0.0;  // equilibrium shift
    for (int i = 0; i < 9; ++i) {
        const size_t m = (size_t)wrapi(y - cyv(i), ny) * nx + wrapi(x - cxv(i), nx);
        double fv = (double)f[i * N + m];
        if (sizeof(T) == 4 && i == 0) fv += (double)f[9 * N + m];  // rest population pair
        if (sizeof(T) == 4)
            fv += i == 0 ? -(5.0 / 9.0) * a : (i <= 4 ? (1.0 / 9.0) * a : (1.0 / 36.0) * a);
        if (fo) fo[i * N + n] = fv;
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
        const double v = fi[i * N + m];
        f[i * N + n] = (T)v;
        if (sizeof(T) == 4 && i == 0) f[9 * N + n] = (T)(v - (double)(T)v);
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
    case PASS_MACROS_T: return launch_pass<T, PASS_MACROS_T>(params, a, s, st);
    case PASS_STATE | PASS_MACROS_T:
        return launch_pass<T, PASS_STATE | PASS_MACROS_T>(params, a, s, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int TX>
cudaError_t launch_batch_t(const BatchCase *cases, const BatchTile *tiles, int ntiles, int parity,
                           cudaStream_t st)
{
    dim3 block(TX, TYB);
    d2q9_batch_kernel<T, TX, PASS_STATE><<<ntiles, block, 0, st>>>(cases, tiles, parity, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t d2q9_batch_step(int precision, int width, const BatchCase *cases,
                            const BatchTile *tiles, int ntiles, int parity, cudaStream_t st)
{
    if (precision == 0)
        return width == 64 ? launch_batch_t<double, 64>(cases, tiles, ntiles, parity, st)
                           : launch_batch_t<double, 128>(cases, tiles, ntiles, parity, st);
    return width == 64 ? launch_batch_t<float, 64>(cases, tiles, ntiles, parity, st)
                       : launch_batch_t<float, 128>(cases, tiles, ntiles, parity, st);
}

namespace {

template <typename T, int TX>
cudaError_t launch_persist_t(const BatchCase *cases, int ncases, const BatchTile *tiles,
                             const int *nbr, int ntiles, int parity, int nsteps, int *flags,
                             int *err, cudaStream_t st)
{
    // the tiles' counters and the spare one that nothing sets (fault-injection tests)
    cudaError_t e = cudaMemsetAsync(flags, 0, ((size_t)ntiles + 1) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&cases, (void *)&tiles, (void *)&nbr, (void *)&parity,
                    (void *)&nsteps, (void *)&flags, (void *)&err};
    e = cudaLaunchCooperativeKernel((const void *)d2q9_batch_persist_kernel<T, TX>, dim3(ntiles),
                                    dim3(TX, TYB), args, 0, st);
    if (e != cudaSuccess) return e;
    d2q9_batch_eqs_final<<<(ncases + 127) / 128, 128, 0, st>>>(cases, ncases,
                                                               parity ^ (nsteps & 1));
    return cudaGetLastError();
}

template <typename T, int TX>
int persist_ctas_per_sm_t()
{
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, d2q9_batch_persist_kernel<T, TX>, TX * TYB, 0);
    return e == cudaSuccess ? n : 0;
}

}  // namespace

cudaError_t d2q9_batch_persist(int precision, int width, const BatchCase *cases, int ncases,
                               const BatchTile *tiles, const int *nbr, int ntiles, int parity,
                               int nsteps, int *flags, int *err, cudaStream_t st)
{
    if (precision == 0)
        return width == 64 ? launch_persist_t<double, 64>(cases, ncases, tiles, nbr, ntiles,
                                                          parity, nsteps, flags, err, st)
                           : launch_persist_t<double, 128>(cases, ncases, tiles, nbr, ntiles,
                                                           parity, nsteps, flags, err, st);
    return width == 64 ? launch_persist_t<float, 64>(cases, ncases, tiles, nbr, ntiles, parity,
                                                     nsteps, flags, err, st)
                       : launch_persist_t<float, 128>(cases, ncases, tiles, nbr, ntiles, parity,
                                                      nsteps, flags, err, st);
}

int d2q9_batch_persist_ctas_per_sm(int precision, int width)
{
    if (precision == 0)
        return width == 64 ? persist_ctas_per_sm_t<double, 64>() : persist_ctas_per_sm_t<double, 128>();
    return width == 64 ? persist_ctas_per_sm_t<float, 64>() : persist_ctas_per_sm_t<float, 128>();
}

LaunchShape d2q9_shape(int nx, int ny, int num_sms)
{
    LaunchShape s;
    s.variant = TXW;
    s.grid_x = (nx + TXW - 1) / TXW;
    // one wave of resident CTAs (4 per SM at the FP32 register budget) when
    // the grid allows it; rows even (two rows per iteration).  Small grids
    // get short marches (down to one iteration) so that more CTAs share the
    // latency of a step.
    const long long slots = 4LL * (num_sms > 0 ? num_sms : 152);
    long long rows = ((long long)s.grid_x * ny + slots - 1) / slots;
    if (rows < 2) rows = 2;
    if (rows > 256) rows = 256;
    rows += rows & 1;
    s.rows = (int)rows;
    s.grid_y = (int)((ny + rows - 1) / rows);
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
                           const void *S, const float *eqs, double *fo, double *go, double *So,
                           cudaStream_t st)
{
    const size_t N = (size_t)nx * ny;
    const int tb = 256;
    const unsigned nb = (unsigned)((N + tb - 1) / tb);
    if (precision == 0)
        d2q9_get_state_k<double><<<nb, tb, 0, st>>>(nx, ny, (const double *)f, (const double *)g,
                                                    (const double *)S, eqs, fo, go, So);
    else
        d2q9_get_state_k<float><<<nb, tb, 0, st>>>(nx, ny, (const float *)f, (const float *)g,
                                                   (const float *)S, eqs, fo, go, So);
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
