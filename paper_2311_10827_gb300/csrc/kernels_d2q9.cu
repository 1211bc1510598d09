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

// The paired FP32 datapath (add/mul/fma.rn.f32x2): two independent lanes per
// instruction, each rounding exactly as the scalar instruction would.  The
// FP32 node update puts independent pairs of its arithmetic on it.
__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 x, float2 y) { return __fadd2_rn(x, y); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y)
{
    return __fadd2_rn(x, make_float2(-y.x, -y.y));
}
__device__ __forceinline__ float2 mul2(float2 x, float2 y) { return __fmul2_rn(x, y); }
__device__ __forceinline__ float2 fma2(float2 x, float2 y, float2 z) { return __ffma2_rn(x, y, z); }

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

template <typename T>
__device__ __forceinline__ void warp_reduce(double &sum0, double &sum1, T &mx, T &mn, T &mxu,
                                            double &sum2, T &bad)
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

// Resident CTAs per SM targeted by the register budget: every FP32 variant
// fits 64 registers (1024 threads per SM; the diagnostics accumulate in
// shared memory); FP64 512 threads.
template <typename T, int PASS, int TX>
struct Occ {
    static constexpr int nth = TX * TYB;
    static constexpr int threads = sizeof(T) == 4 ? 1024 : 512;
    static constexpr int ctas = threads / nth > 0 ? threads / nth : 1;
};

// Shared memory of one tile march: the phi and mu rings, the FP32 staging
// of the f pulls (two stages: the next iteration's phi row is copied in
// while this iteration runs) and the diagnostics' per-warp partials.  One
// instance per kernel, whichever tile variants the kernel runs.
template <typename T, int TX>
struct TileSmem {
    static constexpr int R = 2 * TYB + 3;  // ring depth: writes never hit a row still read
    static constexpr int WP = TX + 4;      // phi ring width (halo 2)
    static constexpr int WM = TX + 2;      // mu ring width (halo 1)
    static constexpr bool STAGE = sizeof(T) == 4;
    static constexpr int NS = 2;  // staging depth (FP32)
    static constexpr int NT = TX * TYB, NFS = sizeof(T) == 4 ? 10 : 9;
    T phs[R * WP];
    T mus[R * WM];
    T fst[STAGE ? NS * NFS * NT : 1];
    T fsh[STAGE ? NS * NFS * 4 * TYB : 1];
    double red[7][NT / 32];
    // Per-thread diagnostics accumulators, kept here rather than in
    // registers so that a diagnostics step needs no more registers than a
    // plain one: the sums of phi, rho |u|^2 / 2, S and S_prev (FP64 for FP64
    // storage; for FP32 each as an exact FP32 (hi, lo) pair, so that the FP32
    // step does no FP64 arithmetic per node), the extrema of |u|^2 and mu,
    // and the tile's non-finite flag.
    static constexpr int NACC = sizeof(T) == 4 ? 8 : 4;
    T acc[NACC][NT];
    T ext[3][NT];
    int bad;
};
static_assert(sizeof(TileSmem<float, 128>) <= 48 * 1024, "static shared memory of a CTA");
static_assert(sizeof(TileSmem<double, 128>) <= 48 * 1024, "static shared memory of a CTA");

// One tile: columns [x0, x0 + TX), rows [y0, yend), marching in direction
// dir (+1 down from y0, -1 up from yend - 1); diagnostics partial record
// `part` (PASS_DIAG).  Shared by the single-grid and the batched kernels.
template <typename T, int TX, int PASS, bool NC = true>
__device__ __forceinline__ void d2q9_tile(TileSmem<T, TX> &sm, const StepParams<T> &P,
                                          const PassArgs &a, int x0, int y0, int yend, int dir,
                                          int part)
{
    using SM = TileSmem<T, TX>;
    constexpr int R = SM::R, WP = SM::WP, WM = SM::WM;
    constexpr bool REST_PAIR = sizeof(T) == 4;
    // Staged pulls (asynchronous copies one iteration ahead) in per-step
    // launches only.  A multi-step launch reads populations that other CTAs
    // wrote in the same launch, and those reads must come from L2: the
    // asynchronous 4-byte copies allocate in L1 (cp.async.ca, the only form
    // at that size) and returned stale values there although each step's
    // reads follow the writers' release through an acquire, a fence and a
    // CTA barrier (measured: batches with more tiles than resident CTAs
    // drifted from per-step launches by 1e-12 to 1e-2).  So a multi-step
    // launch pulls with ld.global.cg into registers, one iteration ahead.
    constexpr bool STAGE = SM::STAGE && NC;
    constexpr int NT = SM::NT, NFS = SM::NFS;
    T *const phs = sm.phs;
    T *const mus = sm.mus;
    T *const fst = sm.fst;
    T *const fsh = sm.fsh;
    T(*const dacc)[NT] = sm.acc;
    T(*const facc)[NT] = sm.ext;
    int *const dbad = &sm.bad;
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

    // issue the copies of phi row `row`'s pulls into stage st
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
    // phi row from stage st (the copies have landed), keeping the own pulls
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

    // diagnostics: sums in FP64; the extrema of |u|^2 and mu and the
    // non-finite flag are exact in the storage type
    if (PASS & PASS_DIAG) {
#pragma unroll
        for (int q = 0; q < SM::NACC; ++q) dacc[q][lin] = T(0);
        facc[0][lin] = T(0);
        facc[1][lin] = T(INFINITY);
        facc[2][lin] = T(-INFINITY);
        if (lin == 0) *dbad = 0;  // read after the march's barriers
    }

    // prologue: phi rows y0-2 .. y0+1 (the own row y0+ty keeps its values),
    // mu rows y0-1 .. y0
    T fcur[9], fnext[9], locur = T(0), lonext = T(0);
    if (STAGE) {
        // every copy of the prologue in flight at once
        issue_phi_row(first + dir * (ty - 2), 1);
        issue_phi_row(first + dir * ty, 0);
        cp_commit();
        cp_wait_all();
        phi_row_staged(slot(first + dir * (ty - 2)), 1, fnext, lonext);
        phi_row_staged(slot(first + dir * ty), 0, fcur, locur);
        __syncthreads();  // stage 0 is read before it is refilled
        issue_phi_row(first + dir * (2 + ty), 0);
        cp_commit();
    } else {
        phi_row(first + dir * (ty - 2), slot(first + dir * (ty - 2)), fnext, lonext);
        phi_row(first + dir * ty, slot(first + dir * ty), fcur, locur);
        __syncthreads();
    }
    {
        const int r = first + dir * (ty - 1);
        mu_row(slot(r - 1), slot(r), slot(r + 1));
    }
    __syncthreads();

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
                Sprev = NC ? __ldcs(static_cast<const T *>(a.S) + (nrow + xo))
                           : __ldcg(static_cast<const T *>(a.S) + (nrow + xo));  // from L2
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
            T gpx, gpy, Fx, Fy, rho, inv_rho, itg, ux, uy, grx, gry, ugr, uu, S;
            // Eq. gradient: grad = 3 sum_{i!=0} w_i c_i Psi(x + c_i)
            //   = (1/3)(axis differences) + (1/12)(diagonal differences)
            if constexpr (sizeof(T) == 4) {
                // x and y components as the two lanes of paired instructions
                const float2 gp = fma2(
                    f2(1.0f / 3.0f), sub2(make_float2(p0[j + 1], pp[j]), make_float2(p0[j - 1], pm[j])),
                    mul2(f2(1.0f / 12.0f),
                         add2(sub2(make_float2(pp[j + 1], pp[j + 1]), make_float2(pp[j - 1], pm[j + 1])),
                              sub2(make_float2(pm[j + 1], pp[j - 1]), make_float2(pm[j - 1], pm[j - 1])))));
                const float2 gm = fma2(
                    f2(1.0f / 3.0f), sub2(make_float2(m0[k + 1], mp[k]), make_float2(m0[k - 1], mm[k])),
                    mul2(f2(1.0f / 12.0f),
                         add2(sub2(make_float2(mp[k + 1], mp[k + 1]), make_float2(mp[k - 1], mm[k + 1])),
                              sub2(make_float2(mm[k + 1], mp[k - 1]), make_float2(mm[k - 1], mm[k - 1])))));
                gpx = gp.x;
                gpy = gp.y;
                // F = -phi grad(mu) + G; rho, nu linear in phi (Eq. vis)
                const float2 F = fma2(f2(-phi), gm, make_float2(P.G[0], P.G[1]));
                Fx = F.x;
                Fy = F.y;
                const float2 rn = fma2(f2(phi - P.phiv), make_float2(P.drho, P.dnu),
                                       make_float2(P.rhov, P.nuv));
                rho = rn.x;
                inv_rho = Arith<T>::rcp(rho);
                itg = Arith<T>::rcp(fmaf(3.0f, rn.y, 0.5f));  // nu = cs2 (tau_g - 1/2)
                // rho u = sum_i c_i g_i + F/2
                const float jx = (gv[2] - gv[4]) + ((gv[5] - gv[6]) + (gv[8] - gv[7]));
                const float jy = (gv[3] - gv[1]) + ((gv[5] + gv[6]) - (gv[7] + gv[8]));
                const float2 u = mul2(fma2(f2(0.5f), F, make_float2(jx, jy)), f2(inv_rho));
                ux = u.x;
                uy = u.y;
                const float2 gr = mul2(f2(P.drho), gp);  // grad rho (chain rule)
                grx = gr.x;
                gry = gr.y;
                // u.grad(rho) and S = u.grad(phi) as the two lanes
                const float2 us = fma2(f2(ux), make_float2(grx, gpx), mul2(f2(uy), make_float2(gry, gpy)));
                ugr = us.x;
                S = us.y;
                uu = fmaf(ux, ux, uy * uy);
            } else {
                gpx = T(1.0 / 3.0) * (p0[j + 1] - p0[j - 1]) +
                      T(1.0 / 12.0) * ((pp[j + 1] - pp[j - 1]) + (pm[j + 1] - pm[j - 1]));
                gpy = T(1.0 / 3.0) * (pp[j] - pm[j]) +
                      T(1.0 / 12.0) * ((pp[j + 1] - pm[j + 1]) + (pp[j - 1] - pm[j - 1]));
                const T gmx = T(1.0 / 3.0) * (m0[k + 1] - m0[k - 1]) +
                              T(1.0 / 12.0) * ((mp[k + 1] - mp[k - 1]) + (mm[k + 1] - mm[k - 1]));
                const T gmy = T(1.0 / 3.0) * (mp[k] - mm[k]) +
                              T(1.0 / 12.0) * ((mp[k + 1] - mm[k + 1]) + (mp[k - 1] - mm[k - 1]));
                // F = -phi grad(mu) + G; rho, nu linear in phi (Eq. vis)
                Fx = -phi * gmx + P.G[0];
                Fy = -phi * gmy + P.G[1];
                const T dphi = phi - P.phiv;
                rho = P.rhov + dphi * P.drho;
                const T nu = P.nuv + dphi * P.dnu;
                inv_rho = Arith<T>::rcp(rho);
                itg = Arith<T>::rcp(T(0.5) + T(3) * nu);  // nu = cs2 (tau_g - 1/2)
                // rho u = sum_i c_i g_i + F/2
                const T jx = (gv[2] - gv[4]) + ((gv[5] - gv[6]) + (gv[8] - gv[7]));
                const T jy = (gv[3] - gv[1]) + ((gv[5] + gv[6]) - (gv[7] + gv[8]));
                ux = (jx + T(0.5) * Fx) * inv_rho;
                uy = (jy + T(0.5) * Fy) * inv_rho;
                grx = P.drho * gpx;  // grad rho (chain rule)
                gry = P.drho * gpy;
                ugr = ux * grx + uy * gry;
                uu = ux * ux + uy * uy;
                S = ux * gpx + uy * gpy;  // u.grad(phi)
            }
            // p = cs2/(1-w0) [sum_{i!=0} g_i + u.grad(rho)/2 + rho s_0(u)],
            // rho s_0 = -(2/3) rho |u|^2 for D2Q9
            const T p = T(0.6) * (sum_moving(gv) + T(0.5) * ugr - T(2.0 / 3.0) * rho * uu);

            if (PASS & PASS_DIAG) {
                if constexpr (sizeof(T) == 4) {
                    // (hi, lo) += x with an exact two-sum on the high word
                    auto acc2 = [&](int q, float x) {
                        const float hi = dacc[q][lin];
                        const float s = hi + x, bp = s - hi;
                        dacc[q + 1][lin] += (hi - (s - bp)) + (x - bp);
                        dacc[q][lin] = s;
                    };
                    acc2(0, phi);
                    acc2(2, 0.5f * rho * uu);
                    acc2(4, S);
                    acc2(6, Sprev);
                } else {
                    dacc[0][lin] += phi;
                    dacc[1][lin] += 0.5 * rho * uu;
                    dacc[2][lin] += S;
                    dacc[3][lin] += Sprev;
                }
                facc[0][lin] = fmax(facc[0][lin], uu);
                facc[1][lin] = fmin(facc[1][lin], mu);
                facc[2][lin] = fmax(facc[2][lin], mu);
                if (!isfinite(phi) || !isfinite(p) || !isfinite(uu) || !isfinite(mu)) *dbad = 1;
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
                if constexpr (sizeof(T) == 4) {
                    // two populations per paired instruction: f 1..4 and 5..8 in
                    // pairs; g the two axis and the two diagonal direction pairs
                    const float2 it2 = f2(itf);
#pragma unroll
                    for (int i = 1; i <= 7; i += 2) {
                        const float2 v = make_float2(fcur[i], fcur[i + 1]);
                        const float2 o = add2(v, fma2(sub2(f2(i < 5 ? ea : ed), v), it2,
                                                      f2(i < 5 ? sa : sd)));
                        st_stream(fd + (i * N + n), o.x);
                        st_stream(fd + ((i + 1) * N + n), o.y);
                    }
                    const float2 itg2 = f2(itg), A2 = f2(A), r45 = f2(4.5f * rho);
#pragma unroll
                    for (int grp = 0; grp < 2; ++grp) {
                        // lanes: directions (2, 3) / (4, 1) on the axes, (5, 6) / (7, 8) on the diagonals
                        const float w = grp == 0 ? 1.0f / 9.0f : 1.0f / 36.0f;
                        const float2 cu = grp == 0 ? make_float2(ux, uy) : make_float2(ux + uy, uy - ux);
                        const float2 cF = grp == 0 ? make_float2(Fx, Fy) : make_float2(Fx + Fy, Fy - Fx);
                        const float2 cg = grp == 0 ? make_float2(grx, gry)
                                                   : make_float2(grx + gry, gry - grx);
                        const int p0i = grp == 0 ? 2 : 5, p1i = grp == 0 ? 3 : 6;
                        const int m0i = grp == 0 ? 4 : 7, m1i = grp == 0 ? 1 : 8;
                        const float2 eq_s = mul2(f2(w), fma2(mul2(r45, cu), cu, A2));
                        const float2 eq_a = mul2(f2(3.0f * w * rho), cu);
                        const float2 wk = f2(3.0f * w * kg);
                        const float2 G_s = mul2(mul2(wk, cu), cg), G_a = mul2(wk, cF);
                        const float2 gp = make_float2(gv[p0i], gv[p1i]);
                        const float2 gm = make_float2(gv[m0i], gv[m1i]);
                        const float2 op = add2(gp, fma2(sub2(add2(eq_s, eq_a), gp), itg2, add2(G_s, G_a)));
                        const float2 om = add2(gm, fma2(sub2(sub2(eq_s, eq_a), gm), itg2, sub2(G_s, G_a)));
                        st_stream(gd + (p0i * N + n), op.x);
                        st_stream(gd + (p1i * N + n), op.y);
                        st_stream(gd + (m0i * N + n), om.x);
                        st_stream(gd + (m1i * N + n), om.y);
                    }
                } else {
#pragma unroll
                    for (int i = 1; i <= 4; ++i)
                        st_stream(fd + (i * N + n), fcur[i] + ((ea - fcur[i]) * itf + sa));
#pragma unroll
                    for (int i = 5; i <= 8; ++i)
                        st_stream(fd + (i * N + n), fcur[i] + ((ed - fcur[i]) * itf + sd));
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
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) fcur[i] = fnext[i];
        locur = lonext;
    }
    if (!NC) cp_wait_all();  // the next step of a multi-step launch reuses the stages

    if (PASS & PASS_DIAG) {
        __syncthreads();  // every flag write of the march is done
        double d_phi, d_E, d_bud;
        if constexpr (sizeof(T) == 4) {
            d_phi = (double)dacc[0][lin] + (double)dacc[1][lin];
            d_E = (double)dacc[2][lin] + (double)dacc[3][lin];
            d_bud = 1.5 * ((double)dacc[4][lin] + (double)dacc[5][lin]) -
                    0.5 * ((double)dacc[6][lin] + (double)dacc[7][lin]);
        } else {
            d_phi = dacc[0][lin];
            d_E = dacc[1][lin];
            d_bud = 1.5 * dacc[2][lin] - 0.5 * dacc[3][lin];
        }
        T d_u2 = facc[0][lin], d_mumin = facc[1][lin], d_mumax = facc[2][lin],
          d_bad = *dbad ? T(1) : T(0);
        warp_reduce(d_phi, d_E, d_u2, d_mumin, d_mumax, d_bud, d_bad);
        constexpr int NW = TX * TYB / 32;
        double(*red)[NW] = sm.red;
        const int lane = (ty * TX + tx) & 31, wid = (ty * TX + tx) >> 5;
        if (lane == 0) {
            red[0][wid] = d_phi;
            red[1][wid] = d_E;
            red[2][wid] = (double)d_u2;
            red[3][wid] = (double)d_mumin;
            red[4][wid] = (double)d_mumax;
            red[5][wid] = d_bud;
            red[6][wid] = (double)d_bad;
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
__global__ void __launch_bounds__((Occ<T, PASS, TX>::nth), (Occ<T, PASS, TX>::ctas))
    d2q9_pass_kernel(const StepParams<T> P, PassArgs a, int rows)
{
    const int y0 = blockIdx.y * rows;
    // march direction: alternating between neighbouring row tiles, and
    // reversed on every other step
    const int dir = ((blockIdx.y & 1) ? -1 : 1) * (a.flip ? -1 : 1);
    __shared__ TileSmem<T, TX> sm;
    d2q9_tile<T, TX, PASS>(sm, P, a, blockIdx.x * TX, y0, min(y0 + rows, P.ny), dir,
                           blockIdx.y * gridDim.x + blockIdx.x);
}

// Batched: CTA k runs tile k of a flat tile table over many independent grids
// (each with its own size and parameters); buffers are picked by the step
// parity shared by all cases.  S is read from S and written to S_out.
template <typename T, int TX, int PASS>
__global__ void __launch_bounds__((Occ<T, PASS, TX>::nth), (Occ<T, PASS, TX>::ctas))
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
    __shared__ TileSmem<T, TX> sm;
    d2q9_tile<T, TX, PASS>(sm, P, a, t.x0, t.y0, t.yend, parity ? -t.dir : t.dir, blockIdx.x);
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Longest wait of a tile for its neighbours, in SM clock cycles (about 2 s):
// a correct launch never comes near it (every CTA is resident: cooperative
// launch, and the oldest unfinished step of any tile can always proceed).
constexpr long long PERSIST_WAIT_CYCLES = 4000000000LL;

// Per-grid reduction of the tiles' FP64 diagnostics partials (a fixed order,
// so the same partials always give the same record), one thread per grid.
// shift_slot >= 0 (FP32 storage): the grid's next equilibrium-shift target,
// alpha times the middle of the mu range (kept if the record is not finite or
// re-centring is off), is written to eqs[shift_slot].
__device__ void reduce_cases(const DiagPartial *part, const int *tile0, const BatchCase *cases,
                             int ncases, DiagPartial *records, int shift_slot, int tid, int nthr)
{
    for (int c = tid; c < ncases; c += nthr) {
        double s0 = 0.0, s1 = 0.0, mx = 0.0, mn = DBL_MAX, mxm = -DBL_MAX, s2 = 0.0, bad = 0.0;
        for (int k = tile0[c]; k < tile0[c + 1]; ++k) {
            const DiagPartial *p = part + k;  // written by other CTAs: read from L2
            s0 += __ldcg(&p->sum_phi);
            s1 += __ldcg(&p->E);
            mx = fmax(mx, __ldcg(&p->u2max));
            mn = fmin(mn, __ldcg(&p->mu_min));
            mxm = fmax(mxm, __ldcg(&p->mu_max));
            s2 += __ldcg(&p->budget);
            bad = fmax(bad, __ldcg(&p->nonfinite));
        }
        DiagPartial r;
        r.sum_phi = s0;
        r.E = s1;
        r.u2max = mx;
        r.mu_min = mn;
        r.mu_max = mxm;
        r.budget = s2;
        r.nonfinite = bad;
        r.pad = 0.0;
        records[c] = r;
        if (shift_slot >= 0) {
            float *e = cases[c].eqs;
            float tgt = e[2];
            const double a = cases[c].pd.alpha * 0.5 * (mn + mxm);
            if (cases[c].recentre && bad == 0.0 && isfinite(a)) tgt = (float)a;
            e[shift_slot] = tgt;
        }
    }
}

// Per-step launches: records of the step that carried the diagnostics; the
// FP32 target moves at once (the next launch writes with it).
__global__ void d2q9_batch_reduce_kernel(const DiagPartial *__restrict__ part,
                                         const int *__restrict__ tile0, const BatchCase *cases,
                                         int ncases, DiagPartial *records, int shift_slot)
{
    reduce_cases(part, tile0, cases, ncases, records, shift_slot, threadIdx.x, blockDim.x);
}

// Several time steps of a batch in one cooperative launch.  The work is a
// queue of (step, tile) pairs taken in order, step-major, from a ticket
// counter: a CTA takes the next pair, waits until the tile itself and every
// tile whose region its stencil reaches (nbr: count, then indices) have
// completed the previous step (flags[tile] = steps completed, acquire), runs
// the tile, and publishes flags[tile] = step + 1 (release).  Neighbours are
// then at most one step apart, so a tile never reads a buffer a neighbour is
// still writing or writes one a neighbour is still reading; there is no
// grid-wide barrier, any number of tiles runs with any number of resident
// CTAs, and tiles of the next step start while the last ones of a step are
// still running.  Progress: the pair with the lowest ticket still unfinished
// only waits on pairs with lower tickets, all finished.
//
// Memory ordering of the pulls.  Every population, S and phi value that
// other tiles write during the launch is read with ld.global.cg (L2 only):
// the tile routine runs without its L1-allocating asynchronous staging here
// (NC false).  The writer CTA stores, passes bar.sync, and its thread 0
// fences and does st.release.gpu on the tile's counter; a polling lane of
// the reader does ld.acquire.gpu, observes the count, fences, and the CTA
// passes bar.sync before any read of the next step.  With the asynchronous
// 4-byte copies (cp.async.ca, which allocate in L1) some reads returned
// values older than that chain allows (batches with more tiles than
// resident CTAs drifted from per-step launches), so no read of this
// launch's data goes through L1.
//
// FP32 equilibrium shift: the source buffer's shift is the stored one at
// step 0 and the target after it (what step 0 wrote with); the target is
// constant during the launch.  With diagnostics (step diag_k), the last tile
// to finish that step reduces every grid's partials into records and writes
// the next target to eqs[3]; the last tile to finish the final step (every
// pair is then done) records the final buffer's shift and moves eqs[3] into
// the target.  Those are the launch's only shared counters: one atomic per
// tile per launch, not per step.
//
// A wait that runs past PERSIST_WAIT_CYCLES sets *err (and *err_host),
// fills the tile's rest population (both buffers) and S with NaN (so the
// diagnostics report non-finite fields) and ends the CTA; CTAs waiting on it
// or taking a new pair see *err and end too.
template <typename T, int TX>
__global__ void __launch_bounds__((Occ<T, PASS_STATE, TX>::nth), (Occ<T, PASS_STATE, TX>::ctas))
    d2q9_batch_persist_kernel(const PersistArgs pa)
{
    constexpr int NTH = Occ<T, PASS_STATE, TX>::nth;
    const int lin = threadIdx.y * blockDim.x + threadIdx.x;
    const int total = pa.nsteps * pa.ntiles;  // < 2^31 (checked on the host)
    // One CTA per tile when they all fit (CTA b runs tile b at every step);
    // else the queue: the first pair is the CTA's index, later ones come from
    // the ticket counter, each taken one tile ahead so that its atomic's
    // latency hides behind the tile's work.
    const bool fixed = pa.ntiles <= (int)gridDim.x;
    if (fixed && (int)blockIdx.x >= pa.ntiles) return;
    __shared__ int s_next, s_abort, s_diag, s_stop;
    __shared__ TileSmem<T, TX> sm;
    int tk = blockIdx.x;
    while (tk < total) {
        const int k = tk / pa.ntiles, ti = tk - k * pa.ntiles;
        // the next pair (queue) and the error word are fetched now and used
        // after the tile, so that neither round trip delays it
        int err_seen = 0;
        if (lin == 0) {
            if (!fixed) s_next = atomicAdd(pa.ctr, 1) + (int)gridDim.x;
            err_seen = ld_relaxed_gpu(pa.err);
        }
        const BatchTile t = pa.tiles[ti];
        const BatchCase &c = pa.cases[t.c];
        const StepParams<T> P = *reinterpret_cast<const StepParams<T> *>(
            sizeof(T) == 4 ? (const void *)&c.pf : (const void *)&c.pd);
        if (k > 0) {
            if (lin < 32) {
                const int *nb = pa.nbr + (size_t)ti * (PERSIST_NBMAX + 1);
                bool bad = false;
                if (lin <= nb[0]) {  // lane 0: the tile itself; lanes 1..: its neighbours
                    const int *fl = pa.flags + (lin == 0 ? ti : nb[lin]);
                    const long long t0 = clock64();
                    while (ld_acquire_gpu(fl) < k) {
                        if (clock64() - t0 > PERSIST_WAIT_CYCLES || ld_acquire_gpu(pa.err) != 0) {
                            bad = true;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                bad = __any_sync(0xffffffffu, bad);
                if (lin == 0) {
                    if (bad) {
                        atomicExch(pa.err, 1);
                        if (pa.err_host) {
                            *(volatile int *)pa.err_host = 1;
                            __threadfence_system();
                        }
                    }
                    s_abort = bad ? 1 : 0;
                }
                __threadfence();  // the polling lanes' acquires reach the CTA through the barrier
            }
            __syncthreads();
            if (s_abort) {
                // the tile's state is invalid: NaN in its rest population of
                // both buffers (so phi, whichever buffer is current) and in S
                T *S = static_cast<T *>(c.S);
                T *f0 = static_cast<T *>(c.f[0]), *f1 = static_cast<T *>(c.f[1]);
                for (int x = t.x0 + threadIdx.x; x < t.x0 + TX && x < P.nx; x += blockDim.x)
                    for (int y = t.y0 + (int)threadIdx.y; y < t.yend; y += TYB) {
                        const size_t n = (size_t)y * P.nx + x;
                        S[n] = T(NAN);
                        f0[n] = T(NAN);
                        f1[n] = T(NAN);
                    }
                return;
            }
        }
        const int parity = pa.parity0 ^ (k & 1);
        PassArgs a;
        a.f_src = c.f[parity];
        a.f_dst = c.f[parity ^ 1];
        a.g_src = c.g[parity];
        a.g_dst = c.g[parity ^ 1];
        a.S = c.S;
        a.S_out = c.S;
        a.out_phi = a.out_p = a.out_u = a.out_mu = nullptr;
        a.mt_phi = a.mt_p = a.mt_u = a.mt_mu = nullptr;
        a.partials = pa.partials;
        a.eqs_src = k == 0 ? c.eqs + pa.parity0 : c.eqs + 2;
        a.eqs_dst = nullptr;
        a.eqs_target = c.eqs + 2;
        a.flip = 0;
        const int dir = parity ? -t.dir : t.dir;
        if (k == pa.diag_k)
            d2q9_tile<T, TX, PASS_STATE | PASS_DIAG, false>(sm, P, a, t.x0, t.y0, t.yend, dir, ti);
        else
            d2q9_tile<T, TX, PASS_STATE, false>(sm, P, a, t.x0, t.y0, t.yend, dir, ti);
        __syncthreads();  // every output of the step (and its partial) is stored
        // counters of the launch's last steps (one atomic per tile each):
        // the last tile of the diagnostics step reduces the partials; the
        // last tile of the final step (then every pair is done) records the
        // final shift, after the reduction (ctr[3] = 1 once it is written)
        if (lin == 0) {
            __threadfence();
            st_release_gpu(pa.flags + ti, k + 1);
            int fl = 0;
            if (k == pa.diag_k && atomicAdd(pa.ctr + 1, 1) == pa.ntiles - 1) fl |= 1;
            if (k == pa.nsteps - 1 && atomicAdd(pa.ctr + 2, 1) == pa.ntiles - 1) fl |= 2;
            s_diag = fl;
            s_stop = err_seen;
        }
        __syncthreads();
        const int next = fixed ? tk + pa.ntiles : s_next;  // read before the next barrier
        const int fl = s_diag, stop = s_stop;
        if (fl & 1) {  // every partial of the diagnostics step is written
            __threadfence();
            reduce_cases(pa.partials, pa.tile0, pa.cases, pa.ncases, pa.records,
                         sizeof(T) == 4 ? 3 : -1, lin, NTH);
            __syncthreads();
            if (lin == 0) {
                __threadfence();
                st_release_gpu(pa.ctr + 3, 1);
            }
        }
        if (fl & 2) {  // every pair is done; wait for the reduction if there is one
            if (lin == 0 && pa.diag_k >= 0) {
                const long long t0 = clock64();
                while (ld_acquire_gpu(pa.ctr + 3) == 0 && clock64() - t0 < PERSIST_WAIT_CYCLES)
                    __nanosleep(64);
            }
            __syncthreads();
            __threadfence();
            const int pend = pa.parity0 ^ (pa.nsteps & 1);  // buffer holding the final state
            for (int ci = lin; ci < pa.ncases; ci += NTH) {
                float *e = pa.cases[ci].eqs;
                e[pend] = e[2];
                if (pa.diag_k >= 0 && sizeof(T) == 4) e[2] = e[3];
            }
        }
        if (stop) break;  // another tile timed out: stop taking pairs
        tk = next;
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
                           DiagPartial *partials, cudaStream_t st)
{
    dim3 block(TX, TYB);
    if (partials)
        d2q9_batch_kernel<T, TX, PASS_STATE | PASS_DIAG>
            <<<ntiles, block, 0, st>>>(cases, tiles, parity, partials);
    else
        d2q9_batch_kernel<T, TX, PASS_STATE><<<ntiles, block, 0, st>>>(cases, tiles, parity, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t d2q9_batch_step(int precision, int width, const BatchCase *cases,
                            const BatchTile *tiles, int ntiles, int parity, DiagPartial *partials,
                            cudaStream_t st)
{
    if (precision == 0)
        return width == 64 ? launch_batch_t<double, 64>(cases, tiles, ntiles, parity, partials, st)
                           : launch_batch_t<double, 128>(cases, tiles, ntiles, parity, partials, st);
    return width == 64 ? launch_batch_t<float, 64>(cases, tiles, ntiles, parity, partials, st)
                       : launch_batch_t<float, 128>(cases, tiles, ntiles, parity, partials, st);
}

cudaError_t d2q9_batch_reduce(int precision, const DiagPartial *partials, const int *tile0,
                              const BatchCase *cases, int ncases, DiagPartial *records,
                              cudaStream_t st)
{
    d2q9_batch_reduce_kernel<<<1, 256, 0, st>>>(partials, tile0, cases, ncases, records,
                                                 precision == 0 ? -1 : 2);
    return cudaGetLastError();
}

namespace {

template <typename T, int TX>
cudaError_t launch_persist_t(const PersistArgs &pa, int nctas, cudaStream_t st)
{
    // counters (ticket, diagnostics tiles done, final-step tiles done, the
    // reduction's flag), then the tiles' step counters and the spare one
    // that nothing sets (fault-injection tests)
    cudaError_t e = cudaMemsetAsync(pa.ctr, 0, (4 + (size_t)pa.ntiles + 1) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&pa};
    e = cudaLaunchCooperativeKernel((const void *)d2q9_batch_persist_kernel<T, TX>, dim3(nctas),
                                    dim3(TX, TYB), args, 0, st);
    return e;
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

cudaError_t d2q9_batch_persist(int precision, int width, const PersistArgs &pa, int nctas,
                               cudaStream_t st)
{
    if (pa.flags != pa.ctr + 4) return cudaErrorInvalidValue;
    if (precision == 0)
        return width == 64 ? launch_persist_t<double, 64>(pa, nctas, st)
                           : launch_persist_t<double, 128>(pa, nctas, st);
    return width == 64 ? launch_persist_t<float, 64>(pa, nctas, st)
                       : launch_persist_t<float, 128>(pa, nctas, st);
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
