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
// The pulls are loaded by each thread into registers, or (the FP32
// multi-step kernel) staged in shared memory one iteration ahead by bulk
// asynchronous copies of whole row segments.
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

// Bulk asynchronous copies global -> shared (the copy engine; 16-byte
// aligned addresses, sizes a multiple of 16 bytes) completing on an
// mbarrier: the barrier's phase completes once its one expected arrival
// has come and every byte it was told to expect has landed.
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(float *dst, const float *src, unsigned bytes,
                                         unsigned long long *b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}
// Orders this thread's earlier view of global memory (what it acquired from
// other CTAs' ordinary stores) before its later copy-engine reads.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Longest wait for a stage's bulk copies, in SM clock cycles (about 1 s).
constexpr long long STAGE_WAIT_CYCLES = 2000000000LL;

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
// shared memory), with small register spills in the multi-step kernels
// (measured: removing them did not change the step time); FP64 512 threads.
template <typename T, int PASS, int TX>
struct Occ {
    static constexpr int nth = TX * TYB;
    static constexpr int threads = sizeof(T) == 4 ? 1024 : 512;
    static constexpr int ctas = threads / nth > 0 ? threads / nth : 1;
};

// Shared memory of one tile march outside the staging: the phi and mu rings
// and the diagnostics' per-warp partials.  One instance per kernel,
// whichever tile variants the kernel runs.
template <typename T, int TX>
struct TileSmem {
    static constexpr int R = 2 * TYB + 3;  // ring depth: writes never hit a row still read
    static constexpr int WP = TX + 4;      // phi ring width (halo 2)
    static constexpr int WM = TX + 2;      // mu ring width (halo 1)
    static constexpr int NT = TX * TYB;
    T phs[R * WP];
    T mus[R * WM];
    double red[7][NT / 32];
    unsigned long long bar[2];  // the stages' mbarriers (bulk-copy staging)
    int bad;
    int stage_timeout;          // a stage's wait gave up (set, never cleared here)
};

// Row-segment staging of the pulls (FP32, rows of a multiple of 4 nodes).
// Per iteration a stage holds, for each of the TYB thread rows, the ten f
// segments (populations 0..8 and the rest population's low word) of the phi
// row two rows ahead, the nine g segments and the S segment of the row being
// updated.  An f or g segment is the source row of its population (the row
// shifted by -c_y) over columns x0 - 4 .. x0 + TX + 3, so that a thread's pull
// from x - c_x is element tx + 4 - c_x; the S segment spans x0 .. x0 + TX - 1.
// Each segment is one bulk asynchronous copy (two where it wraps the
// periodic seam), which the copy engine reads from L2, completing on the
// stage's mbarrier.  Two stages: the copies for the next iteration fly
// while this one computes.
template <int TX>
struct SegLayout {
    static constexpr int W = TX + 8;                      // elements per f / g segment
    static constexpr int NF = 10, NG = 9;                 // segments per thread row
    static constexpr int GOFF = TYB * NF * W;             // g segments of a stage
    static constexpr int SOFF = GOFF + TYB * NG * W;      // S segments of a stage
    static constexpr int STAGE = SOFF + TYB * TX;         // floats per stage
    static constexpr int NSEG = TYB * (NF + NG + 1);      // segments per stage
    static constexpr int LPS = TX / 4;                    // lanes per segment (one main chunk each)
    static constexpr int SPW = 32 / LPS;                  // segments per warp pass
    static_assert(TX % 4 == 0 && 32 % LPS == 0 && NSEG % SPW == 0, "segment split");
    // A diagnostics step lays the same memory out as one f buffer (refilled
    // once the phi rows are read), two g buffers and then the per-thread
    // accumulators; S is loaded into registers.
    static constexpr int DG = TYB * NF * W;               // g buffer 0
    static constexpr int DACC = DG + 2 * TYB * NG * W;    // accumulators
    static_assert(DACC + 11 * TX * TYB <= 2 * STAGE, "diagnostics layout");
};

// Per-thread diagnostics accumulators, in the kernel's dynamic shared memory
// (at its start on the register path, after the buffers of the staged
// diagnostics layout): the sums of phi,
// rho |u|^2 / 2, S and S_prev (FP64 for FP64 storage; for FP32 each as an
// exact FP32 (hi, lo) pair, so that the FP32 step does no FP64 arithmetic per
// node), then the extrema of |u|^2 and mu.
template <typename T>
struct DiagAcc {
    static constexpr int NACC = sizeof(T) == 4 ? 8 : 4;
};

// Dynamic shared memory of a kernel running tiles of width TX: the
// diagnostics accumulators and, in a kernel that stages (SEGK, FP32), the
// two stages, whichever is larger.  Only the multi-step kernel stages: the
// stages take most of the unified L1 / shared memory, which the register
// path needs as L1 for its loads in flight.
template <typename T, int TX, bool SEGK = false>
constexpr int tile_dyn_bytes()
{
    constexpr int diag = (DiagAcc<T>::NACC + 3) * TX * TYB * (int)sizeof(T);
    constexpr int seg = SEGK && sizeof(T) == 4 ? 2 * SegLayout<TX>::STAGE * 4 : 0;
    return diag > seg ? diag : seg;
}
static_assert(sizeof(TileSmem<float, 128>) + tile_dyn_bytes<float, 128, true>() + 1024 <=
                  228 * 1024 / 4,
              "four staging FP32 CTAs of width 128 per SM");

// The packed c_y of populations 0..9 (9: the rest population's low word),
// 2 bits each as c_y + 1.
constexpr unsigned cy_packed()
{
    unsigned v = 0;
    for (int i = 0; i < 9; ++i) v |= (unsigned)(cyv(i) + 1) << (2 * i);
    return v | (1u << 18);
}

// Whether a grid's pulls can be staged by tiles of width TX: FP32 storage,
// rows of a multiple of 4 nodes and at least TX + 8 nodes (a segment then
// wraps the periodic seam at most once), 16-byte aligned buffers.
template <typename T, int TX>
__device__ __forceinline__ bool seg_ok(int nx, const void *f, const void *g, const void *S)
{
    return sizeof(T) == 4 && (nx & 3) == 0 && nx >= TX + 8 &&
           (((unsigned long long)f | (unsigned long long)g | (unsigned long long)S) & 15) == 0;
}

// One tile: columns [x0, x0 + TX), rows [y0, yend), marching in direction
// dir (+1 down from y0, -1 up from yend - 1); diagnostics partial record
// `part` (PASS_DIAG).  Shared by the single-grid and the batched kernels.
// dyn is the kernel's dynamic shared memory (tile_dyn_bytes).  SEG: the pulls
// are staged as row segments (FP32; seg_ok must hold) by bulk copies on the
// stages' mbarriers (sm.bar, initialised by the kernel; bph holds the parity
// each stage waits for next, carried from tile to tile); else each thread
// loads its own pulls into registers, through the read-only path (NC: data
// constant for the launch) or from L2 only (multi-step launches).
template <typename T, int TX, int PASS, bool NC = true, bool SEG = false>
__device__ __forceinline__ void d2q9_tile(TileSmem<T, TX> &sm, T *dyn, const StepParams<T> &P,
                                          const PassArgs &a, int x0, int y0, int yend, int dir,
                                          int part, unsigned &bph)
{
    using SM = TileSmem<T, TX>;
    using SL = SegLayout<TX>;
    static_assert(!SEG || sizeof(T) == 4, "row-segment staging is FP32");
    // staged diagnostics step (its own layout of the staging memory)
    constexpr bool DSEG = SEG && (PASS & PASS_DIAG);
    constexpr int R = SM::R, WP = SM::WP, WM = SM::WM;
    constexpr bool REST_PAIR = sizeof(T) == 4;
    constexpr int NT = SM::NT, NACC = DiagAcc<T>::NACC, NW = NT / 32;
    T *const phs = sm.phs;
    T *const mus = sm.mus;
    T(*const dacc)[NT] = reinterpret_cast<T(*)[NT]>(dyn + (DSEG ? SL::DACC : 0));
    T(*const facc)[NT] = dacc + NACC;
    float *const stg = reinterpret_cast<float *>(dyn);
    int *const dbad = &sm.bad;
    const int lin = threadIdx.y * TX + threadIdx.x;

    const int nx = P.nx, ny = P.ny;
    const unsigned N = (unsigned)P.N;
    const bool small = ny < 4;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const T *__restrict__ fsrc = static_cast<const T *>(a.f_src);
    const T *__restrict__ gsrc = static_cast<const T *>(a.g_src);
    constexpr bool NEED_S = (PASS & (PASS_STATE | PASS_DIAG)) != 0;
    constexpr bool STAGE_S = NEED_S && SEG && !DSEG;  // S staged (else loaded into registers)

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
    // halo columns, from the thread's own loads.
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

    // where the f segments of stage st go and where its g segments go
    auto fbuf = [&](int st) { return stg + (DSEG ? 0 : st * SL::STAGE); };
    auto gbuf = [&](int st) {
        return stg + (DSEG ? SL::DG + st * TYB * SL::NG * SL::W : st * SL::STAGE + SL::GOFF);
    };
    // Bulk staging: one thread arrives on the stage's mbarrier expecting the
    // stage's bytes (before a barrier that precedes the copies), then the
    // thread (ty, 32 + r), r < 20, copies segment r of thread row ty as one
    // bulk copy (two where it wraps the periodic seam) completing on that
    // mbarrier.  Those threads sit in warps without halo work (the phi and mu
    // halo columns belong to threads tx < 4), so the copies do not lengthen
    // the busiest warp.
    constexpr int NSR = SL::NF + SL::NG + 1;  // segments per thread row
    const int rseg = tx - 32;
    auto bulk_expect = [&](int st, int mG, bool doG) {
        if (lin == 32) {
            int rowsG = 0;
#pragma unroll
            for (int j = 0; j < TYB; ++j) rowsG += (doG && mG + j < nout) ? 1 : 0;
            const unsigned bytes = (unsigned)((TYB * SL::NF + rowsG * SL::NG) * SL::W) * 4u +
                                   (STAGE_S ? (unsigned)(rowsG * TX) * 4u : 0u);
            mbar_arrive_expect_tx(&sm.bar[st], bytes);
        }
    };
    auto bulk_copy = [&](int st, int mF, int mG, bool doG) {
        float *const sb = stg + st * SL::STAGE;
        unsigned long long *const bar = &sm.bar[st];
        if (rseg >= 0 && rseg < NSR) {
            const int j = ty, r = rseg;
            const float *src;
            float *dst;
            int m, u0, len;
            if (r < SL::NF) {
                m = mF + j;
                src = reinterpret_cast<const float *>(fsrc) + (unsigned)r * N;
                dst = fbuf(st) + (j * SL::NF + r) * SL::W;
                u0 = x0 - 4;
                len = SL::W;
            } else if (r < SL::NF + SL::NG) {
                m = mG + j;
                src = reinterpret_cast<const float *>(gsrc) + (unsigned)(r - SL::NF) * N;
                dst = gbuf(st) + (j * SL::NG + r - SL::NF) * SL::W;
                u0 = x0 - 4;
                len = SL::W;
            } else {
                m = mG + j;
                src = static_cast<const float *>(a.S);
                dst = sb + SL::SOFF + j * TX;
                u0 = x0;
                len = TX;
            }
            const bool go = r < SL::NF || (doG && m < nout && (r < SL::NF + SL::NG || STAGE_S));
            if (go) {
                const int pop = r < SL::NF ? r : r - SL::NF;
                const int cy =
                    r < SL::NF + SL::NG ? (int)((cy_packed() >> (2 * pop)) & 3u) - 1 : 0;
                const float *const row =
                    src + (unsigned)wrap_row(first + dir * m - cy, ny, small) * nx;
                // columns u0 .. u0 + len - 1, wrapped: at most one seam (nx >= TX + 8)
                const int c0 = u0 < 0 ? u0 + nx : u0;
                const int n1 = len < nx - c0 ? len : nx - c0;
                bulk_g2s(dst, row + c0, (unsigned)n1 * 4u, bar);
                if (n1 < len) bulk_g2s(dst + n1, row, (unsigned)(len - n1) * 4u, bar);
            }
        }
    };
    // wait until stage st's bulk copies have landed (bounded: on a timeout
    // the tile records it in sm.stage_timeout and goes on)
    auto wait_stage = [&](int st) {
        const unsigned par = (bph >> st) & 1u;
        if (!mbar_try_wait(&sm.bar[st], par)) {
            const long long t0 = clock64();
            while (!mbar_try_wait(&sm.bar[st], par)) {
                if (clock64() - t0 > STAGE_WAIT_CYCLES) {
                    sm.stage_timeout = 1;
                    break;
                }
            }
        }
        bph ^= 1u << st;
    };
    // phi row from stage st (thread row ty), keeping the own pulls
    auto phi_row_seg = [&](int sl, int st, T v[9], T &lo) {
        const float *F = fbuf(st) + ty * SL::NF * SL::W;
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = F[i * SL::W + tx + 4 - cxv(i)];
        lo = F[9 * SL::W + tx + 4];
        put_phi(sl, tx + 2, v[0], lo + sum_moving(v));
        if (tx < 4) {
            T h[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = F[i * SL::W + jH + 2 - cxv(i)];
            const T hlo = F[9 * SL::W + jH + 2];
            put_phi(sl, jH, h[0], hlo + sum_moving(h));
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

    // diagnostics: sums in FP64 (FP32: exact pairs); the extrema of |u|^2 and
    // mu and the non-finite flag are exact in the storage type
    if (PASS & PASS_DIAG) {
#pragma unroll
        for (int q = 0; q < NACC; ++q) dacc[q][lin] = T(0);
        facc[0][lin] = T(0);
        facc[1][lin] = T(INFINITY);
        facc[2][lin] = T(-INFINITY);
        if (lin == 0) *dbad = 0;  // read after the march's barriers
    }

    // prologue: phi rows y0-2 .. y0+1 (the own row y0+ty keeps its values),
    // mu rows y0-1 .. y0
    T fcur[9], fnext[9], locur = T(0), lonext = T(0);
    if constexpr (DSEG) {
        // one f buffer: the two phi row pairs one after the other
        if (rseg >= 0 && rseg < NSR) fence_proxy_async_global();
        bulk_expect(1, 0, false);
        __syncthreads();
        bulk_copy(1, -2, 0, false);
        wait_stage(1);
        phi_row_seg(slot(first + dir * (ty - 2)), 1, fnext, lonext);
        bulk_expect(0, 0, false);
        __syncthreads();  // the f buffer is read before it is refilled
        bulk_copy(0, 0, 0, false);
        wait_stage(0);
        phi_row_seg(slot(first + dir * ty), 0, fcur, locur);
        bulk_expect(0, 0, true);
        __syncthreads();
        bulk_copy(0, 2, 0, true);
    } else if constexpr (SEG) {
        // the acquired view of the other tiles' stores precedes the copies
        if (rseg >= 0 && rseg < NSR) fence_proxy_async_global();
        bulk_expect(1, 0, false);
        bulk_expect(0, 0, false);
        __syncthreads();
        bulk_copy(1, -2, 0, false);
        bulk_copy(0, 0, 0, false);
        wait_stage(1);
        wait_stage(0);
        phi_row_seg(slot(first + dir * (ty - 2)), 1, fnext, lonext);
        phi_row_seg(slot(first + dir * ty), 0, fcur, locur);
        bulk_expect(0, 0, true);
        __syncthreads();  // stage 0 is read before it is refilled
        bulk_copy(0, 2, 0, true);
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
        const int st = (t / TYB) & 1;
        T gv[9];
        T Sprev = T(0);
        const unsigned nrow = (unsigned)wrap_row(row, ny, small) * nx;
        if constexpr (SEG) {
            // this iteration's stage has landed (the other stage, and a
            // diagnostics step's one f buffer, are refilled after the barrier
            // below, once every read of them by this iteration's phi rows and
            // the previous iteration is done)
            wait_stage(st);
            if (DSEG && NEED_S && out_ok)
                Sprev = __ldcg(static_cast<const T *>(a.S) + (nrow + xo));  // from L2
            phi_row_seg(ring(2 + ty), st, fnext, lonext);
            if (t + TYB < nout) bulk_expect(st ^ 1, t + TYB, true);
        } else {
            // issue the loads of the own node first so they overlap the stencil work
            const unsigned rm = (unsigned)wrap_row(row - 1, ny, small) * nx;
            const unsigned rp = (unsigned)wrap_row(row + 1, ny, small) * nx;
            pull9<NC>(gsrc, N, rm, nrow, rp, xOm, xO, xOp, gv);
            if (NEED_S && out_ok)
                Sprev = NC ? __ldcs(static_cast<const T *>(a.S) + (nrow + xo))
                           : __ldcg(static_cast<const T *>(a.S) + (nrow + xo));  // from L2
            phi_row(first + dir * (t + 2 + ty), ring(2 + ty), fnext, lonext);
        }
        __syncthreads();
        if (SEG && t + TYB < nout) bulk_copy(st ^ 1, t + TYB + 2, t + TYB, true);
        mu_row(ring(1 + ty - dir), ring(1 + ty), ring(1 + ty + dir));
        __syncthreads();

        const int sm = ring(ty - dir), s0 = ring(ty), sp = ring(ty + dir);
        rb += TYB;
        rb = rb >= R ? rb - R : rb;
        if (out_ok) {
            if constexpr (SEG) {
                const float *G = gbuf(st) + ty * SL::NG * SL::W;
#pragma unroll
                for (int i = 0; i < 9; ++i) gv[i] = G[i * SL::W + tx + 4 - cxv(i)];
                if (STAGE_S) Sprev = stg[st * SL::STAGE + SL::SOFF + ty * TX + tx];
            }
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
        double(*red)[NW] = sm.red;
        const int lane = lin & 31, wid = lin >> 5;
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

// The kernels' dynamic shared memory (tile_dyn_bytes of their tile width).
extern __shared__ float4 tile_dyn[];

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
    unsigned bph = 0;  // no bulk staging here
    d2q9_tile<T, TX, PASS>(sm, reinterpret_cast<T *>(tile_dyn), P, a, blockIdx.x * TX, y0,
                           min(y0 + rows, P.ny), dir, blockIdx.y * gridDim.x + blockIdx.x, bph);
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
    unsigned bph = 0;  // no bulk staging here
    d2q9_tile<T, TX, PASS>(sm, reinterpret_cast<T *>(tile_dyn), P, a, t.x0, t.y0, t.yend,
                           parity ? -t.dir : t.dir, blockIdx.x, bph);
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
__device__ __forceinline__ void st_relaxed_gpu(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Longest wait of a tile for its neighbours, in SM clock cycles (about 2 s):
// a correct launch never comes near it (every CTA is resident: cooperative
// launch, and the oldest unfinished step of any tile can always proceed).
constexpr long long PERSIST_WAIT_CYCLES = 4000000000LL;

// Threads that reduce one grid's diagnostics partials.
constexpr int RG = 128;

// Reduction of grid c's tile partials (tiles k0 .. k1-1) into its record, in
// a fixed order whatever the caller: thread i < RG sums tiles k0 + i,
// k0 + i + RG, ... in turn, a fixed xor butterfly combines each warp, and
// thread 0 combines the four warps as (w0 + w1) + (w2 + w3).  Every thread
// of the CTA calls it (two barriers); red holds 7 x 4 doubles of shared
// memory.  shift_slot >= 0 (FP32 storage): the grid's next
// equilibrium-shift target, alpha times the middle of the mu range (kept if
// the record is not finite or re-centring is off), is written to
// eqs[shift_slot].
__device__ void reduce_case(const DiagPartial *part, int k0, int k1, const BatchCase &cs,
                            DiagPartial *record, int shift_slot, int tid, double *red)
{
    if (tid < RG) {
        double s0 = 0.0, s1 = 0.0, mx = 0.0, mn = DBL_MAX, mxm = -DBL_MAX, s2 = 0.0, bad = 0.0;
#pragma unroll 4
        for (int k = k0 + tid; k < k1; k += RG) {
            const DiagPartial *p = part + k;  // written by other CTAs: read from L2
            s0 += __ldcg(&p->sum_phi);
            s1 += __ldcg(&p->E);
            mx = fmax(mx, __ldcg(&p->u2max));
            mn = fmin(mn, __ldcg(&p->mu_min));
            mxm = fmax(mxm, __ldcg(&p->mu_max));
            s2 += __ldcg(&p->budget);
            bad = fmax(bad, __ldcg(&p->nonfinite));
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mxm = fmax(mxm, __shfl_xor_sync(0xffffffffu, mxm, o));
            bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, o));
        }
        if ((tid & 31) == 0) {
            const int w = tid >> 5;
            red[0 * 4 + w] = s0;
            red[1 * 4 + w] = s1;
            red[2 * 4 + w] = mx;
            red[3 * 4 + w] = mn;
            red[4 * 4 + w] = mxm;
            red[5 * 4 + w] = s2;
            red[6 * 4 + w] = bad;
        }
    }
    __syncthreads();
    if (tid == 0) {
        auto sum4 = [&](int f) { return (red[f * 4] + red[f * 4 + 1]) + (red[f * 4 + 2] + red[f * 4 + 3]); };
        auto max4 = [&](int f) { return fmax(fmax(red[f * 4], red[f * 4 + 1]), fmax(red[f * 4 + 2], red[f * 4 + 3])); };
        auto min4 = [&](int f) { return fmin(fmin(red[f * 4], red[f * 4 + 1]), fmin(red[f * 4 + 2], red[f * 4 + 3])); };
        DiagPartial r;
        r.sum_phi = sum4(0);
        r.E = sum4(1);
        r.u2max = max4(2);
        r.mu_min = min4(3);
        r.mu_max = max4(4);
        r.budget = sum4(5);
        r.nonfinite = max4(6);
        r.pad = 0.0;
        *record = r;
        if (shift_slot >= 0) {
            float *e = cs.eqs;
            float tgt = e[2];
            const double al = cs.pd.alpha * 0.5 * (r.mu_min + r.mu_max);
            if (cs.recentre && r.nonfinite == 0.0 && isfinite(al)) tgt = (float)al;
            e[shift_slot] = tgt;
        }
    }
    __syncthreads();
}

// Per-step launches: records of the step that carried the diagnostics; the
// FP32 target moves at once (the next launch writes with it).
// One CTA of RG threads per grid.
__global__ void __launch_bounds__(RG) d2q9_batch_reduce_kernel(const DiagPartial *__restrict__ part,
                                                               const int *__restrict__ tile0,
                                                               const BatchCase *cases,
                                                               DiagPartial *records, int shift_slot)
{
    __shared__ double red[7 * 4];
    const int c = blockIdx.x;
    reduce_case(part, tile0[c], tile0[c + 1], cases[c], records + c, shift_slot, threadIdx.x, red);
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
// SEGK (FP32): the variant that stages each tile's pulls as row segments
// (grids whose rows are a multiple of 4 nodes; others run the register
// path), diagnostics steps included, with the shared-memory carveout that
// the staging CTAs need.
//
// Memory ordering of the pulls.  Every population, S and phi value that
// other tiles write during the launch is read from L2 only: by the bulk
// row-segment copies (the copy engine reads L2) or, on the register path,
// by ld.global.cg.  The writer CTA stores, passes bar.sync, and its thread 0
// executes fence.acq_rel.gpu and writes the tile's counter (relaxed: fence
// and write form a release); a polling lane of the reader does
// ld.acquire.gpu, observes the count, fences, and the CTA passes bar.sync
// before any copy or load of the next step is issued; a
// thread that issues bulk copies first executes fence.proxy.async.global,
// which orders what it has observed through ordinary loads before its
// copy-engine reads.  No read of this launch's data goes through L1.
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
template <typename T, int TX, bool SEGK>
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
    // the next launch's counters (this launch uses the other set)
    for (int i = blockIdx.x * NTH + lin; i < pa.nctr; i += gridDim.x * NTH) pa.ctr_next[i] = 0;
    if (fixed && (int)blockIdx.x >= pa.ntiles) return;
    // s_next and s_stop (the next pair, the error word) are written by thread
    // 0 before the barrier that ends a pair and read after it; they are
    // double-buffered by the CTA's pair count, so that a slot is written again
    // only after every thread has passed the barriers of the pair between
    __shared__ int s_next[2], s_stop[2], s_abort, s_diag;
    // s_stepdone: every tile has finished the steps before this one.  It is
    // read by every thread at the top of a pair and written only by thread 0
    // between the two barriers that end a pair; lane 31 of the waiting warp
    // records what it observed in s_seen, which thread 0 folds in there.
    __shared__ int s_stepdone, s_seen;
    if (lin == 0) s_stepdone = s_seen = 0;
    __syncthreads();
    int it = 0;
    // a tile whose state is invalid: NaN in its rest population of both
    // buffers (so phi, whichever buffer is current) and in S
    auto poison = [&](const BatchCase &c, const BatchTile &t, const StepParams<T> &P) {
        T *S = static_cast<T *>(c.S);
        T *f0 = static_cast<T *>(c.f[0]), *f1 = static_cast<T *>(c.f[1]);
        for (int x = t.x0 + threadIdx.x; x < t.x0 + TX && x < P.nx; x += blockDim.x)
            for (int y = t.y0 + (int)threadIdx.y; y < t.yend; y += TYB) {
                const size_t n = (size_t)y * P.nx + x;
                S[n] = T(NAN);
                f0[n] = T(NAN);
                f1[n] = T(NAN);
            }
    };
    __shared__ TileSmem<T, TX> sm;
    // the stages' mbarriers (bulk-copy staging), their next parities
    unsigned bph = 0;
    if (SEGK) {
        if (lin == 0) {
            mbar_init(&sm.bar[0], 1);
            mbar_init(&sm.bar[1], 1);
            sm.stage_timeout = 0;
            mbar_init_fence();
        }
        __syncthreads();
    }
    int tk = blockIdx.x;
    while (tk < total) {
        const int k = tk / pa.ntiles, ti = tk - k * pa.ntiles;
        // the next pair (queue) and the error word are fetched now and used
        // after the tile, so that neither round trip delays it
        int tk_next = 0, err_seen = 0;  // thread 0's, kept in registers until the tile ends
        if (lin == 0) {
            if (!fixed) tk_next = atomicAdd(pa.ctr, 1) + (int)gridDim.x;
            err_seen = ld_relaxed_gpu(pa.err);
        }
        const BatchTile t = pa.tiles[ti];
        const BatchCase &c = pa.cases[t.c];
        const StepParams<T> P = *reinterpret_cast<const StepParams<T> *>(
            sizeof(T) == 4 ? (const void *)&c.pf : (const void *)&c.pd);
        // Before step k > 0 of a tile: once this CTA has seen every tile finish
        // step k - 1 (the step's completion count, acquired), no wait is
        // needed; else lane 31 reads that count while the other lanes wait
        // for the tile and its neighbours.
        if (k > 0 && !(s_stepdone >= k && ti != pa.stall_tile)) {
            if (lin < 32) {
                const int *nb = pa.nbr + (size_t)ti * (PERSIST_NBMAX + 1);
                bool bad = false;
                if (lin == 31 && ld_acquire_gpu(pa.step_done + (k - 1)) == pa.ntiles) s_seen = k;
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
                poison(c, t, P);
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
        T *const dyn = reinterpret_cast<T *>(tile_dyn);
        const bool seg = SEGK && seg_ok<T, TX>(P.nx, a.f_src, a.g_src, a.S);
        if (k == pa.diag_k) {
            if (seg)
                d2q9_tile<T, TX, PASS_STATE | PASS_DIAG, false, SEGK>(sm, dyn, P, a, t.x0, t.y0,
                                                                       t.yend, dir, ti, bph);
            else
                d2q9_tile<T, TX, PASS_STATE | PASS_DIAG, false>(sm, dyn, P, a, t.x0, t.y0, t.yend,
                                                                 dir, ti, bph);
        } else if (seg) {
            d2q9_tile<T, TX, PASS_STATE, false, SEGK>(sm, dyn, P, a, t.x0, t.y0, t.yend, dir, ti,
                                                      bph);
        } else {
            d2q9_tile<T, TX, PASS_STATE, false>(sm, dyn, P, a, t.x0, t.y0, t.yend, dir, ti, bph);
        }
        // every thread read s_stepdone at this pair's top, before the tile's
        // barriers: thread 0 folds in what lane 31 saw, for the next pair, and
        // publishes the next pair and the error word it fetched
        if (lin == 0) {
            if (s_seen > s_stepdone) s_stepdone = s_seen;
            s_next[it & 1] = tk_next;
            s_stop[it & 1] = err_seen;
        }
        __syncthreads();  // every output of the step (and its partial) is stored
        if (SEGK && sm.stage_timeout) {
            // a stage's copies did not land in time: the tile is invalid; the
            // error word stops the other CTAs
            if (lin == 0) {
                atomicExch(pa.err, 1);
                if (pa.err_host) {
                    *(volatile int *)pa.err_host = 1;
                    __threadfence_system();
                }
            }
            poison(c, t, P);
            return;
        }
        const int next = fixed ? tk + pa.ntiles : s_next[it & 1];
        const int stop = s_stop[it & 1];
        ++it;
        // Thread 0 publishes the tile's step (release) and counts it, and the
        // CTA waits for it before the next pair (letting the other warps run
        // ahead into the next tile's copies made a step 27% slower).  The
        // counters of the launch's last steps (one atomic per tile each): the
        // last tile of a grid in the diagnostics step reduces that grid's
        // partials (ctr[3] counts the grids reduced); the last tile of the
        // final step (then every pair is done) records the final shift, after
        // every reduction.
        const bool last_steps = k == pa.diag_k || k == pa.nsteps - 1;
        // One release fence, then the counters as relaxed writes and atomics
        // (each a release pattern): the barrier above orders every thread's
        // stores of the tile before the fence.  A fence followed by a release
        // store (two fences) cost about 3% of a step.
        if (lin == 0) {
            fence_acq_rel_gpu();
            st_relaxed_gpu(pa.flags + ti, k + 1);
            atomicAdd(pa.step_done + k, 1);  // the step's completion count
            if (last_steps) {
                int fl = 0;
                if (k == pa.diag_k &&
                    atomicAdd(pa.case_ctr + t.c, 1) == pa.tile0[t.c + 1] - pa.tile0[t.c] - 1)
                    fl |= 1;
                if (k == pa.nsteps - 1 && atomicAdd(pa.ctr + 2, 1) == pa.ntiles - 1) fl |= 2;
                s_diag = fl;
            }
        }
        __syncthreads();
        const int fl = last_steps ? s_diag : 0;
        if (fl & 1) {  // every partial of this grid's diagnostics step is written
            __threadfence();
            reduce_case(pa.partials, pa.tile0[t.c], pa.tile0[t.c + 1], pa.cases[t.c],
                        pa.records + t.c, sizeof(T) == 4 ? 3 : -1, lin, &sm.red[0][0]);
            if (lin == 0) {
                __threadfence();
                atomicAdd(pa.ctr + 3, 1);
            }
        }
        if (fl & 2) {  // every pair is done; wait for the reductions if there are any
            if (lin == 0 && pa.diag_k >= 0) {
                const long long t0 = clock64();
                while (ld_acquire_gpu(pa.ctr + 3) < pa.ncases &&
                       clock64() - t0 < PERSIST_WAIT_CYCLES)
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

// The staging multi-step kernel's dynamic shared memory limit (above the
// default 48 KB) and shared-memory carveout (all of the unified L1 / shared
// memory: four staging CTAs per SM, whose copies bypass L1), set once per
// device.
template <int TX>
cudaError_t seg_attrs()
{
    static int done[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    const void *k = (const void *)d2q9_batch_persist_kernel<float, TX, true>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tile_dyn_bytes<float, TX, true>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
    return e;
}

template <typename T, int PASS>
cudaError_t launch_pass(const void *params, const PassArgs &a, const LaunchShape &s,
                        cudaStream_t st)
{
    const StepParams<T> &P = *static_cast<const StepParams<T> *>(params);
    constexpr int dyn = tile_dyn_bytes<T, TXW>();
    dim3 grid(s.grid_x, s.grid_y), block(TXW, TYB);
    d2q9_pass_kernel<T, TXW, PASS><<<grid, block, dyn, st>>>(P, a, s.rows);
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
    constexpr int dyn = tile_dyn_bytes<T, TX>();
    if (partials)
        d2q9_batch_kernel<T, TX, PASS_STATE | PASS_DIAG>
            <<<ntiles, block, dyn, st>>>(cases, tiles, parity, partials);
    else
        d2q9_batch_kernel<T, TX, PASS_STATE><<<ntiles, block, dyn, st>>>(cases, tiles, parity, nullptr);
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
    d2q9_batch_reduce_kernel<<<ncases, RG, 0, st>>>(partials, tile0, cases, records,
                                                     precision == 0 ? -1 : 2);
    return cudaGetLastError();
}

namespace {

template <typename T, int TX, bool SEGK>
cudaError_t launch_persist_t(const PersistArgs &pa, int nctas, cudaStream_t st)
{
    constexpr int dyn = tile_dyn_bytes<T, TX, SEGK>();
    cudaError_t e = SEGK ? seg_attrs<TX>() : cudaSuccess;
    if (e != cudaSuccess) return e;
    // The counters (ticket, unused, final-step tiles done, grids reduced; the
    // tiles' step counters; the spare one that nothing sets, for
    // fault-injection tests; the grids' diagnostics tiles done) are zero:
    // the previous launch on the other set zeroed this one.
    void *args[] = {(void *)&pa};
    return cudaLaunchCooperativeKernel((const void *)d2q9_batch_persist_kernel<T, TX, SEGK>,
                                       dim3(nctas), dim3(TX, TYB), args, dyn, st);
}

template <typename T, int TX, bool SEGK>
int persist_ctas_per_sm_t()
{
    int n = 0;
    constexpr int dyn = tile_dyn_bytes<T, TX, SEGK>();
    if (SEGK && seg_attrs<TX>() != cudaSuccess) return 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, d2q9_batch_persist_kernel<T, TX, SEGK>, TX * TYB, dyn);
    return e == cudaSuccess ? n : 0;
}

}  // namespace

cudaError_t d2q9_prepare()
{
    const cudaError_t e = seg_attrs<128>();
    return e != cudaSuccess ? e : seg_attrs<64>();
}

cudaError_t d2q9_batch_persist(int precision, int width, bool seg, const PersistArgs &pa,
                               int nctas, cudaStream_t st)
{
    if (pa.flags != pa.ctr + 4 || pa.case_ctr != pa.flags + pa.ntiles + 1 ||
        pa.step_done != pa.case_ctr + pa.ncases ||
        pa.nctr != pa.ntiles + 5 + pa.ncases + PERSIST_STEP_CAP || pa.nsteps > PERSIST_STEP_CAP)
        return cudaErrorInvalidValue;
    if (precision == 0)
        return width == 64 ? launch_persist_t<double, 64, false>(pa, nctas, st)
                           : launch_persist_t<double, 128, false>(pa, nctas, st);
    if (seg)
        return width == 64 ? launch_persist_t<float, 64, true>(pa, nctas, st)
                           : launch_persist_t<float, 128, true>(pa, nctas, st);
    return width == 64 ? launch_persist_t<float, 64, false>(pa, nctas, st)
                       : launch_persist_t<float, 128, false>(pa, nctas, st);
}

int d2q9_batch_persist_ctas_per_sm(int precision, int width, bool seg)
{
    if (precision == 0)
        return width == 64 ? persist_ctas_per_sm_t<double, 64, false>()
                           : persist_ctas_per_sm_t<double, 128, false>();
    if (seg)
        return width == 64 ? persist_ctas_per_sm_t<float, 64, true>()
                           : persist_ctas_per_sm_t<float, 128, true>();
    return width == 64 ? persist_ctas_per_sm_t<float, 64, false>()
                       : persist_ctas_per_sm_t<float, 128, false>();
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
