// The D3Q19 lattice (velocities, weights, periodic neighbour offsets) shared
// by the D3Q19 kernels of the library.  Internal header.
#pragma once

#include <cuda_runtime.h>

namespace wblbm {
namespace d3 {

// column tile of the z-marching pass kernels (threads x, y)
constexpr int TX3 = 32, TY3 = 8;

// velocity order: rest; +x, -x, +y, -y, +z, -z; then the 12 edges
// (+x+y, +x-y, -x+y, -x-y), (+x+z, +x-z, -x+z, -x-z), (+y+z, +y-z, -y+z, -y-z)
__host__ __device__ constexpr int c3x(int i)
{
    return (i == 1 || i == 7 || i == 8 || i == 11 || i == 12)
               ? 1
               : ((i == 2 || i == 9 || i == 10 || i == 13 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int c3y(int i)
{
    return (i == 3 || i == 7 || i == 9 || i == 15 || i == 16)
               ? 1
               : ((i == 4 || i == 8 || i == 10 || i == 17 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr int c3z(int i)
{
    return (i == 5 || i == 11 || i == 13 || i == 15 || i == 17)
               ? 1
               : ((i == 6 || i == 12 || i == 14 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr double w3(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
__device__ __forceinline__ int wrapi(int c, int n)
{
    int r = c % n;
    return r < 0 ? r + n : r;
}
// wrap of c in [-n, 2n) without a division
__device__ __forceinline__ int wrap1(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }
// wrap of any c; `small` (a uniform flag) when c may leave [-n, 2n)
__device__ __forceinline__ int wrapc(int c, int n, bool small) { return small ? wrapi(c, n) : wrap1(c, n); }

template <typename T>
struct Arith3;
template <>
struct Arith3<float> {
    __device__ static float rcp(float x) { return __fdividef(1.0f, x); }
};
template <>
struct Arith3<double> {
    __device__ static double rcp(double x) { return 1.0 / x; }
};

// offsets of the 27 neighbours (dx, dy, dz in -1..1) of a node from wrapped
// coordinates
struct Nb {
    unsigned xs[3], ys[3], zs[3];  // x-1, x, x+1 etc. (already multiplied: y*nx, z*nx*ny)
    __device__ unsigned at(int dx, int dy, int dz) const { return zs[dz + 1] + ys[dy + 1] + xs[dx + 1]; }
};

// per-thread asynchronous 4-byte copy global -> shared; a thread's own
// copies are visible to it after cp_wait_all
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// x, y, z in [0, n): the neighbours at -1..1 wrap without a division
__device__ __forceinline__ void nb_plane(Nb &b, int z, int nx, int ny, int nz)
{
    for (int d = -1; d <= 1; ++d) b.zs[d + 1] = (unsigned)wrap1(z + d, nz) * (unsigned)(nx * ny);
}
__device__ __forceinline__ Nb make_nb(int x, int y, int z, int nx, int ny, int nz)
{
    Nb b;
    for (int d = -1; d <= 1; ++d) {
        b.xs[d + 1] = (unsigned)wrap1(x + d, nx);
        b.ys[d + 1] = (unsigned)wrap1(y + d, ny) * nx;
    }
    nb_plane(b, z, nx, ny, nz);
    return b;
}

}  // namespace d3
}  // namespace wblbm
