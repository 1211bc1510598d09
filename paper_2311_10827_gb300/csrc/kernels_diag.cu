// Second pass of the diagnostics reduction: the per-CTA FP64 partials of a
// pass over the grid are combined by one CTA in a fixed order (deterministic:
// the same partials always give bit-identical results).
#include <float.h>
#include <math.h>

#include "lbm_internal.h"

namespace wblbm {
namespace {

constexpr int RT = 256;

__global__ void __launch_bounds__(RT) diag_reduce_kernel(const DiagPartial *__restrict__ part,
                                                         int n, DiagPartial *__restrict__ out)
{
    double s0 = 0.0, s1 = 0.0, mx = 0.0, mn = DBL_MAX, mxm = -DBL_MAX, s2 = 0.0, bad = 0.0;
    for (int k = threadIdx.x; k < n; k += RT) {
        const DiagPartial p = part[k];
        s0 += p.sum_phi;
        s1 += p.E;
        mx = fmax(mx, p.u2max);
        mn = fmin(mn, p.mu_min);
        mxm = fmax(mxm, p.mu_max);
        s2 += p.budget;
        bad = fmax(bad, p.nonfinite);
    }
    __shared__ double red[7][RT];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = mx;
    red[3][threadIdx.x] = mn;
    red[4][threadIdx.x] = mxm;
    red[5][threadIdx.x] = s2;
    red[6][threadIdx.x] = bad;
    __syncthreads();
    for (int h = RT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const int o = threadIdx.x + h;
            red[0][threadIdx.x] += red[0][o];
            red[1][threadIdx.x] += red[1][o];
            red[2][threadIdx.x] = fmax(red[2][threadIdx.x], red[2][o]);
            red[3][threadIdx.x] = fmin(red[3][threadIdx.x], red[3][o]);
            red[4][threadIdx.x] = fmax(red[4][threadIdx.x], red[4][o]);
            red[5][threadIdx.x] += red[5][o];
            red[6][threadIdx.x] = fmax(red[6][threadIdx.x], red[6][o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DiagPartial r;
        r.sum_phi = red[0][0];
        r.E = red[1][0];
        r.u2max = red[2][0];
        r.mu_min = red[3][0];
        r.mu_max = red[4][0];
        r.budget = red[5][0];
        r.nonfinite = red[6][0];
        r.pad = 0.0;
        *out = r;
    }
}

// equilibrium shift target: alpha times the middle of the mu range (at
// equilibrium mu is uniform, so the stored moving populations become the
// small non-equilibrium parts)
__global__ void eq_recentre_kernel(const DiagPartial *rec, double alpha, float *target)
{
    const DiagPartial r = *rec;
    const double a = alpha * 0.5 * (r.mu_min + r.mu_max);
    if (r.nonfinite == 0.0 && isfinite(a)) *target = (float)a;
}

}  // namespace

cudaError_t diag_reduce(const DiagPartial *partials, int n, DiagPartial *out, cudaStream_t st)
{
    diag_reduce_kernel<<<1, RT, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

cudaError_t eq_recentre(const DiagPartial *rec, double alpha, float *target, cudaStream_t st)
{
    eq_recentre_kernel<<<1, 1, 0, st>>>(rec, alpha, target);
    return cudaGetLastError();
}

}  // namespace wblbm
