// Diagnostics of a caller-held state without any device allocation.
//
// lbm_create allocates the context's buffers with cudaMalloc, and so does
// the diagnostics reduction's scratch (one partial record per CTA).  Some
// callers cannot allocate device memory at all: code that runs inside a
// host framework's memory pool or a pre-sized arena, code that must not
// disturb the allocator while another component is capturing work, or a
// library boundary whose owner forbids device allocations after start-up.
// For them lbm_diagnostics_noalloc runs the same two kernels as
// lbm_diagnostics, with the per-CTA partials in the file-scope array below
// instead of allocated scratch.
#include <cuda_runtime.h>

#include <math.h>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

using wblbm::DiagPartial;

// Fixed scratch: one partial record per CTA of the diagnostics pass.
// 4096 records x 64 B = 256 KiB, held by every GPU that loads the library
// until the process exits (enough for grids up to about 134 million nodes).
constexpr int NOALLOC_MAX_CTAS = 4096;
static __device__ __align__(256) DiagPartial g_noalloc_partials[NOALLOC_MAX_CTAS];

// Device address of g_noalloc_partials per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current (cudaGetSymbolAddress).
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
DiagPartial *g_addr[MAX_DEVICES];

int scratch_address(DiagPartial **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return LBM_ERR_CUDA;
    if (dev >= MAX_DEVICES) return LBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p)
            return LBM_ERR_CUDA;
        g_addr[dev] = static_cast<DiagPartial *>(p);
    }
    *out = g_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_diagnostics_noalloc(const lbm_grid *grid, int lattice, const lbm_params *params,
                                       const void *f, const void *g, const void *S_prev,
                                       double *out, void *cuda_stream)
{
    if (!grid || !params || !f || !g || !S_prev || !out) return LBM_ERR_INVALID_ARG;
    const lbm_params &p = *params;
    // the checks of lbm_create, then what this entry point supports
    if (int rc = wblbm::validate_problem(grid, lattice, params)) return rc;
    if (lattice != LBM_D2Q9 || (p.precision != LBM_FP64 && p.precision != LBM_FP32))
        return LBM_ERR_INVALID_ARG;

    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;
    const wblbm::LaunchShape shape = wblbm::d2q9_shape(grid->nx, grid->ny, nsm);
    if (shape.nblocks > NOALLOC_MAX_CTAS) return LBM_ERR_INVALID_ARG;

    DiagPartial *partials = nullptr;
    if (int rc = scratch_address(&partials)) return rc;

    const wblbm::Derived d = wblbm::derive_params(p);
    wblbm::StepParams<double> pd;
    wblbm::StepParams<float> pf;
    wblbm::fill_step_params(pd, *grid, p, d);
    wblbm::fill_step_params(pf, *grid, p, d);
    const void *prm = p.precision == LBM_FP64 ? (const void *)&pd : (const void *)&pf;

    wblbm::PassArgs a = {};
    a.f_src = f;
    a.g_src = g;
    a.S = const_cast<void *>(S_prev);  // read only: the diagnostics pass writes no state
    a.partials = partials;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // every partial record is written by its CTA before the reduction reads
    // it, so the scratch needs no clearing between calls
    if (wblbm::d2q9_pass(p.precision, wblbm::PASS_DIAG, prm, a, shape, st) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (wblbm::diag_reduce(partials, shape.nblocks, reinterpret_cast<DiagPartial *>(out), st) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}
