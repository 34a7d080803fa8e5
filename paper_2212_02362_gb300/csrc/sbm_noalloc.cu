// sbm_noalloc.cu — sbm_residual_noalloc: the FP64 residual and its norm on
// caller-owned buffers, for callers that must not allocate device memory.
//
// Its only scratch (the per-block partial sums of r^2 and the reduced result) is
// the fixed file-scope device array below, so the call needs neither a grid
// handle (whose creation allocates) nor any allocation of its own.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/sbm.h"
#include "sbm_common.cuh"

using namespace sbm;

namespace {

// Partial sums of r^2 for up to SBM_NOALLOC_MAX_BLOCKS stencil blocks, then 8
// result slots.  Every GPU that loads the library holds this array until exit.
constexpr int kResultSlots = 8;
static __device__ __align__(256) double g_noalloc_scratch[SBM_NOALLOC_MAX_BLOCKS + kResultSlots];

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};   // device address of the array, per device
std::mutex g_scratch_mutex;

// Resolve the array's device address on the current device (once per device).
cudaError_t scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

sbm_status fail(sbm_status s, const char *msg)
{
    set_library_error(msg);
    return s;
}

}  // namespace

extern "C" sbm_status sbm_residual_noalloc(int dim, const int n[3], double h, const double moduli[3],
                                           const unsigned dirichlet_faces[3], const double *psi, const double *f,
                                           const double *u, double *r, double *norm, void *stream)
{
    if ((dim != 2 && dim != 3) || !n || !moduli || !dirichlet_faces || !psi || !f || !u || !r || !norm)
        return fail(SBM_ERR_ARG, "bad dimension or null argument");
    if (n[0] < 2 || n[1] < 2 || (dim == 3 && n[2] < 2) || (dim == 2 && n[2] != 1))
        return fail(SBM_ERR_ARG, "node counts must be >= 2 (n[2] == 1 in 2D)");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(SBM_ERR_ARG, "h must be positive");
    if (!moduli_definite(dim, moduli[0], moduli[1], moduli[2]))
        return fail(SBM_ERR_ARG, "moduli are not positive definite");
    Geom g{};
    g.dim = dim;
    g.nx = n[0];
    g.ny = n[1];
    g.nz = n[2];
    g.sx = n[0];                       // the caller's packed layout
    g.sy = (long long)n[0] * n[1];
    g.cs = g.sy * n[2];
    for (int p = 0; p < 3; ++p) g.dm[p] = p < dim ? (dirichlet_faces[p] & (dim == 3 ? 63u : 15u)) : 0u;
    const long long nblocks = sweep_blocks(g, true);
    if (nblocks > SBM_NOALLOC_MAX_BLOCKS) {
        char msg[160];
        snprintf(msg, sizeof(msg), "grid needs %lld partial sums; the fixed scratch holds %d", nblocks,
                 (int)SBM_NOALLOC_MAX_BLOCKS);
        return fail(SBM_ERR_ARG, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SBM_ERR_CUDA, "cudaGetDevice failed");
    // every array must be memory of the current device: a host pointer or another
    // GPU's pointer is refused here instead of reaching the kernel
    if (!is_dev_ptr(psi, dev) || !is_dev_ptr(f, dev) || !is_dev_ptr(u, dev) || !is_dev_ptr(r, dev))
        return fail(SBM_ERR_ARG, "psi, f, u and r must be device memory of the current device");
    double *scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return fail(SBM_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SweepArgs<double, double> a;
    a.g = g;
    a.u = u;
    a.f = f;
    a.psi = psi;
    a.out = r;
    a.part = scratch;
    a.c = make_coef<double>(dim, h, moduli[0], moduli[1], moduli[2]);
    a.wk[0] = a.wk[1] = a.wk[2] = 0.0;
    a.kchunk = 0;
    if ((e = launch_sweep<double, double>(kResidual, a, st)) != cudaSuccess) return fail(SBM_ERR_CUDA, cudaGetErrorString(e));
    double *res = scratch + SBM_NOALLOC_MAX_BLOCKS;
    if ((e = launch_norm_final(scratch, (int)nblocks, res, 0, st)) != cudaSuccess) return fail(SBM_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(norm, res + 1, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return fail(SBM_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(SBM_ERR_CUDA, cudaGetErrorString(e));
    return SBM_OK;
}
