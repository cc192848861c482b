// gs_noalloc.cu -- gs_render_static: the forward render with its scratch in a
// fixed-size array that lives in the library's own device memory.
//
// Some callers cannot hand the renderer a workspace: a sensor plugin running
// inside a host simulator whose device memory is owned and fully reserved by
// another framework's allocator, or code on a real-time path that is not
// allowed to allocate after start-up.  They can call gs_render_static, which
// takes no workspace and allocates nothing; it renders into the caller's
// output buffers using the static array below.  gs_render_static_status reads
// (and clears) the device status word a gs_render_static call leaves in that
// array, since the caller has no workspace pointer to pass to gs_get_status.
#include <cuda_runtime.h>

#include <mutex>

#include "gs.h"
#include "gs_launch.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)GS_STATIC_SCRATCH_BYTES;

// One copy per GPU that loads the library, held until the process exits.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices]; // device address of the array, per device; null until looked up

// The array's host-side name is only a stand-in: its device address is looked
// up with the device current, once per device.  A failed lookup is not kept
// (the next call tries again), so a transient failure -- the module's memory
// could not be reserved yet -- does not disable the entry point for good.
gs_status static_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gs::record_cuda_error(e);
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError(); // not sticky: leave no error behind for later launch checks
            return gs::record_cuda_error(e);
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

} // namespace

extern "C" gs_status gs_render_static(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams,
                                      const gs_render_config *cfg, float *out_rgb, float *out_depth, float *out_T,
                                      int32_t *out_ncontrib, void *stream)
{
    size_t need = 0;
    gs_status st = gs_render_workspace_size(cfg, batch, &need);
    if (st != GS_OK) return st;
    if (need > kStaticScratchBytes) return GS_ERR_WORKSPACE_TOO_SMALL; // problem larger than the static scratch
    void *scratch = nullptr;
    st = static_scratch(&scratch);
    if (st != GS_OK) return st;
    gs::ProfileSuppress no_events; // stage profiling would create CUDA events
    return gs_render(g, batch, cams, cfg, scratch, kStaticScratchBytes, out_rgb, out_depth, out_T, out_ncontrib,
                     stream);
}

extern "C" gs_status gs_render_static_status(void *stream, int32_t *device_status)
{
    if (!device_status) return GS_ERR_INVALID_ARG;
    void *scratch = nullptr;
    gs_status st = static_scratch(&scratch);
    if (st != GS_OK) return st;
    return gs_get_status(scratch, kStaticScratchBytes, stream, device_status);
}
