// gs_noalloc.cu -- gs_render_static: the forward render with its scratch in a
// fixed-size array that lives in the library's own device memory.
//
// Some callers cannot hand the renderer a workspace: a sensor plugin running
// inside a host simulator whose device memory is owned and fully reserved by
// another framework's allocator, or code on a real-time path that is not
// allowed to allocate after start-up.  They can call gs_render_static, which
// takes no workspace and allocates nothing; it renders into the caller's
// output buffers using the static array below.
#include <cuda_runtime.h>

#include <mutex>

#include "gs.h"
#include "gs_launch.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)GS_STATIC_SCRATCH_BYTES;

// One copy per GPU that loads the library, held until the process exits.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
void *g_scratch_ptr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

} // namespace

extern "C" gs_status gs_render_static(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams,
                                      const gs_render_config *cfg, float *out_rgb, float *out_depth, float *out_T,
                                      int32_t *out_ncontrib, void *stream)
{
    size_t need = 0;
    gs_status st = gs_render_workspace_size(cfg, batch, &need);
    if (st != GS_OK) return st;
    if (need > kStaticScratchBytes) return GS_ERR_WORKSPACE_TOO_SMALL; // problem larger than the static scratch
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gs::record_cuda_error(e);
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
    // The array's host-side name is only a stand-in: its device address is
    // looked up once per device, with that device current.
    std::call_once(g_once[dev], [dev]() {
        g_scratch_err[dev] = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_static_scratch);
    });
    if (g_scratch_err[dev] != cudaSuccess) return gs::record_cuda_error(g_scratch_err[dev]);
    gs::ProfileSuppress no_events; // stage profiling would create CUDA events
    return gs_render(g, batch, cams, cfg, g_scratch_ptr[dev], kStaticScratchBytes, out_rgb, out_depth, out_T,
                     out_ncontrib, stream);
}
