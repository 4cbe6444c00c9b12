// loss_noalloc.cu -- sg_pyramid_loss for callers that cannot allocate device memory.
//
// Some callers are handed their input and output buffers by a host framework that owns
// the whole device memory pool and gives this library no way to obtain scratch memory.
// Others run on a latency-critical thread where cudaMalloc is off limits because it can
// block on, or synchronise with, other work on the device.  For them this entry point
// uses a fixed scratch area compiled into the library instead of a caller workspace.
//
// The scratch is a file-scope device array of SG_LOSS_NOALLOC_SCRATCH_BYTES (16 MiB) that
// every GPU loading the library holds until the process exits.  On the host its name is
// only a stand-in, so the device address is looked up with cudaGetSymbolAddress once per
// device (on the first call made with that device current) and cached for the life of the
// process.  A device reset (cudaDeviceReset, or the primary context destroyed and created
// again) reloads the module, possibly elsewhere, and leaves that cached address stale: do not
// use this entry point across a device reset.  Every call uses the same array and leaves its
// contents behind; the loss clears the counters it needs (with a memset on the stream) and
// overwrites every partial sum, so stale contents never matter -- but two calls whose GPU
// work overlaps (different streams, same device) race on the array.
#include <mutex>

#include "sg_common.cuh"

namespace sg {
size_t loss_workspace_size_kc(const sg_view *vh, int n_views, int KC);
int loss_decoder_partials(const sg_loss_config *lc, int C);
sg_status check_loss_args(const sg_images *rendered, const sg_targets *gt, const sg_view *views,
                          const sg_view *views_host, int32_t n_views, int32_t C, const sg_loss_config *lcfg,
                          float *terms, sg_images *dL, uint32_t *status);
}

using namespace sg;

static __device__ __align__(256) unsigned char g_loss_scratch[SG_LOSS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_loss_scratch on the current device (looked up once per device).
sg_status scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("pyramid_loss_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("pyramid_loss_noalloc: device %d beyond the supported %d", dev, kMaxDevices);
        return SG_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_loss_scratch);
        if (e != cudaSuccess || !p) {
            set_error("pyramid_loss_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SG_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SG_OK;
}
}  // namespace

extern "C" sg_status sg_pyramid_loss_noalloc(const sg_images *rendered, const sg_targets *gt,
                                             const sg_view *views, const sg_view *views_host,
                                             int32_t n_views, int32_t C, const sg_loss_config *lcfg,
                                             float *terms, sg_images *dL, uint32_t *status,
                                             sg_stream_t stream) {
    // the arguments are checked exactly as sg_pyramid_loss checks them before the scratch
    // need is computed from them
    const sg_status ok = check_loss_args(rendered, gt, views, views_host, n_views, C, lcfg, terms, dL, status);
    if (ok != SG_OK) return ok;
    const size_t need = loss_workspace_size_kc(views_host, n_views, loss_decoder_partials(lcfg, C));
    if (need > (size_t)SG_LOSS_NOALLOC_SCRATCH_BYTES) {
        set_error("pyramid_loss_noalloc: these images need %zu bytes of scratch, more than the "
                  "built-in %u bytes; use sg_pyramid_loss with a workspace",
                  need, (unsigned)SG_LOSS_NOALLOC_SCRATCH_BYTES);
        return SG_ERR_CAPACITY;
    }
    void *scratch = nullptr;
    const sg_status s = scratch_address(&scratch);
    if (s != SG_OK) return s;
    return sg_pyramid_loss(rendered, gt, views, views_host, n_views, C, lcfg, terms, dL, scratch,
                           (size_t)SG_LOSS_NOALLOC_SCRATCH_BYTES, status, stream);
}
