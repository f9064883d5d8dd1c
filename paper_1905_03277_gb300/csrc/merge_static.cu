// hmfsr_merge_static: the merge without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they merge: code running
// inside another framework's memory pool or a real-time capture path that must not
// call cudaMalloc (which can synchronise the device and stall other streams), and plugin
// hosts that hand over only input and output buffers.  For them this entry point takes
// its scratch from one file-scope device array of fixed size, created when the library's
// module is loaded on a device and held by every GPU that loads it until the process
// exits.  Calls share that array, so calls whose work overlaps on the GPU (different
// streams, or several host threads) race with each other; serialise them.
#include <mutex>

#include "hmfsr_internal.cuh"

using namespace hmfsr;

namespace {

// Largest scratch a call may use: 32 MiB, enough for e.g. 8 frames of 768 x 512.
constexpr size_t kStaticScratchBytes = 32u << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; resolved once per device
// (the array's name is only a host-side stand-in in host code) and kept until the
// process exits: it belongs to the device's primary context, which cudaDeviceReset ends,
// so the entry point is not for use on a device after a reset (the header says so).
hmfsr_status scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HMFSR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HMFSR_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return HMFSR_OK;
}

}  // namespace

extern "C" hmfsr_status hmfsr_merge_static(const uint16_t *burst_dev, const hmfsr_burst_desc *desc,
                                           const float *motion_dev, const hmfsr_merge_params *params, int scale_num,
                                           int scale_den, float *rgb_dev, float *den_dev, void *stream) {
    const size_t need = hmfsr_workspace_size(HMFSR_OP_MERGE, desc, params ? params->tile : 0, scale_num, scale_den);
    if (need == 0) return hmfsr_merge(burst_dev, desc, motion_dev, params, scale_num, scale_den, rgb_dev, den_dev,
                                      nullptr, 0, stream);  // reports the argument error, launches nothing
    if (need > kStaticScratchBytes) return HMFSR_ERR_WORKSPACE;
    void *ws = nullptr;
    hmfsr_status st = scratch_address(&ws);
    if (st != HMFSR_OK) return st;
    // every plane the merge reads is written earlier in the same call, so nothing in the
    // shared array needs clearing between calls
    return hmfsr_merge(burst_dev, desc, motion_dev, params, scale_num, scale_den, rgb_dev, den_dev, ws,
                       kStaticScratchBytes, stream);
}
