// noalloc.cu -- supra_bmode_noalloc: the fused B-mode chain of one frame for
// callers that may not allocate device memory.
//
// supra_bmode needs a caller-provided device workspace for the log-compressed
// lines it scan-converts.  Some callers cannot obtain one: a real-time
// acquisition loop that is not allowed to call cudaMalloc after start-up
// (cudaMalloc can synchronize the device and has no latency bound, which breaks
// a per-frame deadline), or a host application whose device memory is owned by
// another framework's pool that this library cannot reach.  This entry point
// takes its scratch from a fixed array in the library's own device memory
// instead, and otherwise runs exactly the kernels supra_bmode runs.
#include <cuda_runtime.h>

#include <mutex>

#include "supra.h"

namespace {

// Scratch for the log-compressed lines of one frame.  Every GPU that loads the
// library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name only stands for the symbol, so its address has to be asked for
// once per device with that device current.
int scratch_on_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SUPRA_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SUPRA_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SUPRA_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SUPRA_OK;
}

}  // namespace

extern "C" SUPRA_API int supra_bmode_noalloc(const supra_plan *plan, const int16_t *ch, uint8_t *out, void *stream) {
    if (!plan || !ch || !out) return SUPRA_EINVAL;
    const size_t need = supra_bmode_workspace_size(1, &plan);
    if (need > kNoAllocScratchBytes) return SUPRA_EINVAL;
    void *scratch = nullptr;
    const int rc = scratch_on_current_device(&scratch);
    if (rc != SUPRA_OK) return rc;
    return supra_bmode(plan, ch, out, need ? scratch : nullptr, need ? kNoAllocScratchBytes : 0, stream);
}
