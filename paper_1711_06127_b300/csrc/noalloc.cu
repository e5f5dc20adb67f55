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
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "supra.h"

namespace {

// Scratch for the log-compressed lines of one frame.  Every GPU that loads the
// library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchAddr {
    unsigned long long ctx_id;   // context the address belongs to (0: unknown)
    void *ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// Unique id of the calling thread's current context (0 if the driver cannot
// tell), through the runtime's driver entry points (no libcuda link).  A device
// reset destroys the primary context and the next one gets a new id, so an
// address looked up in the old context is never reused.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(p);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device.  In host code the
// array's name only stands for the symbol, so its address has to be asked for
// once per device (and context) with that device current.
int scratch_on_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SUPRA_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SUPRA_EINVAL;
    // (0 when no context is current yet: the address is then looked up again, which makes
    // the primary context current, and cached from the next call on)
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchAddr &s = g_scratch[dev];
    if (!s.ptr || s.ctx_id != ctx || ctx == 0) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SUPRA_ECUDA;
        }
        s.ptr = p;
        s.ctx_id = ctx;
    }
    *out = s.ptr;
    return SUPRA_OK;
}

}  // namespace

extern "C" SUPRA_API int supra_bmode_noalloc(const supra_plan *plan, const int16_t *ch, uint8_t *out, void *stream) {
    if (!plan || !ch || !out) return SUPRA_EINVAL;
    const size_t need = supra::bmode_min_workspace(1, &plan);
    if (need > kNoAllocScratchBytes) return SUPRA_EINVAL;
    // the scratch also holds depth-segment boundary records when they fit (else the
    // segments beamform their halos: the same images)
    const bool use = supra_bmode_workspace_size(1, &plan) > 0;
    void *scratch = nullptr;
    if (use) {
        const int rc = scratch_on_current_device(&scratch);
        if (rc != SUPRA_OK) return rc;
    }
    return supra_bmode(plan, ch, out, use ? scratch : nullptr, use ? kNoAllocScratchBytes : 0, stream);
}
