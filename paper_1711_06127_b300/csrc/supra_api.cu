// supra_api.cu -- host side of libsupra: plan creation (the geometry-dependent
// work SUPRA does "once for a fixed acquisition", Sec. 2), parameter
// validation, launches of the beamforming / post-processing kernels, and the
// C ABI declared in include/supra.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "das_kernel.cuh"
#include "post_kernels.cuh"
#include "mv_kernel.cuh"
#include "apod_kernel.cuh"
#include "render_kernel.cuh"
#include "internal.h"

using namespace supra;

struct supra_plan {
    DevPlan host;           // host copy of the device record (pointers are device pointers)
    DevPlan *dev = nullptr; // device record
    void *blob = nullptr;   // one device allocation holding every table
    supra_plan_info info{};
    int device = 0;
    int max_active = 0;     // upper bound on the elements inside one pixel's aperture
    std::atomic<int> max_group{kMaxGroup};   // frames per DAS tile (autotuned)
    std::atomic<int> stage_shape{0};         // 16-frame groups: 0 = 3 elements x 3 stages, 1 = 2 x 4
    std::atomic<int> depth_segments{0};      // segments per line, 0 = automatic (fill one wave)
    std::atomic<int> ctas_per_sm{0};         // one-frame launches: 0 = automatic, 2 or 3
    bool ext = false;   // extended transmit model (a plane-wave line or compounding): its own kernels
};

namespace {

constexpr double kPi = 3.14159265358979323846;

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Blackman windowed-sinc low-pass, unit DC gain (odd length, centred).
std::vector<double> lowpass_taps(int K, double cutoff_hz, double rate_hz) {
    std::vector<double> h(K);
    const double fc = cutoff_hz / rate_hz;
    double sum = 0.0;
    for (int k = 0; k < K; ++k) {
        const double mm = k - (K - 1) / 2.0;
        const double x = 2.0 * fc * mm;
        const double sinc = (x == 0.0) ? 1.0 : std::sin(kPi * x) / (kPi * x);
        const double win = K > 1 ? 0.42 - 0.5 * std::cos(2.0 * kPi * k / (K - 1)) + 0.08 * std::cos(4.0 * kPi * k / (K - 1))
                                 : 1.0;
        h[k] = 2.0 * fc * sinc * win;
        sum += h[k];
    }
    for (auto &v : h) v /= sum;
    return h;
}

struct Regular {
    bool ok = false;
    int nx = 0, ny = 0;
    double x0 = 0, y0 = 0, px = 0, py = 0;
};

// Detects elements on a row-major grid: e = iy * nx + ix, x = x0 + ix px, y = y0 + iy py.
Regular detect_regular(int n, const double *p) {
    Regular r;
    int nx = 1;
    while (nx < n && std::fabs(p[3 * nx + 1] - p[1]) <= 1e-12) ++nx;
    if (n % nx) return r;
    const int ny = n / nx;
    const double px = nx > 1 ? p[3] - p[0] : 0.0;
    const double py = ny > 1 ? p[3 * nx + 1] - p[1] : 0.0;
    if ((nx > 1 && !(px > 0)) || (ny > 1 && !(py > 0))) return r;
    const double tol = 1e-9 + 1e-6 * std::max(px, py);
    for (int e = 0; e < n; ++e) {
        const int ix = e % nx, iy = e / nx;
        if (std::fabs(p[3 * e] - (p[0] + ix * px)) > tol || std::fabs(p[3 * e + 1] - (p[1] + iy * py)) > tol) return r;
    }
    r.ok = true;
    r.nx = nx;
    r.ny = ny;
    r.x0 = p[0];
    r.y0 = p[1];
    r.px = px;
    r.py = py;
    return r;
}

// index range of grid nodes x0 + k p (k in [0, n)) within [lo, hi], widened by `margin` nodes
void node_range(double lo, double hi, double x0, double p, int n, int margin, int &a, int &b) {
    if (n == 1 || p <= 0) {
        a = 0;
        b = 0;
        return;
    }
    a = (int)std::ceil((lo - x0) / p - 1e-9) - margin;
    b = (int)std::floor((hi - x0) / p + 1e-9) + margin;
    a = std::max(a, 0);
    b = std::min(b, n - 1);
    if (a > b) {  // nothing inside: keep one node so the box is well formed
        a = std::min(std::max(a, 0), n - 1);
        b = a;
    }
}

// number of nodes x0 + k p, k in [0, n), with |x - q| <= a
long long count_nodes(double q, double a, double x0, double p, int n) {
    if (n == 1 || p <= 0) return std::fabs(x0 - q) <= a ? 1 : 0;
    long long lo = (long long)std::ceil((q - a - x0) / p);
    long long hi = (long long)std::floor((q + a - x0) / p);
    lo = std::max(lo, 0LL);
    hi = std::min(hi, (long long)n - 1);
    return hi >= lo ? hi - lo + 1 : 0;
}

int check_cuda(cudaError_t e) { return e == cudaSuccess ? SUPRA_OK : SUPRA_ECUDA; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// cuTensorMapEncodeTiled is a pure function of its arguments and takes host time on every call
// (a training step of one tile per CTA was host-bound on it): encoded maps are kept by their
// arguments.  A map holds only an address, sizes and strides, so a kept map is the same map for
// a freed and reallocated buffer at the same address.
struct MapKey {
    uintptr_t base;
    int dtype, rank, interleave, swizzle, l2, oob;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5];
    bool operator==(const MapKey &o) const { return std::memcmp(this, &o, sizeof(MapKey)) == 0; }
};
struct MapKeyHash {
    size_t operator()(const MapKey &k) const {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(&k);
        uint64_t h = 1469598103934665603ull;   // FNV-1a
        for (size_t i = 0; i < sizeof(MapKey); ++i) h = (h ^ b[i]) * 1099511628211ull;
        return (size_t)h;
    }
};
bool encode_map(CUtensorMap *map, CUtensorMapDataType dtype, int rank, const void *base, const cuuint64_t *dims,
                const cuuint64_t *strides, const cuuint32_t *box, const cuuint32_t *estr, CUtensorMapL2promotion l2) {
    if (rank < 1 || rank > 5) return false;
    MapKey k;
    std::memset(&k, 0, sizeof k);   // padding bytes too: keys compare as bytes
    k.base = reinterpret_cast<uintptr_t>(base);
    k.dtype = (int)dtype, k.rank = rank, k.interleave = (int)CU_TENSOR_MAP_INTERLEAVE_NONE;
    k.swizzle = (int)CU_TENSOR_MAP_SWIZZLE_NONE, k.l2 = (int)l2, k.oob = (int)CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE;
    for (int i = 0; i < rank; ++i) k.dims[i] = dims[i], k.box[i] = box[i], k.estr[i] = estr[i];
    for (int i = 0; i + 1 < rank; ++i) k.strides[i] = strides[i];
    static std::mutex mu;
    static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> kept;
    {
        std::lock_guard<std::mutex> g(mu);
        const auto it = kept.find(k);
        if (it != kept.end()) {
            *map = it->second;
            return true;
        }
    }
    EncodeTiledFn fn = encode_tiled();
    if (!fn || fn(map, dtype, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, l2,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    std::lock_guard<std::mutex> g(mu);
    if (kept.size() >= 16384) kept.clear();
    kept.emplace(k, *map);
    return true;
}

// 4D map over a group's records viewed as int32 sample pairs: (n_s / 2, n_el, n_tx, frames),
// box (W / 2, 1, 1, G); reads outside the records fill zeros.
bool make_frame_map(CUtensorMap *map, const void *base, long long frame_stride, int frames, const DevPlan &H,
                    int width, int G) {
    if ((reinterpret_cast<uintptr_t>(base) & 15) || frame_stride <= 0 || (frame_stride & 15)) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)H.n_s / 2, (cuuint64_t)H.n_el, (cuuint64_t)H.n_tx, (cuuint64_t)frames};
    const cuuint64_t strides[3] = {(cuuint64_t)H.n_s * 2, (cuuint64_t)H.n_s * 2 * H.n_el, (cuuint64_t)frame_stride};
    const cuuint32_t box[4] = {(cuuint32_t)width / 2, 1, 1, (cuuint32_t)G};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_INT32, 4, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_L2_PROMOTION_NONE);
}

// Multiprocessors of the current device (queried once per device).
int sm_count() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cached[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
    if (dev < kMaxDev) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    if (dev < kMaxDev) cached[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

// Depth segments per line for a launch of `items` lines whose shortest line has
// min_tiles depth tiles: a launch that leaves SMs idle (fewer lines than two
// resident CTAs per SM) splits its lines so that the segments still fit in one
// wave.  16-frame B-mode launches (the tensor-core FIR) keep whole lines.  A
// plan's depth_segments setting k >= 1 asks for k segments per line instead.
int depth_segments(int items, int min_tiles, int G, int mode, int setting = 0) {
    if (mode == 1 && G == 16) return 1;
    if (setting > 0) return std::max(1, std::min(setting, min_tiles));
    const int slots = 2 * sm_count();
    const int s = items > 0 ? slots / items : 1;
    return std::max(1, std::min(s, min_tiles));
}

// kernel choice for a frame group size
int group_template(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : 16; }

template <int G, int MODE, bool EXT, int MINB = 2, int SH = 0>
int launch_das_t(const LaunchGroups &L, cudaStream_t st) {
    // the shared-memory opt-in is set once per device (it outlives the call)
    constexpr int kMaxDev = 64;
    static std::atomic<int> ready[kMaxDev];
    const SmemLayout lay(G, MODE, kSlotSamples, SH);
    auto kern = das_kernel<G, MODE, EXT, MINB, SH>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SUPRA_ECUDA;
    if (dev >= kMaxDev || ready[dev].load(std::memory_order_acquire) == 0) {
        int max_optin = 0;
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (lay.total > max_optin) return SUPRA_EINVAL;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total) != cudaSuccess)
            return SUPRA_ECUDA;
        if (dev < kMaxDev) ready[dev].store(1, std::memory_order_release);
    }
    kern<<<L.total_lines * std::max(L.n_seg, 1), das_threads<G, MODE>(), lay.total, st>>>(L);
    return check_cuda(cudaGetLastError());
}

// Launch-level tile settings of a launch (those of its first frame's plan).
struct LaunchShape {
    int stage_shape = 0;   // 16-frame groups
    int ctas_per_sm = 0;   // one-frame launches: 0 = automatic, 2 or 3
};

template <bool EXT>
int launch_das_c(int G, int mode, const LaunchGroups &L, const LaunchShape &S, cudaStream_t st) {
    if (G == 1) {
        // one frame per CTA: three resident CTAs per SM (fewer registers) when the launch has
        // work for them, e.g. the many lines of a volume; two otherwise, so that a launch of
        // fewer CTAs than three per SM still spreads over all SMs
        const bool three = S.ctas_per_sm ? S.ctas_per_sm == 3
                                         : (long long)L.total_lines * std::max(L.n_seg, 1) >= 3LL * sm_count();
        if (three) return mode == 0 ? launch_das_t<1, 0, EXT, 3>(L, st) : launch_das_t<1, 1, EXT, 3>(L, st);
        return mode == 0 ? launch_das_t<1, 0, EXT>(L, st) : launch_das_t<1, 1, EXT>(L, st);
    }
    if (mode == 0) return SUPRA_EINVAL;
    switch (G) {
        case 2: return launch_das_t<2, 1, EXT>(L, st);
        case 4: return launch_das_t<4, 1, EXT>(L, st);
        case 8: return launch_das_t<8, 1, EXT>(L, st);
        default:
            return S.stage_shape == 1 ? launch_das_t<16, 1, EXT, 2, 1>(L, st) : launch_das_t<16, 1, EXT>(L, st);
    }
}

// ext: the groups' plans use an extended transmit model (plane waves and/or
// compounding several transmits per line).  They run their own kernel
// instantiation, so plans with spherical single transmits keep the plain code.
int launch_das(int G, int mode, bool ext, const LaunchGroups &L, const LaunchShape &S, cudaStream_t st) {
    if (L.total_lines == 0) return SUPRA_OK;
    return ext ? launch_das_c<true>(G, mode, L, S, st) : launch_das_c<false>(G, mode, L, S, st);
}

// Frames of one scan-conversion launch and their host-side plan records (grid sizing).
struct ScanBatch {
    ScanLaunch launch{};
    const DevPlan *host[kMaxScanFrames] = {};
    void add(const supra_plan *p, const uint8_t *bm, uint8_t *img);
};

int launch_scan(const ScanBatch &S, cudaStream_t st) {
    if (S.launch.n == 0) return SUPRA_OK;
    const int sms = sm_count();
    // linear layouts go to the separable kernel, the others to the tiled one
    ScanLaunch lin{}, gen{};
    long long lin_blocks = 1, gen_tiles = 1;
    for (int k = 0; k < S.launch.n; ++k) {
        const DevPlan &H = *S.host[k];
        if (H.geometry == SUPRA_GEOM_LINEAR) {
            // consecutive frames of one plan share a CTA (up to kScanGroup)
            const int g = lin.n_groups - 1;
            if (g >= 0 && lin.gn[g] < kScanGroup && lin.f[lin.n - 1].plan == S.launch.f[k].plan) {
                ++lin.gn[g];
            } else {
                lin.g0[lin.n_groups] = (short)lin.n;
                lin.gn[lin.n_groups++] = 1;
            }
            lin.f[lin.n++] = S.launch.f[k];
            lin_blocks = std::max(lin_blocks, (long long)((H.gnx + 31) / 32) * ((H.gnz + 63) / 64));
        } else {
            gen.f[gen.n++] = S.launch.f[k];
            const bool is3d = H.geometry == SUPRA_GEOM_PYRAMID;
            const int TX = is3d ? 16 : 64, TY = is3d ? 16 : 1, TZ = is3d ? 8 : 32;
            gen_tiles = std::max(gen_tiles, (long long)((H.gnx + TX - 1) / TX) * ((H.gny + TY - 1) / TY) *
                                                ((H.gnz + TZ - 1) / TZ));
        }
    }
    if (lin.n) {
        // every CTA of the largest frame; smaller frames' extra CTAs return at once
        if (lin_blocks > 0x7fffffffLL) return SUPRA_EINVAL;
        scanconvert_linear_kernel<<<dim3((unsigned)lin_blocks, lin.n_groups), 256, 0, st>>>(lin);
        const int rc = check_cuda(cudaGetLastError());
        if (rc) return rc;
    }
    if (gen.n) {
        const int per_frame = (int)std::max(1LL, std::min(gen_tiles, (long long)(sms * 16 + gen.n - 1) / gen.n));
        scanconvert_kernel<<<dim3(per_frame, gen.n), 256, 0, st>>>(gen);
        return check_cuda(cudaGetLastError());
    }
    return SUPRA_OK;
}

void ScanBatch::add(const supra_plan *p, const uint8_t *bm, uint8_t *img) {
    host[launch.n] = &p->host;
    launch.f[launch.n++] = ScanFrame{p->dev, bm, img};
}

// One CTA, 96 threads: two waits on an mbarrier that never completes (see
// supra_selftest_bounded_wait).
__global__ void __launch_bounds__(96) bounded_wait_selftest_kernel(long long budget, int *out) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_word;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_word = 0;
        fence_mbar_init();
    }
    __syncthreads();
    volatile int *abort_flag = &abort_word;
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait_bounded(&bar, 0u, budget);
        out[0] = ok ? 0 : 1;
        if (!ok) set_status(SUPRA_ETIMEOUT);
    } else if (threadIdx.x == 32) {
        const bool ok = wait_phase(&bar, 0u, abort_flag);
        out[1] = ok ? 0 : 1;
        if (!ok) set_status(SUPRA_ETIMEOUT);
    } else if (threadIdx.x == 64) {
        const long long t0 = clock64();
        while (clock64() - t0 <= budget) {
        }
        *abort_flag = 1;
    }
}

__device__ int g_selftest[2];

}  // namespace

// ---------------------------------------------------------------- learned-apodization launch helpers

static int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The feature rows of a training launch as a 3D tensor map for the kernel's prefetch by the
// copy engine: (feature within an 8-feature chunk, virtual row, chunk), where virtual row v is
// row v * stride of feat (tiles start at multiples of stride), up to the last pixel's row (rows
// past it read the zero fill).  A box of 8 x 128 x 16 lands as the kernel's chunked layout
// (chunk j of row r at j * 2048 + r * 16 bytes).  Leaves rows_tma 0 (per-thread copies) when
// the rows do not fit that form.
static void set_rows_map(apod::Args &a, CUtensorMap &map) {
    a.rows_tma = 0;
    if (a.n < 1 || a.stride < 1 || a.tile_stride < 1 || a.tile_stride % a.stride ||
        (reinterpret_cast<uintptr_t>(a.feat) & 15))
        return;
    const long long last = a.n - 1;
    const long long vmax = ((last / apod::kTile) * a.tile_stride + (last % apod::kTile) * a.stride) / a.stride;
    if (vmax >= (1LL << 31) - apod::kTile) return;   // the kernel's row coordinates are int32
    const cuuint64_t dims[3] = {8, (cuuint64_t)(vmax + 1), (cuuint64_t)apod::kIn / 8};
    const cuuint64_t strides[2] = {(cuuint64_t)a.stride * apod::kIn * 2, 16};
    const cuuint32_t box[3] = {8, (cuuint32_t)apod::kTile, (cuuint32_t)apod::kIn / 8};
    const cuuint32_t estr[3] = {1, 1, 1};
    a.rows_tma = encode_map(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, a.feat, dims, strides, box, estr,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B);
}

template <int MODE>
static int launch_apod(const apod::Args &a0, long long n_tiles, int per_sm, cudaStream_t st, int *grid_out = nullptr) {
    const int sms = device_sms();
    if (sms <= 0) return SUPRA_ECUDA;
    const int grid = (int)std::min<long long>(n_tiles, (long long)sms * per_sm);
    if (grid_out) *grid_out = grid;
    const int smem = apod::Smem<MODE>::TOTAL;
    if (cudaFuncSetAttribute(apod::apod_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return SUPRA_ECUDA;
    apod::Args a = a0;
    CUtensorMap map;
    std::memset(&map, 0, sizeof map);
    if (MODE == apod::kTrain) set_rows_map(a, map);
    apod::apod_kernel<MODE><<<grid, apod::apod_threads<MODE>(), smem, st>>>(a, map);
    return check_cuda(cudaGetLastError());
}

extern "C" {

const char *supra_version(void) { return "supra-b300 0.1 (sm_103a)"; }

const char *supra_strerror(int code) {
    switch (code) {
        case SUPRA_OK: return "ok";
        case SUPRA_EINVAL: return "invalid argument";
        case SUPRA_ENOMEM: return "out of memory";
        case SUPRA_ECUDA: return "CUDA runtime error";
        case SUPRA_ETIMEOUT: return "bounded device wait ran out";
        case SUPRA_EINTERNAL: return "internal consistency check failed";
        case SUPRA_EWORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown error";
    }
}

int supra_plan_create(const supra_probe *probe, const supra_scan *scan, const supra_rx *rx, const supra_post *post,
                      const supra_grid *grid, supra_plan **out) {
    if (!out) return SUPRA_EINVAL;
    *out = nullptr;
    if (!probe || !scan || !rx || !post) return SUPRA_EINVAL;
    const int n_el = probe->n_el, n_tx = scan->n_tx, n_lines = scan->n_lines, n_d = scan->n_depth,
              n_s = rx->n_samples;
    if (n_el < 1 || n_tx < 1 || n_lines < 1 || n_d < 1 || n_s < 1) return SUPRA_EINVAL;
    if (n_el > 65536 || n_d > (1 << 24) || n_s > (1 << 24)) return SUPRA_EINVAL;
    if (!probe->elem_pos || !scan->tx_origin || !scan->line_origin || !scan->line_dir || !scan->line_tx)
        return SUPRA_EINVAL;
    if (!finite_pos(rx->c) || !finite_pos(rx->fs) || !finite_pos(rx->fc) || !(rx->fc < rx->fs / 2) ||
        !finite_pos(rx->fnumber) || !finite_pos(rx->min_half_aperture) ||
        !std::isfinite(rx->t0))
        return SUPRA_EINVAL;
    if (rx->window < SUPRA_WINDOW_RECT || rx->window > SUPRA_WINDOW_HAMMING) return SUPRA_EINVAL;
    if (!(scan->depth0 >= 0) || !finite_pos(scan->depth_step) || !std::isfinite(scan->depth0)) return SUPRA_EINVAL;
    if (post->fir_taps < 1 || post->fir_taps > kMaxTaps || (post->fir_taps % 2) == 0) return SUPRA_EINVAL;
    if (!finite_pos(post->fir_cutoff) || !finite_pos(post->dyn_range_db) || !finite_pos(post->log_ref))
        return SUPRA_EINVAL;
    const int n_bands = post->n_bands <= 1 ? 1 : post->n_bands;
    if (n_bands > kMaxBands || (n_bands > 1 && !(std::isfinite(post->band_step) && post->band_step >= 0.0)))
        return SUPRA_EINVAL;
    for (int e = 0; e < 3 * n_el; ++e)
        if (!std::isfinite(probe->elem_pos[e])) return SUPRA_EINVAL;
    for (int t = 0; t < 3 * n_tx; ++t)
        if (!std::isfinite(scan->tx_origin[t]) || (scan->tx_dir && !std::isfinite(scan->tx_dir[t])))
            return SUPRA_EINVAL;
    if (scan->compound != 0 && scan->compound != 1) return SUPRA_EINVAL;
    if (scan->compound && n_tx > 4096) return SUPRA_EINVAL;   // transmit index in the stage metadata
    for (int l = 0; l < n_lines; ++l) {
        const double *d = scan->line_dir + 3 * l;
        const double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!std::isfinite(nn) || std::fabs(nn - 1.0) > 1e-6) return SUPRA_EINVAL;
        if (scan->line_tx[l] < 0 || scan->line_tx[l] >= n_tx) return SUPRA_EINVAL;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(scan->line_origin[3 * l + k])) return SUPRA_EINVAL;
    }
    const double depth_rate = rx->c / (2.0 * scan->depth_step);   // samples per second of the depth axis
    if (!(post->fir_cutoff < depth_rate / 2)) return SUPRA_EINVAL;

    // ---- scan conversion layout
    DevPlan H{};
    H.has_grid = grid != nullptr;
    H.geometry = scan->geometry;
    H.lines_x = scan->lines_x;
    H.lines_y = scan->lines_y;
    if (grid) {
        if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return SUPRA_EINVAL;
        if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 34)) return SUPRA_EINVAL;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(grid->origin[k]) || !std::isfinite(grid->spacing[k])) return SUPRA_EINVAL;
        if (scan->lines_x < 2 || scan->lines_y < 1 || (long long)scan->lines_x * scan->lines_y != n_lines || n_d < 2)
            return SUPRA_EINVAL;
        const double *lo = scan->line_origin, *ld = scan->line_dir;
        const double tol = 1e-6;
        H.gnx = grid->nx;
        H.gny = grid->ny;
        H.gnz = grid->nz;
        H.gox = (float)grid->origin[0];
        H.goy = (float)grid->origin[1];
        H.goz = (float)grid->origin[2];
        H.gsx = (float)grid->spacing[0];
        H.gsy = (float)grid->spacing[1];
        H.gsz = (float)grid->spacing[2];
        H.v0 = (float)scan->depth0;
        H.dv_inv = (float)(1.0 / scan->depth_step);
        if (scan->geometry == SUPRA_GEOM_LINEAR) {
            if (scan->lines_y != 1) return SUPRA_EINVAL;
            const double x0 = lo[0], x1 = lo[3 * (n_lines - 1)];
            const double dx = (x1 - x0) / (n_lines - 1);
            if (!(dx > 0)) return SUPRA_EINVAL;
            for (int l = 0; l < n_lines; ++l) {
                if (std::fabs(lo[3 * l] - (x0 + l * dx)) > tol * (std::fabs(dx) + 1e-6) + 1e-12) return SUPRA_EINVAL;
                if (std::fabs(lo[3 * l + 1] - lo[1]) > 1e-12 || std::fabs(lo[3 * l + 2] - lo[2]) > 1e-12)
                    return SUPRA_EINVAL;
                if (std::fabs(ld[3 * l + 2] - 1.0) > 1e-9) return SUPRA_EINVAL;
            }
            H.apx = 0;
            H.apy = 0;
            H.apz = (float)lo[2];
            H.u0 = (float)x0;
            H.du_inv = (float)(1.0 / dx);
        } else if (scan->geometry == SUPRA_GEOM_SECTOR) {
            if (scan->lines_y != 1) return SUPRA_EINVAL;
            std::vector<double> th(n_lines);
            for (int l = 0; l < n_lines; ++l) {
                for (int k = 0; k < 3; ++k)
                    if (std::fabs(lo[3 * l + k] - lo[k]) > 1e-12) return SUPRA_EINVAL;
                if (std::fabs(ld[3 * l + 1]) > 1e-9) return SUPRA_EINVAL;
                th[l] = std::atan2(ld[3 * l], ld[3 * l + 2]);
            }
            const double dth = (th[n_lines - 1] - th[0]) / (n_lines - 1);
            if (!(dth > 0)) return SUPRA_EINVAL;
            for (int l = 0; l < n_lines; ++l)
                if (std::fabs(th[l] - (th[0] + l * dth)) > tol * dth) return SUPRA_EINVAL;
            H.apx = (float)lo[0];
            H.apy = (float)lo[1];
            H.apz = (float)lo[2];
            H.u0 = (float)th[0];
            H.du_inv = (float)(1.0 / dth);
        } else if (scan->geometry == SUPRA_GEOM_PYRAMID) {
            const int nlx = scan->lines_x, nly = scan->lines_y;
            if (nly < 2) return SUPRA_EINVAL;
            std::vector<double> tx(nlx), ty(nly);
            for (int l = 0; l < n_lines; ++l) {
                for (int k = 0; k < 3; ++k)
                    if (std::fabs(lo[3 * l + k] - lo[k]) > 1e-12) return SUPRA_EINVAL;
                if (!(ld[3 * l + 2] > 0)) return SUPRA_EINVAL;
            }
            for (int ix = 0; ix < nlx; ++ix) tx[ix] = std::atan(ld[3 * ix] / ld[3 * ix + 2]);
            for (int iy = 0; iy < nly; ++iy) ty[iy] = std::atan(ld[3 * iy * nlx + 1] / ld[3 * iy * nlx + 2]);
            const double dtx = (tx[nlx - 1] - tx[0]) / (nlx - 1), dty = (ty[nly - 1] - ty[0]) / (nly - 1);
            if (!(dtx > 0) || !(dty > 0)) return SUPRA_EINVAL;
            for (int l = 0; l < n_lines; ++l) {
                const int ix = l % nlx, iy = l / nlx;
                const double a = std::atan(ld[3 * l] / ld[3 * l + 2]), b = std::atan(ld[3 * l + 1] / ld[3 * l + 2]);
                if (std::fabs(a - (tx[0] + ix * dtx)) > tol * dtx || std::fabs(b - (ty[0] + iy * dty)) > tol * dty)
                    return SUPRA_EINVAL;
            }
            H.apx = (float)lo[0];
            H.apy = (float)lo[1];
            H.apz = (float)lo[2];
            H.u0 = (float)tx[0];
            H.du_inv = (float)(1.0 / dtx);
            H.w0 = (float)ty[0];
            H.dw_inv = (float)(1.0 / dty);
        } else {
            return SUPRA_EINVAL;
        }
    }

    // ---- receive geometry
    H.n_el = n_el;
    H.n_tx = n_tx;
    H.n_lines = n_lines;
    H.n_depth = n_d;
    H.n_s = n_s;
    H.n_tiles = (n_d + kDepthTile - 1) / kDepthTile;
    H.window = rx->window;
    H.win_a = rx->window == SUPRA_WINDOW_HANN ? 0.5f : rx->window == SUPRA_WINDOW_HAMMING ? 0.54f : 1.0f;
    H.win_b = rx->window == SUPRA_WINDOW_HANN ? 0.5f : rx->window == SUPRA_WINDOW_HAMMING ? 0.46f : 0.0f;
    H.bulk_ok = (n_s % 8) == 0;
    const double fsc = rx->fs / rx->c;
    const double a1 = 2.0 * scan->depth_step * fsc;
    if (a1 > 2.0 + 1e-9) return SUPRA_EINVAL;  // depth steps coarser than c / fs: no staging row fits
    H.fsc = (float)fsc;
    H.a1 = (float)a1;
    H.t0fs = (float)(rx->t0 * rx->fs);
    H.depth0 = (float)scan->depth0;
    H.depth_step = (float)scan->depth_step;
    H.inv2f = (float)(1.0 / (2.0 * rx->fnumber));
    H.amin = (float)rx->min_half_aperture;
    H.win_row = kSlotSamples;
    double ext[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
    for (int e = 0; e < n_el; ++e) {
        ext[0] = std::min(ext[0], probe->elem_pos[3 * e]);
        ext[1] = std::max(ext[1], probe->elem_pos[3 * e]);
        ext[2] = std::min(ext[2], probe->elem_pos[3 * e + 1]);
        ext[3] = std::max(ext[3], probe->elem_pos[3 * e + 1]);
    }
    H.xmin = (float)ext[0];
    H.xmax = (float)ext[1];
    H.ymin = (float)ext[2];
    H.ymax = (float)ext[3];
    const Regular reg = detect_regular(n_el, probe->elem_pos);
    if (reg.ok && (reg.nx > 32767 || reg.ny > 32767)) return SUPRA_EINVAL;   // element boxes are int16
    H.regular = reg.ok;
    H.el_nx = reg.ok ? reg.nx : n_el;
    H.el_ny = reg.ok ? reg.ny : 1;

    // host tables
    std::vector<float4> elem(n_el);
    for (int e = 0; e < n_el; ++e)
        elem[e] = make_float4((float)probe->elem_pos[3 * e], (float)probe->elem_pos[3 * e + 1],
                              (float)probe->elem_pos[3 * e + 2], 0.f);
    H.row_y = reg.ok;
    for (int e = 0; e < n_el && H.row_y; ++e) H.row_y = elem[e].y == elem[e - e % H.el_nx].y;
    // transmit terms of a (line, transmit) pair: spherical (b = d.(o_l - o_t), g = |o_l - o_t|^2)
    // or plane wave (b = n.(o_l - o_t), g = n.d - 1)
    auto tx_term = [&](int l, int t) {
        const double *o = scan->line_origin + 3 * l, *d = scan->line_dir + 3 * l;
        const double *ot = scan->tx_origin + 3 * t;
        const double m0 = o[0] - ot[0], m1 = o[1] - ot[1], m2 = o[2] - ot[2];
        TxTerm tt{};
        tt.tx = t;
        const double *n = scan->tx_dir ? scan->tx_dir + 3 * t : nullptr;
        const double nl = n ? std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]) : 0.0;
        if (nl > 0.0) {
            const double n0 = n[0] / nl, n1 = n[1] / nl, n2 = n[2] / nl;
            tt.plane = 1;
            tt.b = (float)(n0 * m0 + n1 * m1 + n2 * m2);
            tt.g = (float)(n0 * d[0] + n1 * d[1] + n2 * d[2] - 1.0);
        } else {
            tt.b = (float)(d[0] * m0 + d[1] * m1 + d[2] * m2);
            tt.g = (float)(m0 * m0 + m1 * m1 + m2 * m2);
        }
        return tt;
    };
    const int n_comp = scan->compound ? n_tx : 1;
    H.n_comp = n_comp;
    std::vector<LineGeo> lines(n_lines);
    std::vector<TxTerm> txterms(n_comp > 1 ? (size_t)n_lines * n_comp : 0);
    for (int l = 0; l < n_lines; ++l) {
        const double *o = scan->line_origin + 3 * l, *d = scan->line_dir + 3 * l;
        LineGeo g{};
        g.ox = (float)o[0];
        g.oy = (float)o[1];
        g.oz = (float)o[2];
        g.dx = (float)d[0];
        g.dy = (float)d[1];
        g.dz = (float)d[2];
        const TxTerm own = tx_term(l, n_comp > 1 ? 0 : scan->line_tx[l]);
        g.bt = own.b;
        g.gt = own.g;
        g.tx = own.tx;
        g.plane = own.plane;
        lines[l] = g;
        for (int t = 0; t < (n_comp > 1 ? n_comp : 0); ++t) txterms[(size_t)l * n_comp + t] = tx_term(l, t);
    }
    const int NT = H.n_tiles;
    std::vector<int> tile_k(NT);
    std::vector<float> tile_f(NT);
    const double A0 = (2.0 * scan->depth0 / rx->c - rx->t0) * rx->fs;
    for (int t = 0; t < NT; ++t) {
        const double v = A0 + a1 * (double)t * kDepthTile;
        const double k = std::floor(v);
        tile_k[t] = (int)k;
        tile_f[t] = (float)(v - k);
    }
    // per (line, tile) element box and the count of in-aperture element-samples
    std::vector<short4> box((size_t)n_lines * NT);
    long long ap_count = 0;
    {
        const double F2 = 2.0 * rx->fnumber;
        for (int l = 0; l < n_lines; ++l) {
            const double *o = scan->line_origin + 3 * l, *d = scan->line_dir + 3 * l;
            for (int t = 0; t < NT; ++t) {
                int bx0 = 1 << 30, bx1 = -1, by0 = 1 << 30, by1 = -1;
                for (int i = t * kDepthTile; i < std::min(n_d, (t + 1) * kDepthTile); ++i) {
                    const double r = scan->depth0 + i * scan->depth_step;
                    const double p0 = o[0] + r * d[0], p1 = o[1] + r * d[1], p2 = o[2] + r * d[2];
                    const double qx = std::min(std::max(p0, ext[0]), ext[1]);
                    const double qy = std::min(std::max(p1, ext[2]), ext[3]);
                    const double a = std::max(p2 / F2, rx->min_half_aperture);
                    if (reg.ok) {
                        int a0, a1i, b0, b1;
                        node_range(qx - a, qx + a, reg.x0, reg.px, reg.nx, 1, a0, a1i);
                        node_range(qy - a, qy + a, reg.y0, reg.py, reg.ny, 1, b0, b1);
                        bx0 = std::min(bx0, a0);
                        bx1 = std::max(bx1, a1i);
                        by0 = std::min(by0, b0);
                        by1 = std::max(by1, b1);
                        ap_count += count_nodes(qx, a, reg.x0, reg.px, reg.nx) * count_nodes(qy, a, reg.y0, reg.py, reg.ny);
                    } else {
                        for (int e = 0; e < n_el; ++e) {
                            const double *x = probe->elem_pos + 3 * e;
                            if (std::fabs(x[0] - qx) <= a && std::fabs(x[1] - qy) <= a) ++ap_count;
                        }
                    }
                }
                if (!reg.ok) {
                    bx0 = 0;
                    bx1 = n_el - 1;
                    by0 = 0;
                    by1 = 0;
                }
                box[(size_t)l * NT + t] = make_short4((short)bx0, (short)bx1, (short)by0, (short)by1);
            }
        }
    }
    if (!reg.ok && n_el > 32767) return SUPRA_EINVAL;
    // lines by decreasing beamforming work, so the heaviest CTAs start first
    std::vector<int> line_order(n_lines);
    {
        std::vector<long long> cost(n_lines, 0);
        for (int l = 0; l < n_lines; ++l)
            for (int t = 0; t < NT; ++t) {
                const short4 bb = box[(size_t)l * NT + t];
                cost[l] += (long long)(bb.y - bb.x + 1) * (bb.w - bb.z + 1);
            }
        for (int l = 0; l < n_lines; ++l) line_order[l] = l;
        std::stable_sort(line_order.begin(), line_order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    }

    // ---- envelope + log compression
    const int K = post->fir_taps;
    H.taps = K;
    {
        const auto h = lowpass_taps(K, post->fir_cutoff, depth_rate);
        const double w = 2.0 * kPi * rx->fc / depth_rate;
        const int Hh = (K - 1) / 2;
        for (int k = 0; k < kTapSlots; ++k) H.taps_c[k] = H.taps_s[k] = 0.0f;
        for (int k = 0; k < K; ++k) {
            const int kp = k + (kMaxTaps - 1) / 2 - Hh;   // centred slot
            H.taps_c[kp] = (float)(h[k] * std::cos(w * (k - Hh)));
            H.taps_s[kp] = (float)(h[k] * std::sin(w * (k - Hh)));
        }
        // frequency-compounding bank: band centres fc + (k - (K-1)/2) step, each in (0, rate/2)
        H.n_bands = n_bands;
        for (int b = 0; b < kMaxBands; ++b)
            for (int k = 0; k < kTapSlots; ++k) H.bank_c[b][k] = H.bank_s[b][k] = 0.0f;
        for (int b = 0; b < n_bands; ++b) {
            const double fk = rx->fc + (b - (n_bands - 1) / 2.0) * (n_bands > 1 ? post->band_step : 0.0);
            if (!(fk > 0.0 && fk < depth_rate / 2)) return SUPRA_EINVAL;
            const double wk = 2.0 * kPi * fk / depth_rate;
            for (int k = 0; k < K; ++k) {
                const int kp = k + (kMaxTaps - 1) / 2 - Hh;
                H.bank_c[b][kp] = (float)(h[k] * std::cos(wk * (k - Hh)));
                H.bank_s[b][kp] = (float)(h[k] * std::sin(wk * (k - Hh)));
            }
        }
        const double D = post->dyn_range_db;
        const double la = 255.0 / D * 20.0 * std::log10(2.0);
        const double lb = 255.0 / D * (D - 20.0 * std::log10(post->log_ref)) + 0.5;
        H.log_a = (float)la;
        H.log_b = (float)lb;
        // env = 2 sqrt(q): log2(env) = 1 + log2(q) / 2
        H.log_a2 = (float)(la / 2.0);
        H.log_b2 = (float)(la + lb);
    }

    // ---- device allocation: one blob for all tables
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = align_up(off, 256);
        off = o + bytes;
        return o;
    };
    const size_t o_plan = take(sizeof(DevPlan));
    const size_t o_elem = take(sizeof(float4) * n_el);
    const size_t o_lines = take(sizeof(LineGeo) * n_lines);
    const size_t o_tk = take(sizeof(int) * NT);
    const size_t o_tf = take(sizeof(float) * NT);
    const size_t o_box = take(sizeof(short4) * box.size());
    const size_t o_ord = take(sizeof(int) * n_lines);
    const size_t o_txt = take(sizeof(TxTerm) * std::max<size_t>(txterms.size(), 1));
    auto *plan = new (std::nothrow) supra_plan();
    if (!plan) return SUPRA_ENOMEM;
    cudaGetDevice(&plan->device);
    if (cudaMalloc(&plan->blob, off) != cudaSuccess) {
        delete plan;
        cudaGetLastError();
        return SUPRA_ENOMEM;
    }
    char *b = static_cast<char *>(plan->blob);
    H.elem = reinterpret_cast<const float4 *>(b + o_elem);
    H.lines = reinterpret_cast<const LineGeo *>(b + o_lines);
    H.tile_k = reinterpret_cast<const int *>(b + o_tk);
    H.tile_f = reinterpret_cast<const float *>(b + o_tf);
    H.ap_box = reinterpret_cast<const short4 *>(b + o_box);
    H.line_order = reinterpret_cast<const int *>(b + o_ord);
    H.txterms = reinterpret_cast<const TxTerm *>(b + o_txt);
    plan->dev = reinterpret_cast<DevPlan *>(b + o_plan);
    plan->host = H;
    plan->ext = n_comp > 1;
    for (int l = 0; l < n_lines && !plan->ext; ++l) plan->ext = lines[l].plane != 0;
    cudaError_t err = cudaSuccess;
    err = err ? err : cudaMemcpy(b + o_plan, &H, sizeof(DevPlan), cudaMemcpyHostToDevice);
    err = err ? err : cudaMemcpy(b + o_elem, elem.data(), sizeof(float4) * n_el, cudaMemcpyHostToDevice);
    err = err ? err : cudaMemcpy(b + o_lines, lines.data(), sizeof(LineGeo) * n_lines, cudaMemcpyHostToDevice);
    err = err ? err : cudaMemcpy(b + o_tk, tile_k.data(), sizeof(int) * NT, cudaMemcpyHostToDevice);
    err = err ? err : cudaMemcpy(b + o_tf, tile_f.data(), sizeof(float) * NT, cudaMemcpyHostToDevice);
    err = err ? err : cudaMemcpy(b + o_box, box.data(), sizeof(short4) * box.size(), cudaMemcpyHostToDevice);
    err = err ? err : cudaMemcpy(b + o_ord, line_order.data(), sizeof(int) * n_lines, cudaMemcpyHostToDevice);
    if (!txterms.empty())
        err = err ? err : cudaMemcpy(b + o_txt, txterms.data(), sizeof(TxTerm) * txterms.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaFree(plan->blob);
        delete plan;
        return SUPRA_ECUDA;
    }
    supra_plan_info &I = plan->info;
    I.n_tx = n_tx;
    I.n_el = n_el;
    I.n_samples = n_s;
    I.n_lines = n_lines;
    I.n_depth = n_d;
    I.channel_bytes = 2LL * n_tx * n_el * n_s;
    // with compounding every line reads its aperture from every transmit's records
    I.aperture_element_samples = ap_count * n_comp;
    I.aperture_bytes = 2 * ap_count * n_comp;
    I.rf_bytes = 4LL * n_lines * n_d;
    I.bmode_bytes = (long long)n_lines * n_d;
    I.image_bytes = grid ? (long long)grid->nx * grid->ny * grid->nz : I.bmode_bytes;
    I.has_grid = grid != nullptr;
    I.depth_tile = kDepthTile;
    for (const short4 &bb : box) plan->max_active = std::max(plan->max_active, (bb.y - bb.x + 1) * (bb.w - bb.z + 1));
    *out = plan;
    return SUPRA_OK;
}

void supra_plan_destroy(supra_plan *plan) {
    if (!plan) return;
    if (plan->blob) cudaFree(plan->blob);
    delete plan;
}

int supra_plan_get_info(const supra_plan *plan, supra_plan_info *info) {
    if (!plan || !info) return SUPRA_EINVAL;
    *info = plan->info;
    return SUPRA_OK;
}

int supra_beamform(const supra_plan *plan, const int16_t *ch, float *rf, void *stream) {
    if (!plan || !ch || !rf) return SUPRA_EINVAL;
    LaunchGroups L{};
    L.n_groups = 1;
    L.total_lines = plan->host.n_lines;
    L.g[0].plan = plan->dev;
    L.g[0].n = 1;
    L.g[0].line0 = 0;
    L.g[0].bulk = plan->host.bulk_ok && (reinterpret_cast<uintptr_t>(ch) & 15) == 0;
    L.g[0].ch[0] = ch;
    L.g[0].out[0] = rf;
    L.uniform = 1;
    L.n_seg = depth_segments(L.total_lines, plan->host.n_tiles, 1, 0, plan->depth_segments.load());
    LaunchShape S;
    S.ctas_per_sm = plan->ctas_per_sm.load();
    return launch_das(1, 0, plan->ext, L, S, static_cast<cudaStream_t>(stream));
}

int supra_envelope(const supra_plan *plan, const float *rf, float *env, void *stream) {
    if (!plan || !rf || !env || rf == env) return SUPRA_EINVAL;
    dim3 grid((plan->host.n_depth + kEnvTile - 1) / kEnvTile, plan->host.n_lines);
    envelope_kernel<<<grid, kEnvTile, 0, static_cast<cudaStream_t>(stream)>>>(plan->dev, rf, env);
    return check_cuda(cudaGetLastError());
}

int supra_logcompress(const supra_plan *plan, const float *env, uint8_t *bm, void *stream) {
    if (!plan || !env || !bm) return SUPRA_EINVAL;
    const long long n = (long long)plan->host.n_lines * plan->host.n_depth;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    logcompress_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(plan->dev, env, bm, n);
    return check_cuda(cudaGetLastError());
}

int supra_scanconvert(const supra_plan *plan, const uint8_t *bm, uint8_t *img, void *stream) {
    if (!plan || !bm || !img || !plan->host.has_grid) return SUPRA_EINVAL;
    ScanBatch S;
    S.add(plan, bm, img);
    return launch_scan(S, static_cast<cudaStream_t>(stream));
}

// Workspace of one frame in the batched chain: its log-compressed lines when it is
// scan-converted; frames of a compounding plan (n_bands > 1) run the unfused chain
// and also hold their RF and envelope lines.
static size_t frame_workspace(const supra_plan *p) {
    size_t b = p->host.has_grid ? align_up((size_t)p->info.bmode_bytes, 256) : 0;
    if (p->host.n_bands > 1) b += 2 * align_up((size_t)p->info.rf_bytes, 256);
    return b;
}

// The part of the workspace a batched chain cannot run without (the frames' workspaces).
static size_t min_workspace(int32_t n, const supra_plan *const *plans) {
    size_t total = 0;
    for (int k = 0; k < n; ++k)
        if (plans[k]) total += frame_workspace(plans[k]);
    return total;
}

// Boundary records a frame's one-frame launch with depth segments uses (its plan's setting,
// or the automatic split of a launch of its lines alone, which bounds that of any launch it
// shares): 128 RF samples per line and boundary.
static size_t frame_boundary_bytes(const supra_plan *p) {
    if (p->host.n_bands > 1) return 0;
    const int segs = depth_segments(p->host.n_lines, p->host.n_tiles, 1, 1, p->depth_segments.load());
    return segs > 1 ? (size_t)p->host.n_lines * (size_t)(segs - 1) * 2 * kHalo * sizeof(float) : 0;
}

size_t supra_bmode_workspace_size(int32_t n, const supra_plan *const *plans) {
    if (n < 1 || !plans) return 0;
    size_t bnd = 0;
    for (int k = 0; k < n; ++k)
        if (plans[k]) bnd += frame_boundary_bytes(plans[k]);
    const size_t need = min_workspace(n, plans);
    return bnd ? align_up(need, 256) + bnd : need;
}

int supra_bmode_batched(int32_t n, const supra_plan *const *plans, const int16_t *const *ch, uint8_t *const *out,
                        void *workspace, size_t workspace_bytes, void *stream) {
    if (n < 1 || !plans || !ch || !out) return SUPRA_EINVAL;
    for (int k = 0; k < n; ++k)
        if (!plans[k] || !ch[k] || !out[k]) return SUPRA_EINVAL;
    const size_t need = min_workspace(n, plans);
    if (need > 0 && (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)))
        return SUPRA_EWORKSPACE;
    // what the workspace holds beyond the frames' own parts takes the depth-segment boundary
    // records (launches run in stream order, so each launch reuses the region from its start)
    float *bnd_base = nullptr;
    size_t bnd_bytes = 0;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255) == 0 && workspace_bytes > align_up(need, 256)) {
        bnd_base = reinterpret_cast<float *>(static_cast<char *>(workspace) + align_up(need, 256));
        bnd_bytes = workspace_bytes - align_up(need, 256);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // log-compressed lines of scan-converted frames go to the workspace; frames of
    // compounding plans run beamform -> envelope (band bank) -> log compression there
    std::vector<uint8_t *> bm(n);
    {
        size_t off = 0;
        for (int k = 0; k < n; ++k) {
            char *w = static_cast<char *>(workspace) + off;
            if (plans[k]->host.has_grid) {
                bm[k] = reinterpret_cast<uint8_t *>(w);
                w += align_up((size_t)plans[k]->info.bmode_bytes, 256);
            } else {
                bm[k] = out[k];
            }
            if (plans[k]->host.n_bands > 1) {
                float *rf = reinterpret_cast<float *>(w);
                float *env = reinterpret_cast<float *>(w + align_up((size_t)plans[k]->info.rf_bytes, 256));
                int rc = supra_beamform(plans[k], ch[k], rf, stream);
                if (!rc) rc = supra_envelope(plans[k], rf, env, stream);
                if (!rc) rc = supra_logcompress(plans[k], env, bm[k], stream);
                if (rc) return rc;
            }
            off += frame_workspace(plans[k]);
        }
    }
    // Frames of one plan that are adjacent form groups of up to kMaxGroup; one launch
    // per group size class and row length, up to kMaxGroupsPerLaunch groups each.
    struct Grp {
        const supra_plan *p;
        int first, n;
    };
    std::vector<Grp> groups;
    for (int k = 0; k < n;) {
        if (plans[k]->host.n_bands > 1) {   // done above by the unfused chain
            ++k;
            continue;
        }
        Grp g{plans[k], k, 0};
        const int gmax = std::min(kMaxGroup, std::max(1, g.p->max_group.load(std::memory_order_relaxed)));
        while (k < n && plans[k] == g.p && g.n < gmax) {
            ++g.n;
            ++k;
        }
        groups.push_back(g);
    }
    // One launch per (group-size class, compounding, stage shape) that has groups; launch-level
    // settings (depth segments, CTAs per SM) come from the launch's first plan.
    auto shape_of = [](const Grp &gr, int Gc) { return Gc == 16 ? gr.p->stage_shape.load(std::memory_order_relaxed) : 0; };
    bool present[5][2][kStageShapes] = {};
    auto class_of = [](int Gc) { return Gc == 16 ? 0 : Gc == 8 ? 1 : Gc == 4 ? 2 : Gc == 2 ? 3 : 4; };
    for (const Grp &gr : groups) {
        const int Gc = group_template(gr.n);
        present[class_of(Gc)][gr.p->ext ? 1 : 0][shape_of(gr, Gc)] = true;
    }
    for (int Gc : {16, 8, 4, 2, 1}) {
        for (int comp = 0; comp < 2; ++comp) {
          for (int sh = 0; sh < kStageShapes; ++sh) {
            if (!present[class_of(Gc)][comp][sh]) continue;
            LaunchGroups L{};
            L.uniform = 1;
            int min_tiles = 1 << 30;
            const supra_plan *first = nullptr;
            auto flush = [&]() -> int {
                if (L.n_groups == 0) return SUPRA_OK;
                L.n_seg = depth_segments(L.total_lines, min_tiles, Gc, 1, first->depth_segments.load());
                LaunchShape S;
                S.stage_shape = sh;
                S.ctas_per_sm = first->ctas_per_sm.load();
                const size_t rec_floats =
                    L.n_seg > 1 ? (size_t)L.total_lines * Gc * (size_t)(L.n_seg - 1) * 2 * kHalo : 0;
                if (rec_floats > 0 && rec_floats * sizeof(float) <= bnd_bytes) {
                    L.bnd = bnd_base;
                    L.bnd_floats = (long long)rec_floats;
                }
                int rc = launch_das(Gc, 1, comp == 1, L, S, st);
                if (!rc && L.bnd) {
                    // a programmatic dependent: scheduled while the beamforming grid runs, it
                    // waits for that grid's completion on the device instead of a launch later
                    cudaLaunchConfig_t cfg{};
                    cfg.gridDim = dim3((unsigned)(L.total_lines * (L.n_seg - 1)));
                    cfg.blockDim = dim3(kBoundaryThreads);
                    cfg.stream = st;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    rc = check_cuda(cudaLaunchKernelEx(&cfg, boundary_fir_kernel, L, Gc));
                }
                L = LaunchGroups{};
                L.uniform = 1;
                min_tiles = 1 << 30;
                first = nullptr;
                return rc;
            };
            for (const Grp &gr : groups) {
                if (group_template(gr.n) != Gc || gr.p->ext != (comp == 1) || shape_of(gr, Gc) != sh) continue;
                if (!first) first = gr.p;
                FrameGroup &g = L.g[L.n_groups];
                g.plan = gr.p->dev;
                g.line0 = L.total_lines;
                g.n = gr.n;
                g.bulk = gr.p->host.bulk_ok;
                for (int f = 0; f < gr.n; ++f) {
                    if (reinterpret_cast<uintptr_t>(ch[gr.first + f]) & 15) g.bulk = 0;
                    g.ch[f] = ch[gr.first + f];
                    g.out[f] = bm[gr.first + f];
                }
                g.tma = 0;
                if (Gc >= 4 && g.bulk) {
                    // one tensor copy per element for all frames when they sit at a uniform stride
                    const char *b0 = reinterpret_cast<const char *>(ch[gr.first]);
                    const long long stride =
                        gr.n > 1 ? reinterpret_cast<const char *>(ch[gr.first + 1]) - b0 : (long long)gr.p->info.channel_bytes;
                    bool uni = stride > 0;
                    for (int f = 2; f < gr.n && uni; ++f)
                        uni = reinterpret_cast<const char *>(ch[gr.first + f]) - b0 == f * stride;
                    if (uni) {
                        g.tma = 1;
                        for (int w = 0; w < kNumWidths && g.tma; ++w)
                            g.tma = make_frame_map(&g.tmap[w], b0, stride, gr.n, gr.p->host, width_of(w), Gc) ? 1 : 0;
                    }
                }
                if (L.n_groups > 0 && L.g[0].plan != g.plan) L.uniform = 0;
                L.total_lines += gr.p->host.n_lines;
                min_tiles = std::min(min_tiles, gr.p->host.n_tiles);
                ++L.n_groups;
                if (L.n_groups == kMaxGroupsPerLaunch) {
                    const int rc = flush();
                    if (rc) return rc;
                }
            }
            const int rc = flush();
            if (rc) return rc;
          }
        }
    }
    // scan conversion of the frames with a grid
    ScanBatch S;
    for (int f = 0; f < n; ++f) {
        if (!plans[f]->host.has_grid) continue;
        S.add(plans[f], bm[f], out[f]);
        if (S.launch.n == kMaxScanFrames) {
            const int rc = launch_scan(S, st);
            if (rc) return rc;
            S.launch.n = 0;
        }
    }
    return launch_scan(S, st);
}

int supra_bmode(const supra_plan *plan, const int16_t *ch, uint8_t *out, void *workspace, size_t workspace_bytes,
                void *stream) {
    const supra_plan *p[1] = {plan};
    const int16_t *c[1] = {ch};
    uint8_t *o[1] = {out};
    if (!plan) return SUPRA_EINVAL;
    return supra_bmode_batched(1, p, c, o, workspace, workspace_bytes, stream);
}

int supra_mv(const supra_plan *plan, int32_t subaperture, float loading, const int16_t *ch, float *rf, void *stream) {
    if (!plan || !ch || !rf) return SUPRA_EINVAL;
    if (subaperture < 1 || subaperture > kMvMaxL || !(loading > 0.0f) || !std::isfinite(loading)) return SUPRA_EINVAL;
    if (plan->max_active > kMvMaxM || plan->host.n_comp > 1) return SUPRA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((double)subaperture / loading <= 1e4) {
        constexpr int w = mv_warps<float>();
        const dim3 grid((plan->host.n_depth + w - 1) / w, plan->host.n_lines);
        mv_kernel<float><<<grid, w * 32, 0, st>>>(plan->dev, ch, rf, subaperture, loading);
    } else {
        constexpr int w = mv_warps<double>();
        const dim3 grid((plan->host.n_depth + w - 1) / w, plan->host.n_lines);
        mv_kernel<double><<<grid, w * 32, 0, st>>>(plan->dev, ch, rf, subaperture, loading);
    }
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------- volume rendering

int supra_render(const supra_grid *grid, const uint8_t *vol, const supra_camera *cam, float *image, void *stream) {
    if (!grid || !vol || !cam || !image) return SUPRA_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || cam->width < 1 || cam->height < 1 || cam->n_steps < 0 ||
        (cam->mode != SUPRA_RENDER_MIP && cam->mode != SUPRA_RENDER_EA))
        return SUPRA_EINVAL;
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 40) || (long long)grid->nx * grid->ny > 0x7fffffffLL)
        return SUPRA_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!finite_pos(grid->spacing[k]) || !std::isfinite(grid->origin[k])) return SUPRA_EINVAL;
    const double dn = std::sqrt(cam->dir[0] * cam->dir[0] + cam->dir[1] * cam->dir[1] + cam->dir[2] * cam->dir[2]);
    if (!(dn > 0.0) || !std::isfinite(dn) || !std::isfinite(cam->t0) || !std::isfinite(cam->dt)) return SUPRA_EINVAL;
    if (cam->mode == SUPRA_RENDER_EA && !(cam->hi > cam->lo && std::isfinite(cam->alpha))) return SUPRA_EINVAL;
    RenderArgs a{};
    a.vol = vol;
    a.nx = grid->nx, a.ny = grid->ny, a.nz = grid->nz;
    double base[3], R[3], D[3], S[3];
    for (int k = 0; k < 3; ++k) {
        const double d = cam->dir[k] / dn;
        base[k] = (cam->centre[k] - 0.5 * (cam->width - 1) * cam->right[k] - 0.5 * (cam->height - 1) * cam->down[k] +
                   cam->t0 * d - grid->origin[k]) / grid->spacing[k];
        R[k] = cam->right[k] / grid->spacing[k];
        D[k] = cam->down[k] / grid->spacing[k];
        S[k] = cam->dt * d / grid->spacing[k];
        if (!std::isfinite(base[k]) || !std::isfinite(R[k]) || !std::isfinite(D[k])) return SUPRA_EINVAL;
    }
    a.bx = (float)base[0], a.by = (float)base[1], a.bz = (float)base[2];
    a.rx = (float)R[0], a.ry = (float)R[1], a.rz = (float)R[2];
    a.dx = (float)D[0], a.dy = (float)D[1], a.dz = (float)D[2];
    a.sx = (float)S[0], a.sy = (float)S[1], a.sz = (float)S[2];
    a.n_steps = cam->n_steps, a.W = cam->width, a.H = cam->height, a.mode = cam->mode;
    a.lo = (float)cam->lo;
    a.inv_range = cam->mode == SUPRA_RENDER_EA ? (float)(1.0 / (cam->hi - cam->lo)) : 0.0f;
    a.alpha = (float)cam->alpha;
    a.image = image;
    const dim3 grd((cam->width + kRenderTile - 1) / kRenderTile, (cam->height + kRenderTile - 1) / kRenderTile);
    render_kernel<<<grd, dim3(kRenderTile, kRenderTile), 0, static_cast<cudaStream_t>(stream)>>>(a);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------- tuning

int supra_plan_set_max_group(supra_plan *plan, int32_t g) {
    if (!plan || (g != 1 && g != 2 && g != 4 && g != 8 && g != 16)) return SUPRA_EINVAL;
    plan->max_group.store(g, std::memory_order_relaxed);
    return SUPRA_OK;
}

int32_t supra_plan_get_max_group(const supra_plan *plan) {
    return plan ? plan->max_group.load(std::memory_order_relaxed) : SUPRA_EINVAL;
}

int supra_plan_set_tile_shape(supra_plan *plan, const supra_tile_shape *s) {
    if (!plan || !s) return SUPRA_EINVAL;
    const int g = s->frames_per_group;
    if (g != 1 && g != 2 && g != 4 && g != 8 && g != 16) return SUPRA_EINVAL;
    int sh;
    if (s->elements_per_stage == 3 && s->stages == 3) sh = 0;
    else if (s->elements_per_stage == 2 && s->stages == 4) sh = 1;
    else return SUPRA_EINVAL;
    if (s->depth_segments < 0 || s->depth_segments > 64) return SUPRA_EINVAL;
    if (s->ctas_per_sm != 0 && s->ctas_per_sm != 2 && s->ctas_per_sm != 3) return SUPRA_EINVAL;
    plan->max_group.store(g);
    plan->stage_shape.store(sh);
    plan->depth_segments.store(s->depth_segments);
    plan->ctas_per_sm.store(s->ctas_per_sm);
    return SUPRA_OK;
}

int supra_plan_get_tile_shape(const supra_plan *plan, supra_tile_shape *s) {
    if (!plan || !s) return SUPRA_EINVAL;
    s->frames_per_group = plan->max_group.load();
    const int sh = plan->stage_shape.load();
    s->elements_per_stage = sh == 1 ? 2 : 3;
    s->stages = sh == 1 ? 4 : 3;
    s->depth_segments = plan->depth_segments.load();
    s->ctas_per_sm = plan->ctas_per_sm.load();
    return SUPRA_OK;
}

int supra_autotune_tile_shape(supra_plan *plan, int32_t n, const int16_t *const *ch, uint8_t *const *out,
                              void *workspace, size_t workspace_bytes, int32_t reps, void *stream,
                              supra_tile_shape *best_shape, float *best_ms, float *start_ms) {
    if (!plan || n < 1 || !ch || !out || reps < 1) return SUPRA_EINVAL;
    std::vector<const supra_plan *> plans(n, plan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    supra_tile_shape before{};
    supra_plan_get_tile_shape(plan, &before);
    // candidates: the shape in effect first (its time is start_ms), then every frames-per-group
    // class with the settings that class's launches use -- the stage shape for 16-frame groups,
    // depth segments for the others (0 = automatic, then 1 to 6 or 8 per line), resident CTAs
    // per SM for one-frame launches
    std::vector<supra_tile_shape> cand{before};
    for (int g : {16, 8, 4, 2, 1}) {
        if (g > 1 && g / 2 >= n) continue;   // same launches as a smaller class
        const bool tc = g == 16 && n > 8;     // 16-frame groups: whole lines, FIR on the tensor cores
        for (int sh = 0; sh < (tc ? kStageShapes : 1); ++sh)
            for (int seg : {0, 1, 2, 3, 4, 5, 6, 8}) {
                if (tc && seg) continue;
                for (int c : {0, 2, 3}) {
                    if (c && g != 1) continue;
                    cand.push_back({g, sh == 1 ? 2 : 3, sh == 1 ? 4 : 3, seg, c});
                }
            }
    }
    // Trials of shapes with more depth segments than the shape in effect need more boundary
    // records than a workspace sized for it holds: they run in a temporary workspace that
    // holds the largest (the outputs do not depend on the workspace).
    size_t trial_bytes = workspace_bytes;
    for (const supra_tile_shape &c : cand) {
        if (supra_plan_set_tile_shape(plan, &c)) continue;
        trial_bytes = std::max(trial_bytes, supra_bmode_workspace_size(n, plans.data()));
    }
    supra_plan_set_tile_shape(plan, &before);
    void *trial_ws = workspace;
    const bool own = trial_bytes > workspace_bytes;
    if (own && cudaMalloc(&trial_ws, trial_bytes) != cudaSuccess) return SUPRA_ENOMEM;
    auto release = [&]() {
        if (own) {
            cudaStreamSynchronize(st);
            cudaFree(trial_ws);
        }
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) {
        release();
        return SUPRA_ECUDA;
    }
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        release();
        return SUPRA_ECUDA;
    }
    workspace = trial_ws;
    workspace_bytes = trial_bytes;
    int rc = SUPRA_OK;
    supra_tile_shape best = before;
    float best_t = INFINITY, first_t = INFINITY;
    for (size_t c = 0; c < cand.size() && !rc; ++c) {
        rc = supra_plan_set_tile_shape(plan, &cand[c]);
        if (rc) break;
        rc = supra_bmode_batched(n, plans.data(), ch, out, workspace, workspace_bytes, stream);   // warm-up
        if (rc) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && !rc; ++r)
            rc = supra_bmode_batched(n, plans.data(), ch, out, workspace, workspace_bytes, stream);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = SUPRA_ECUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (c == 0) first_t = ms;
        if (ms < best_t) best_t = ms, best = cand[c];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    supra_plan_set_tile_shape(plan, rc ? &before : &best);
    if (rc) return rc;
    if (best_shape) *best_shape = best;
    if (best_ms) *best_ms = best_t;
    if (start_ms) *start_ms = first_t;
    return SUPRA_OK;
}

int supra_autotune_bmode(supra_plan *plan, int32_t n, const int16_t *const *ch, uint8_t *const *out, void *workspace,
                         size_t workspace_bytes, int32_t reps, void *stream, int32_t *best_group, float *best_ms) {
    supra_tile_shape s{};
    const int rc = supra_autotune_tile_shape(plan, n, ch, out, workspace, workspace_bytes, reps, stream, &s, best_ms,
                                             nullptr);
    if (rc) return rc;
    if (best_group) *best_group = s.frames_per_group;
    return SUPRA_OK;
}

// ---------------------------------------------------------------- learned apodization

size_t supra_apod_workspace_size(void) {
    return (size_t)std::max(device_sms(), 1) * apod::kPartStride * sizeof(float);
}

int supra_apod_features(const supra_plan *plan, const int16_t *ch, uint16_t *feat, uint32_t *mask, float *norm,
                        void *stream) {
    if (!plan || !ch || !feat || !mask || !norm) return SUPRA_EINVAL;
    if (plan->host.n_el > apod::kIn || plan->host.n_comp > 1 || !aligned16(feat) || !aligned16(mask))
        return SUPRA_EINVAL;
    const dim3 grid((plan->host.n_depth + 127) / 128, plan->host.n_lines);
    apod::features_kernel<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(plan->dev, ch, feat, mask, norm);
    return check_cuda(cudaGetLastError());
}

int supra_apod_forward(const float *params, int64_t n, int64_t stride, const uint16_t *feat, const uint32_t *mask,
                       const float *norm, float *y, void *stream) {
    if (!params || !feat || !mask || !norm || !y || n <= 0 || stride < 1) return SUPRA_EINVAL;
    if (!aligned16(feat) || !aligned16(mask)) return SUPRA_EINVAL;
    apod::Args a{};
    a.params = params, a.feat = feat, a.mask = mask, a.norm = norm, a.n = n, a.stride = stride, a.y = y;
    a.tile_stride = apod::kTile * stride;
    return launch_apod<apod::kForward>(a, (n + apod::kTile - 1) / apod::kTile, 2, static_cast<cudaStream_t>(stream));
}

int supra_apod_grad(const float *params, int64_t n, int64_t stride, const uint16_t *feat, const uint32_t *mask,
                    const float *norm, const float *label, float *grad, float *loss, void *workspace,
                    size_t workspace_bytes, void *stream) {
    if (!params || !feat || !mask || !norm || !label || !grad || !workspace || n <= 0 || stride < 1)
        return SUPRA_EINVAL;
    if (!aligned16(feat) || !aligned16(mask)) return SUPRA_EINVAL;
    const long long tiles = (n + apod::kTile - 1) / apod::kTile;
    const int sms = device_sms();
    if (sms <= 0) return SUPRA_ECUDA;
    const int grid = (int)std::min<long long>(tiles, sms);
    if (workspace_bytes < (size_t)grid * apod::kPartStride * sizeof(float)) return SUPRA_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    apod::Args a{};
    a.params = params, a.feat = feat, a.mask = mask, a.norm = norm, a.label = label, a.n = n, a.stride = stride;
    a.tile_stride = apod::kTile * stride;
    a.partial = static_cast<float *>(workspace);
    const int rc = launch_apod<apod::kTrain>(a, tiles, 1, st);
    if (rc != SUPRA_OK) return rc;
    apod::reduce_kernel<<<(apod::kParams + 1 + apod::kReduceCols - 1) / apod::kReduceCols,
                          apod::kReduceCols * apod::kReduceGroups, 0, st>>>(a.partial, grid, grad, loss);
    return check_cuda(cudaGetLastError());
}

static int apod_step_impl(float *params, float *m, float *v, int32_t step, float lr, float beta1, float beta2,
                          float eps, int64_t n, int64_t stride, int64_t tile_stride, const uint16_t *feat, const uint32_t *mask, const float *norm,
                    const float *label, float *grad, float *loss, void *workspace, size_t workspace_bytes,
                    void *stream) {
    if (!params || !m || !v || !feat || !mask || !norm || !label || !grad || !workspace || n <= 0 || stride < 1 ||
        step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return SUPRA_EINVAL;
    if (!aligned16(feat) || !aligned16(mask)) return SUPRA_EINVAL;
    const long long tiles = (n + apod::kTile - 1) / apod::kTile;
    const int sms = device_sms();
    if (sms <= 0) return SUPRA_ECUDA;
    const int grid = (int)std::min<long long>(tiles, sms);
    if (workspace_bytes < (size_t)grid * apod::kPartStride * sizeof(float)) return SUPRA_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    apod::Args a{};
    a.params = params, a.feat = feat, a.mask = mask, a.norm = norm, a.label = label, a.n = n, a.stride = stride;
    a.tile_stride = tile_stride;
    a.partial = static_cast<float *>(workspace);
    const int rc = launch_apod<apod::kTrain>(a, tiles, 1, st);
    if (rc != SUPRA_OK) return rc;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
    apod::reduce_adam_kernel<<<(apod::kParams + 1 + apod::kReduceCols - 1) / apod::kReduceCols,
                               apod::kReduceCols * apod::kReduceGroups, 0, st>>>(a.partial, grid, grad, loss, params, m,
                                                                                 v, lr, beta1, beta2, eps, c1, c2);
    return check_cuda(cudaGetLastError());
}

int supra_apod_step(float *params, float *m, float *v, int32_t step, float lr, float beta1, float beta2, float eps,
                    int64_t n, int64_t stride, const uint16_t *feat, const uint32_t *mask, const float *norm,
                    const float *label, float *grad, float *loss, void *workspace, size_t workspace_bytes,
                    void *stream) {
    return apod_step_impl(params, m, v, step, lr, beta1, beta2, eps, n, stride, apod::kTile * stride, feat, mask,
                          norm, label, grad, loss, workspace, workspace_bytes, stream);
}

int supra_apod_epoch(float *params, float *m, float *v, int32_t step0, float lr, float beta1, float beta2, float eps,
                     int64_t n_rows, int32_t n_batches, int32_t chunk, const int32_t *order, const uint16_t *feat,
                     const uint32_t *mask, const float *norm, const float *label, float *grad, float *losses,
                     void *workspace, size_t workspace_bytes, void *stream) {
    if (!order || !losses || n_batches < 1 || step0 < 0 || (chunk != 1 && chunk != apod::kTile)) return SUPRA_EINVAL;
    const int64_t n_chunks = (n_rows + chunk - 1) / chunk;   // the last one may be partial
    if (n_rows < 1 || n_chunks < n_batches) return SUPRA_EINVAL;
    for (int b = 0; b < n_batches; ++b)
        if (order[b] < 0 || order[b] >= n_batches) return SUPRA_EINVAL;
    for (int b = 0; b < n_batches; ++b) {
        const int64_t k = order[b];
        // chunks k, k + n_batches, ... of `chunk` consecutive rows; only the dataset's last chunk can be
        // partial, and it is then the minibatch's last
        const int64_t nc = (n_chunks - k + n_batches - 1) / n_batches;
        const int64_t last = k + (nc - 1) * n_batches;
        const int64_t n = (nc - 1) * chunk + std::min<int64_t>(chunk, n_rows - last * chunk);
        const int64_t r0 = k * chunk;
        const int rc = chunk == 1
                           ? supra_apod_step(params, m, v, step0 + b + 1, lr, beta1, beta2, eps, n, n_batches,
                                             feat + r0 * apod::kIn, mask + r0 * 4, norm + r0, label + r0, grad,
                                             losses + b, workspace, workspace_bytes, stream)
                           : apod_step_impl(params, m, v, step0 + b + 1, lr, beta1, beta2, eps, n, 1,
                                            (int64_t)n_batches * chunk, feat + r0 * apod::kIn, mask + r0 * 4,
                                            norm + r0, label + r0, grad, losses + b, workspace, workspace_bytes,
                                            stream);
        if (rc) return rc;
    }
    return SUPRA_OK;
}

int supra_apod_adam(float *params, float *m, float *v, const float *grad, int32_t step, float lr, float beta1,
                    float beta2, float eps, void *stream) {
    if (!params || !m || !v || !grad || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return SUPRA_EINVAL;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
    apod::adam_kernel<<<(apod::kParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        params, m, v, grad, apod::kParams, lr, beta1, beta2, eps, c1, c2);
    return check_cuda(cudaGetLastError());
}

int supra_apod_mlp(const supra_plan *plan, const float *params, const int16_t *ch, float *rf, void *stream) {
    if (!plan || !params || !ch || !rf) return SUPRA_EINVAL;
    if (plan->host.n_el > apod::kIn || plan->host.n_comp > 1) return SUPRA_EINVAL;
    apod::Args a{};
    a.params = params, a.plan = plan->dev, a.ch = ch, a.rf = rf;
    const long long tiles = (long long)plan->host.n_lines * ((plan->host.n_depth + apod::kTile - 1) / apod::kTile);
    return launch_apod<apod::kInfer>(a, tiles, 2, static_cast<cudaStream_t>(stream));
}

int supra_selftest_bounded_wait(int64_t budget_cycles, int32_t *out_host) {
    if (budget_cycles < (1LL << 10) || budget_cycles > (1LL << 31)) return SUPRA_EINVAL;
    int *d = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void **>(&d), g_selftest) != cudaSuccess) return SUPRA_ECUDA;
    if (cudaMemset(d, 0, 2 * sizeof(int)) != cudaSuccess) return SUPRA_ECUDA;
    bounded_wait_selftest_kernel<<<1, 96>>>((long long)budget_cycles, d);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return SUPRA_ECUDA;
    int h[2] = {0, 0};
    if (cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return SUPRA_ECUDA;
    if (out_host) {
        out_host[0] = h[0];
        out_host[1] = h[1];
    }
    return SUPRA_OK;
}

int supra_device_status(int32_t clear) {
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return SUPRA_ECUDA;
    if (cudaMemcpyFromSymbol(&v, supra::g_status, sizeof(int)) != cudaSuccess) return SUPRA_ECUDA;
    if (clear) {
        const int z = 0;
        if (cudaMemcpyToSymbol(supra::g_status, &z, sizeof(int)) != cudaSuccess) return SUPRA_ECUDA;
    }
    return v;
}

}  // extern "C"

size_t supra::bmode_min_workspace(int32_t n, const supra_plan *const *plans) {
    return n < 1 || !plans ? 0 : min_workspace(n, plans);
}
