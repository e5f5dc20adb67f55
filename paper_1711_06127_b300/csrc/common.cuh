// common.cuh -- device-resident plan record and small PTX wrappers shared by
// the kernels of libsupra (sm_103a).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "supra.h"

namespace supra {

constexpr int kDepthTile = 256;     // depth samples per beamforming tile (one per consumer thread)
constexpr int kMaxTaps = 63;       // IQ low-pass taps; shorter filters are zero-padded to 63, centred
constexpr int kTapSlots = 64;      // 63 centred taps + one zero slot
constexpr int kMaxBands = 4;       // frequency-compounding bank
constexpr int kMaxGroup = 16;       // frames of one plan beamformed together

// Per-line constants (fp32; built from fp64 host geometry).
// Transmit path of one (line, transmit) pair as the excess over r of the path
// to p = o_l + r d: spherical wave from o_t: |p - o_t| - r with b = d.(o_l - o_t),
// g = |o_l - o_t|^2; plane wave of direction n through o_t: n.(p - o_t) - r =
// b + g r with b = n.(o_l - o_t), g = n.d - 1.
struct TxTerm {
    float b, g;
    int tx;             // transmit event (record index)
    int plane;          // 1: plane wave
};

struct LineGeo {
    float ox, oy, oz;   // line origin
    float dx, dy, dz;   // unit direction
    float bt, gt;       // transmit path of the line's own transmit (TxTerm b, g)
    int tx;             // transmit event
    int plane;          // 1: that transmit is a plane wave
    int pad[2];
};

// Resident plan record (lives in device global memory; kernels read it through a pointer).
struct DevPlan {
    // ---- receive geometry
    int n_el, n_tx, n_lines, n_depth, n_s;
    int n_tiles;             // ceil(n_depth / kDepthTile)
    int regular, el_nx, el_ny;   // elements on a row-major nx x ny grid (e = iy * nx + ix)
    int row_y;               // regular, and the elements of each grid row have the same (fp32) y
    int window;
    float win_a, win_b;      // apodization window A + B cos(pi u)
    int win_row;             // staged samples per element row (multiple of 8)
    int bulk_ok;             // n_s % 8 == 0: rows of 16-byte aligned records may be staged with bulk copies
    float fsc;               // fs / c: samples per metre of path
    float t0fs;              // t0 * fs: record start in samples
    float a1;                // two-way delay step per depth sample, in samples
    float depth0, depth_step;
    float inv2f, amin;       // 1 / (2 F), minimum half aperture
    float xmin, xmax, ymin, ymax;
    const float4 *elem;      // [n_el] (x, y, z, 0)
    const LineGeo *lines;    // [n_lines]
    const int *tile_k;       // [n_tiles] integer base of the two-way delay at the tile's first depth
    const float *tile_f;     // [n_tiles] fractional remainder of that base
    const short4 *ap_box;    // [n_lines * n_tiles] element box (ix_lo, ix_hi, iy_lo, iy_hi), inclusive
    const int *line_order;   // [n_lines] lines by decreasing beamforming work
    // ---- envelope + log compression
    int taps;                // odd, <= kMaxTaps (the plan's filter length)
    // Centred form: slot k' = k + 31 - H holds tap k of the plan's filter, the rest are 0,
    // so every filter is applied as a 63-tap one: iq(i) = sum_k' g_k' rf(i + 31 - k').
    float taps_c[kTapSlots]; // h cos(w (k' - 31)): demodulation folded into the taps
    float taps_s[kTapSlots]; // h sin(w (k' - 31))
    float log_a, log_b;      // code = log_a * log2(env) + log_b  (includes the +1/2 of rounding)
    float log_a2, log_b2;    // the same from |iq|^2: code = log_a2 * log2(|iq|^2) + log_b2
    // ---- scan conversion
    int has_grid, geometry, lines_x, lines_y;
    int gnx, gny, gnz;
    float gox, goy, goz, gsx, gsy, gsz;
    float apx, apy, apz;     // apex (sector / pyramid) or line-origin reference (linear)
    float u0, du_inv;        // x-axis line coordinate: u = (t - u0) * du_inv (t = x, angle or tan-angle)
    float w0, dw_inv;        // y-axis line coordinate (pyramid)
    float v0, dv_inv;        // depth coordinate: v = (r - v0) * dv_inv
    // frequency-compounding bank (1 = the taps above only); kept last so the
    // fields the beamforming kernel reads keep their place
    int n_bands;
    float bank_c[kMaxBands][kTapSlots];   // band k: h cos(w_k (k' - 31))
    float bank_s[kMaxBands][kTapSlots];   // band k: h sin(w_k (k' - 31)); env = (2 / K) sum_k |iq_k|
    // coherent compounding: n_comp transmits per line (1 = the line's own transmit);
    // txterms [n_lines][n_comp] when n_comp > 1
    int n_comp;
    const TxTerm *txterms;
};

// A group of up to kMaxGroup frames beamformed together under one plan.
struct FrameGroup {
    CUtensorMap tmap[4];                 // 4D maps (sample pairs, element, transmit, frame), one per staged width
    const DevPlan *plan;
    int n;                               // frames in the group
    int bulk;                            // rows may be staged with 1D bulk async copies (aligned records)
    int tma;                             // frames uniformly strided: stage all frames of a row with one tensor copy
    int line0;                           // first work item (lines) of this group in the launch
    const int16_t *ch[kMaxGroup];
    void *out[kMaxGroup];                // float rf / uint8 bm per frame
};

constexpr int kMaxGroupsPerLaunch = 32;

struct LaunchGroups {
    int n_groups;
    int total_lines;
    int uniform;                         // every group uses the same plan
    int n_seg;                           // depth segments per line (0 or 1: whole lines); CTA = (item, segment)
    // B-mode launches with depth segments: records of the RF around each segment boundary
    // (float [item][frame < G][n_seg - 1][128]), from which a second kernel finishes the
    // outputs there; nullptr: each segment beamforms the halo it needs itself
    float *bnd;
    long long bnd_floats;
    FrameGroup g[kMaxGroupsPerLaunch];
};
static_assert(sizeof(LaunchGroups) <= 32000, "kernel parameter space is 32 KB");

// device status word of this library on each device (first failure code wins);
// libsupra is one translation unit, so the definition lives here.
__device__ int g_status = 0;

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status, 0, code); }

// Checked build (-DSUPRA_CHECKED, a test variant of the library): SUPRA_CHECK(cond) is false, and
// the device status word records SUPRA_EINTERNAL, when an index or alignment invariant fails; the
// caller then skips the access.  The default build compiles every check out (the condition is not
// evaluated).
#ifdef SUPRA_CHECKED
__device__ __forceinline__ bool supra_check(bool ok) {
    if (!ok) set_status(SUPRA_EINTERNAL);
    return ok;
}
#define SUPRA_CHECK(cond) supra_check(cond)
#else
#define SUPRA_CHECK(cond) true
#endif

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~budget clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long budget) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// 1D bulk async copy global -> shared (TMA engine), completion counted on bar.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace supra
