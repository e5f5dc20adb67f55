// das_kernel.cuh -- receive delay-and-sum beamforming (Sec. 1 "receive
// beamforming", Sec. 2 items 1-2, Table 1 "Beamformer") with the envelope and
// log-compression nodes (Sec. 2 items 3-4, Table 1 "Envelope", "Log comp.")
// fused behind it.
//
// One CTA owns one scanline of a group of G frames that share a plan (or one
// depth segment of it, when a launch has too few lines to fill the GPU) and
// streams the line's depth axis in tiles of kTD = 256 samples, one consumer
// thread per depth sample.  The CTA is warp-specialized:
//   * warp 8 (producer) walks the tiles.  Its 32 lanes take 32 elements of the
//     tile's aperture box at a time, bound the depths of the tile at which each
//     element can be inside the F-number aperture, drop elements that never
//     are, and pack the others E to a stage (3 for G = 16 in a ring of three
//     stages; 32 / G otherwise, four stages).  For each element it
//     stages the record window those depths read -- one of four widths (80,
//     144, 208 or 272 samples) -- for all G frames with the TMA engine,
//     completing on the stage's "full" mbarrier.  When the group's frames lie
//     at a uniform stride in memory, one tiled tensor copy (box: width/2 sample
//     pairs x 1 element x 1 transmit x G frames) moves the window for all frames
//     at once and the tensor map's out-of-bounds fill supplies the zero padding
//     outside the record; otherwise the element's lane issues one 1D bulk copy
//     (cp.async.bulk) per frame.
//   * warps 0..7 (consumers) wait on "full", compute the delay, the linear
//     interpolation weights and the apodization weight of each element once,
//     apply them to all G frames, and release the buffer on its "empty"
//     mbarrier.  A ring of stage buffers keeps the HBM stream going while the
//     consumers work; consumers and producer never meet at a CTA barrier.
// Frames of one plan share their delays, which is what makes a batch cheaper
// per frame than a single frame.
//
// The int16 samples are turned into fp32 without the conversion pipe: the
// 16-bit pattern, its sign bit flipped, is placed in the mantissa of 2^23
// (one LOP3), and 2^23 + 2^15 is subtracted (exact).  Pairs of frames share
// packed f32x2 adds and FMAs.
//
// Delay precision.  The two-way delay in samples reaches a few thousand,
// where the fp32 ulp is ~2.4e-4 samples.  The kernel therefore splits it as
//   s = K_tile + f_tile + a1 (i - i0) + (dt + de) fs / c
// with K_tile/f_tile the fp64-built base of the tile's first depth, and
// dt = |p - o_t| - r, de = |p - x_e| - r evaluated without cancellation as
// (|o - q|^2 + 2 r d.(o - q)) / (|p - q| + r).
//
// After the last chunk of a tile (MODE 1) the RF of the tile goes to a
// per-frame ring that keeps the previous tile's last 2H samples, the complex
// demodulating FIR runs over it, and the log-compressed codes are written out.
// With G = 16 the FIR runs on the tensor cores (tcgen05): within a tile it is
// a product of one fixed banded Toeplitz matrix of taps with the ring, so the
// taps sit in tensor memory for the whole CTA, the ring is the B operand in
// shared memory (both split into FP16 hi + lo parts, FP32 accumulation), a
// tenth warp issues the products and the consumers read the accumulators out
// one tile later; other group sizes run it register-blocked on the FP32 cores.
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc.cuh"

namespace supra {

constexpr int kTD = 256;             // depth samples per tile = consumer threads
constexpr int kConsumers = 256;
constexpr int kCtaThreads = 288;     // + one producer warp
// the G = 16 envelope kernel has a tenth warp that issues the tensor-core FIR
template <int G, int MODE>
__host__ __device__ constexpr int das_threads() { return (MODE == 1 && G == 16) ? kCtaThreads + 32 : kCtaThreads; }
// Rows (frame rows of E = rows / G elements) per stage and stages in the ring: 16-frame
// groups stage 3 elements per stage in 3 stages (stage shape SH = 0: fewer hand-overs per
// element) or 2 elements in 4 stages (SH = 1: a deeper ring), the others 32 rows (E <= 32
// producer lanes) in 4.
__host__ __device__ constexpr int rows_of(int G, int SH = 0) { return G == 16 ? (SH == 1 ? 32 : 48) : 32; }
__host__ __device__ constexpr int stages_of(int G, int SH = 0) { return G == 16 ? (SH == 1 ? 4 : 3) : 4; }
constexpr int kStageShapes = 2;
constexpr int kMaxStages = 4;
constexpr float kMagic = 8421376.0f; // 2^23 + 2^15

struct ElemMeta {
    float beta2, gamma, ex, ey;  // 2 d.(o_l - x_e), |o_l - x_e|^2, x_e, y_e
    int ws;                      // absolute sample index of the row's first staged sample
    int ia, ib;                  // depths (absolute indices) this staged window serves
    int flags;                   // bit 0 valid, bits 1-2 width class, bit 3 (slot 0): last stage of the tile,
                                 // bits 4-15: compounded transmit of the stage, bit 16 (slot 0): row stage
};
// A row stage (one-frame tiles of plans with a y window) holds elements of one row of the
// matrix array, so its y window weight is the same for every element.
constexpr int kRowStage = 1 << 16;
__device__ __forceinline__ int meta_valid(const ElemMeta &m) { return m.flags & 1; }
__device__ __forceinline__ int meta_widx(const ElemMeta &m) { return (m.flags >> 1) & 3; }
__device__ __forceinline__ int meta_last(const ElemMeta &m) { return (m.flags >> 3) & 1; }
// compounding: index of the stage's transmit among the line's transmits (a stage never mixes them)
__device__ __forceinline__ int meta_comp(const ElemMeta &m) { return (m.flags >> 4) & 0xFFF; }

// Staged window widths (samples; multiples of 16) and their frame-row strides in shared memory.
constexpr int kNumWidths = 4;
__host__ __device__ constexpr int width_of(int widx) { return 80 + 64 * widx; }   // 80, 144, 208, 272

typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ u64 pack2u(uint32_t lo, uint32_t hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(u64 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// 4D tiled tensor copy global -> shared, completion counted on bar.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// int16 bit pattern (zero-extended) -> float bits of 2^23 + 2^15 + x
__device__ __forceinline__ uint32_t biased(uint32_t u16) { return (u16 ^ 0x8000u) | 0x4B000000u; }

// Apodization window A + B cos(pi u): Hann (1/2, 1/2), Hamming (0.54, 0.46), rect (1, 0).
__device__ __forceinline__ float window_weight(float A, float B, float u) {
    return fmaf(B, __cosf(3.14159265358979f * u), A);
}

// floor(s) and its integer value on the FMA and integer pipes (no rounding or
// conversion instruction): s + 1.5 * 2^23 rounded toward -inf lands in [2^23, 2^24),
// where the floats are the integers and consecutive ones have consecutive bit
// patterns, so it is floor(s) + 1.5 * 2^23 exactly.  Exact for |s| < 2^22 (the
// delays are a few thousand samples; lanes outside the aperture only clamp k).
constexpr float kFloorMagic = 12582912.0f;   // 1.5 * 2^23
__device__ __forceinline__ float floor_split(float s, int &k) {
    const float t = __fadd_rd(s, kFloorMagic);
    k = __float_as_int(t) - __float_as_int(kFloorMagic);
    return t - kFloorMagic;
}

// |o + r d - q| - r without cancellation: (gamma + 2 r beta) / (|p - q| + r),
// beta = d.(o - q), gamma = |o - q|^2.  (0 when p = q = o.)
__device__ __forceinline__ float path_excess(float r, float beta, float gamma) {
    const float r2 = fmaxf(fmaf(r, r + 2.0f * beta, gamma), 1e-30f);
    const float den = fmaxf(fmaf(r2, rsqrtf(r2), r), 1e-20f);
    return __fdividef(fmaf(2.0f * r, beta, gamma), den);
}

// Transmit path excess over r (see TxTerm): spherical or plane wave.
__device__ __forceinline__ float tx_excess(float r, float b, float g, int plane) {
    return plane ? fmaf(g, r, b) : path_excess(r, b, g);
}

// named barrier among the 256 consumer threads (the producer warp never joins)
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ int consumer_sync_or(int p) {
    int r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.s32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, 256, pi;\n\tselp.s32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(p)
        : "memory");
    return r;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// try_wait that lets the thread sleep (up to ~20 us) until the phase completes,
// so waiting warps do not take issue slots from working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Wait for a phase, giving up after ~2^31 cycles or when another thread has
// flagged an abort.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait_sleep(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    return true;
}

// Per-frame RF ring of the envelope stage: position u holds the RF of depth
// i0 - 64 + u (u in [0, kRingLen)): the previous tile's last 64 samples, then the
// current tile.  Tile outputs are depths o = i0 - 32 + t, t in [0, kTD), and use
// positions u = 63 + t - k' (k' = 0..63 over the centred taps).  One pad word every
// 8 positions keeps blocked reads conflict-free.
constexpr int kHalo = 64;
constexpr int kLag = 32;
constexpr int kRingLen = kTD + kHalo;
__device__ __forceinline__ int ring_addr(int p) { return p + (p >> 3); }

// G = 16 FIR on the tensor cores.  The ring holds the RF [kRingLen][16 frames]
// split as x = hi + lo (hi = x rounded to FP16, lo = the rest rounded to FP16),
// as one MN-major B operand of N = 32 columns (hi of frames 0..15, then lo) in
// the canonical no-swizzle layout: the core matrix (8 ring positions x 8
// columns, 128 B) of positions 8a.. and columns 8c.. sits at byte 512 a + 128 c,
// so core matrices adjacent in K (positions) are 512 B apart and adjacent in N
// 128 B apart.
constexpr int kRing16Bytes = kRingLen * 32 * 2;
// tensor memory: taps hi (columns 0-63) and lo (64-127), 128 x 128 FP16 each;
// accumulators D (128-255, 4 blocks x 32 columns: the hi and lo halves of 16 frames)
constexpr uint32_t kFirTmemCols = 256;
constexpr uint32_t kFirColLo = 64, kFirColD = 128;

// Shared-memory layout, identical on host and device.
struct SmemLayout {
    int bars, meta, taps, ring, stage, total, ring_stride;
    __host__ __device__ SmemLayout(int G, int mode, int W, int SH = 0) {
        bars = 0;                                             // full[kMaxStages], empty[kMaxStages], abort flag,
                                                              // FIR done (72), tensor-memory base (80),
                                                              // FIR ring ready (88)
        meta = 128;                                           // [stages][rows] ElemMeta
        taps = meta + stages_of(G, SH) * rows_of(G, SH) * (int)sizeof(ElemMeta); // [kTapSlots] float4 (c, c, s, s)
        ring = taps + (mode == 1 ? kTapSlots * 16 : 0);
        ring_stride = ((kRingLen - 1) + ((kRingLen - 1) >> 3) + 1 + 3) & ~3;
        stage = ring + (mode == 1 ? (G == 16 ? kRing16Bytes : G * ring_stride * 4) : 0);
        stage = (stage + 127) & ~127;
        total = stage + stages_of(G, SH) * rows_of(G, SH) * W * 2;
    }
};

// Item -> (group, line).  Launches of one plan interleave groups so that the
// heaviest lines (plan-sorted) go first over all groups.
__device__ __forceinline__ void locate_item(const LaunchGroups &L, int item, int &gi, int &line) {
    if (L.uniform) {
        gi = item % L.n_groups;
        line = L.g[gi].plan->line_order[item / L.n_groups];
        return;
    }
    gi = 0;
    while (gi + 1 < L.n_groups && L.g[gi + 1].line0 <= item) ++gi;
    line = L.g[gi].plan->line_order[item - L.g[gi].line0];
}

// -------------------------------------------------------------------------------------------------
// Plan constants the producer needs, held in registers (the mbarrier/fence asm
// statements clobber memory, which would otherwise force reloads every stage).
struct ProdConst {
    const short4 *ap_box;
    const float4 *elem;
    const int *tile_k;
    const float *tile_f;
    int n_tiles, el_nx, n_depth, n_s, n_el;
    float depth0, depth_step, fsc, a1, t0fs, inv2f, amin, xmin, xmax, ymin, ymax;
    __device__ ProdConst(const DevPlan *P)
        : ap_box(P->ap_box), elem(P->elem), tile_k(P->tile_k), tile_f(P->tile_f), n_tiles(P->n_tiles),
          el_nx(P->el_nx), n_depth(P->n_depth), n_s(P->n_s), n_el(P->n_el), depth0(P->depth0),
          depth_step(P->depth_step), fsc(P->fsc), a1(P->a1), t0fs(P->t0fs), inv2f(P->inv2f), amin(P->amin),
          xmin(P->xmin), xmax(P->xmax), ymin(P->ymin), ymax(P->ymax) {}
};

// Depths of the tile at which element slot j of the box can be inside the
// aperture: the test max(|x_e - q_x|, |y_e - q_y|) <= a is evaluated every 32
// depths; the left side minus a changes by at most lip per metre of r (q is a
// clamp of a point moving along d, a grows at d_z / (2F)), so a depth within
// 16 samples of a test point can pass only if that point is within
// lip * 16 * depth_step of passing (plus the consumers' rounding): [ia, ib]
// holds every depth of the tile whose aperture test passes.  Returns false if
// no depth can.
// With `halves`, item j is half j % 2 of box element j / 2 (depth steps coarser
// than c / (2 fs) make a whole tile's window too wide for one slot).
__device__ __forceinline__ bool element_range(const ProdConst &C, const LineGeo &lg, float lip, short4 b, int tile,
                                              bool halves, int j, int &e, float4 &xe, int &ia, int &ib) {
    const int nbx = b.y - b.x + 1, nby = b.w - b.z + 1;
    const int je = halves ? j >> 1 : j;
    if (je >= nbx * nby) return false;
    e = (b.z + je / nbx) * C.el_nx + b.x + je % nbx;
    xe = __ldg(&C.elem[e]);
    int i0 = tile * kTD;
    int i1 = min(i0 + kTD - 1, C.n_depth - 1);
    if (halves) {
        if (j & 1) i0 += kTD / 2;
        else i1 = min(i1, i0 + kTD / 2 - 1);
        if (i0 > i1) return false;
    }
    // (+ 2e-6 a: the consumers' test |x_e - q_x| / a <= 1 passes up to a few float roundings
    // beyond a, so every depth whose test passes lies in [ia, ib])
    const float margin = lip * 16.0f * C.depth_step * 1.001f + 1e-9f;
    int first = -1, last = -1;
#pragma unroll
    for (int k = 0; k <= kTD / 32; ++k) {
        const int i = min(i0 + 32 * k, i1);
        if (k > 0 && i0 + 32 * (k - 1) >= i1) break;
        const float r = C.depth0 + (float)i * C.depth_step;
        const float px = fmaf(r, lg.dx, lg.ox), py = fmaf(r, lg.dy, lg.oy), pz = fmaf(r, lg.dz, lg.oz);
        const float qx = fminf(fmaxf(px, C.xmin), C.xmax), qy = fminf(fmaxf(py, C.ymin), C.ymax);
        const float a = fmaxf(pz * C.inv2f, C.amin);
        const float g = fmaxf(fabsf(xe.x - qx), fabsf(xe.y - qy)) - a;
        if (g <= fmaf(2e-6f, a, margin)) {
            if (first < 0) first = k;
            last = k;
        }
    }
    if (first < 0) return false;
    ia = max(i0, i0 + 32 * first - 16);
    ib = min(i1, i0 + 32 * last + 16);
    return true;
}

// Record window of depths [ia, ib] for element e: start ws (a multiple of 8) and
// the width class that covers every sample those depths interpolate.
__device__ __forceinline__ void element_window(const ProdConst &C, const LineGeo &lg, const TxTerm &tt, int ci,
                                               int tile, int ia, int ib, float4 xe, ElemMeta &m) {
    const float mx = lg.ox - xe.x, my = lg.oy - xe.y, mz = lg.oz - xe.z;
    const float beta = lg.dx * mx + lg.dy * my + lg.dz * mz;
    const float gamma = mx * mx + my * my + mz * mz;
    const int i0 = tile * kTD;   // the tile's delay base is at its first depth
    const float r0 = C.depth0 + (float)ia * C.depth_step;
    const float r1 = C.depth0 + (float)ib * C.depth_step;
    const int kt = __ldg(&C.tile_k[tile]);
    const float ft = __ldg(&C.tile_f[tile]);
    const float s0 = ft + C.a1 * (float)(ia - i0) + (tx_excess(r0, tt.b, tt.g, tt.plane) + path_excess(r0, beta, gamma)) * C.fsc;
    const float s1 = ft + C.a1 * (float)(ib - i0) + (tx_excess(r1, tt.b, tt.g, tt.plane) + path_excess(r1, beta, gamma)) * C.fsc;
    float lo = fminf(s0, s1), hi = fmaxf(s0, s1);
    // The two-way path is convex in r (a plane wave's path is linear): its maximum is at
    // an end, its minimum may be inside; bound that minimum by the sum of the two paths' minima.
    const bool tx_min_inside = !tt.plane && -tt.b > r0 && -tt.b < r1;
    if ((-beta > r0 && -beta < r1) || tx_min_inside) {
        const float re = fminf(fmaxf(-beta, r0), r1);
        const float de = sqrtf(fmaxf(fmaf(re, re + 2.0f * beta, gamma), 0.0f));
        float dtp;
        if (tt.plane) {
            dtp = fminf(fmaf(1.0f + tt.g, r0, tt.b), fmaf(1.0f + tt.g, r1, tt.b));
        } else {
            const float rt = fminf(fmaxf(-tt.b, r0), r1);
            dtp = sqrtf(fmaxf(fmaf(rt, rt + 2.0f * tt.b, tt.g), 0.0f));
        }
        lo = fminf(lo, (de + dtp) * C.fsc - C.t0fs - (float)kt);
    }
    const int lo_i = kt + (int)floorf(lo) - 1;
    const int ws = (lo_i >> 3) << 3;                              // 16-byte aligned window start
    const int need = kt + (int)floorf(hi) + 2 - ws;               // samples up to x1 of the last depth
    int widx = need <= width_of(0) ? 0 : (need - width_of(0) + 63) / 64;   // smallest width >= need
    if (widx >= kNumWidths) {
        set_status(SUPRA_EINTERNAL);
        widx = kNumWidths - 1;
    }
    m.beta2 = beta + beta;
    m.gamma = gamma;
    m.ex = xe.x;
    m.ey = xe.y;
    m.ws = ws;
    m.ia = ia;
    m.ib = ib;
    m.flags = 1 | (widx << 1) | (ci << 4);
}

// The same for the line's own spherical transmit (the kernel without extended
// transmit models; kept separate so that kernel compiles to the spherical-only code).
__device__ __forceinline__ void element_window_line(const ProdConst &C, const LineGeo &lg, int tile, int ia, int ib,
                                               float4 xe, ElemMeta &m) {
    const float mx = lg.ox - xe.x, my = lg.oy - xe.y, mz = lg.oz - xe.z;
    const float beta = lg.dx * mx + lg.dy * my + lg.dz * mz;
    const float gamma = mx * mx + my * my + mz * mz;
    const int i0 = tile * kTD;   // the tile's delay base is at its first depth
    const float r0 = C.depth0 + (float)ia * C.depth_step;
    const float r1 = C.depth0 + (float)ib * C.depth_step;
    const int kt = __ldg(&C.tile_k[tile]);
    const float ft = __ldg(&C.tile_f[tile]);
    const float s0 = ft + C.a1 * (float)(ia - i0) + (path_excess(r0, lg.bt, lg.gt) + path_excess(r0, beta, gamma)) * C.fsc;
    const float s1 = ft + C.a1 * (float)(ib - i0) + (path_excess(r1, lg.bt, lg.gt) + path_excess(r1, beta, gamma)) * C.fsc;
    float lo = fminf(s0, s1), hi = fmaxf(s0, s1);
    // The two-way path is convex in r: its maximum is at an end, its minimum may be
    // inside; bound that minimum by the sum of the two paths' minima.
    if ((-beta > r0 && -beta < r1) || (-lg.bt > r0 && -lg.bt < r1)) {
        const float re = fminf(fmaxf(-beta, r0), r1), rt = fminf(fmaxf(-lg.bt, r0), r1);
        const float de = sqrtf(fmaxf(fmaf(re, re + 2.0f * beta, gamma), 0.0f));
        const float dtp = sqrtf(fmaxf(fmaf(rt, rt + 2.0f * lg.bt, lg.gt), 0.0f));
        lo = fminf(lo, (de + dtp) * C.fsc - C.t0fs - (float)kt);
    }
    const int lo_i = kt + (int)floorf(lo) - 1;
    const int ws = (lo_i >> 3) << 3;                              // 16-byte aligned window start
    const int need = kt + (int)floorf(hi) + 2 - ws;               // samples up to x1 of the last depth
    int widx = need <= width_of(0) ? 0 : (need - width_of(0) + 63) / 64;   // smallest width >= need
    if (widx >= kNumWidths) {
        set_status(SUPRA_EINTERNAL);
        widx = kNumWidths - 1;
    }
    m.beta2 = beta + beta;
    m.gamma = gamma;
    m.ex = xe.x;
    m.ey = xe.y;
    m.ws = ws;
    m.ia = ia;
    m.ib = ib;
    m.flags = 1 | (widx << 1);
}

// Stages the element's window of all frames into slot `slot` of a stage (frame
// rows of width_of(widx) samples, packed).  Returns the bytes that will land.
template <int G>
__device__ __forceinline__ uint32_t stage_element(const ProdConst &C, const FrameGroup &fg, int nf, int tx,
                                                  int e, const ElemMeta &m, int16_t *slot_base, uint64_t *full) {
    const int wsamp = width_of(meta_widx(m));
    if (fg.tma) {
        // the tensor map counts sample pairs: x = ws / 2 must be 16-byte aligned (ws % 8 == 0)
        if (!SUPRA_CHECK((m.ws & 7) == 0)) return 0u;
        tma_load_4d(slot_base, &fg.tmap[meta_widx(m)], m.ws >> 1, e, tx, 0, full);
        return (uint32_t)(G * wsamp * 2);
    }
    const int ws = m.ws, n_s = C.n_s;
    const int c0 = max(ws, 0), c1 = min(ws + wsamp, n_s);
    const long long rec = ((long long)tx * C.n_el + e) * (long long)n_s;
    uint32_t total = 0;
    for (int f = 0; f < nf; ++f) {
        int16_t *row = slot_base + f * wsamp;
        if (c0 > ws || c1 < ws + wsamp) {   // zero padding outside the record
            const int a_end = min(c0, ws + wsamp) - ws;
            for (int k = 0; k < a_end; ++k) row[k] = 0;
            for (int k = max(c1, c0) - ws; k < wsamp; ++k) row[k] = 0;
        }
        if (fg.bulk) {
            if (c1 > c0 &&
                SUPRA_CHECK(((reinterpret_cast<uintptr_t>(row + (c0 - ws)) | reinterpret_cast<uintptr_t>(fg.ch[f] + rec + c0) |
                              (uintptr_t)((c1 - c0) * 2)) & 15) == 0)) {
                fence_proxy_async_smem();
                bulk_g2s(row + (c0 - ws), fg.ch[f] + rec + c0, (uint32_t)(c1 - c0) * 2u, full);
                total += (uint32_t)(c1 - c0) * 2u;
            }
        } else {
            const int16_t *src = fg.ch[f] + rec;
            for (int k = c0; k < c1; ++k) row[k - ws] = src[k];
        }
    }
    return total;
}

// -------------------------------------------------------------------------------------------------
// Consumer: the element slots of one stage for this thread's depth sample.
struct Geo {
    float w0, w1, w;
    int idx;
    bool go;   // some lane of the warp is inside this element's aperture
};

__device__ __forceinline__ Geo element_geo(const ElemMeta &md, int i, float r, float qx, float qy, float inv_a,
                                           float base, int kt, bool use_y, float wa, float wb, float fsc) {
    Geo g;
    const float ux = (md.ex - qx) * inv_a;
    bool in = fabsf(ux) <= 1.0f && i >= md.ia && i <= md.ib;
    float w = window_weight(wa, wb, ux);
    if (use_y) {
        const float uy = (md.ey - qy) * inv_a;
        in = in && fabsf(uy) <= 1.0f;
        w *= window_weight(wa, wb, uy);
    }
    g.go = __any_sync(0xffffffffu, in) && meta_valid(md);
    w = in ? w : 0.0f;
    const float num = fmaf(r, md.beta2, md.gamma);                       // |p - x_e|^2 - r^2
    const float r2 = fmaxf(fmaf(r, r, num), 1e-30f);                      // |p - x_e|^2
    const float den = fmaxf(fmaf(r2, rsqrtf(r2), r), 1e-20f);            // |p - x_e| + r
    const float s = fmaf(__fdividef(num, den), fsc, base);
    int k;
    const float fl = floor_split(s, k);
#ifdef SUPRA_CHECKED
    // every sample pair an in-aperture depth reads lies inside the element's staged window
    const int raw = kt + k - md.ws;
    SUPRA_CHECK(!in || !meta_valid(md) || (raw >= 0 && raw + 1 < width_of(meta_widx(md))));
#endif
    g.w = w;
    g.w1 = w * (s - fl);
    g.w0 = w - g.w1;
    // (clamped for lanes outside the aperture, whose weights are 0; a negative index wraps high)
    g.idx = (int)min((unsigned)(kt + k - md.ws), (unsigned)(width_of(kNumWidths - 1) - 2));
    return g;
}

// The same for one-frame tiles, without the warp vote: an element's frame work is a few
// instructions, less than the vote and branch that would skip it, so every slot is applied
// and a lane outside the aperture, or a slot past the stage's valid prefix, has weight 0.
// YM: 0 no y window (linear arrays), 1 the element's own, 2 the row stage's (wy, iny).
// RANGE: test the depth against the slot's depth range [ia, ib] -- needed when an element is
// staged as two half-tile slots (depth steps coarser than c / (2 fs)); otherwise every depth of
// the record inside the aperture lies in its slot's range (element_range), and depths past the
// record's end (nd: the last tile's padding threads, whose values are discarded) are skipped by
// the checked build's window test, which verifies the rest.
template <int YM, bool RANGE>
__device__ __forceinline__ Geo element_geo1(const ElemMeta &md, int i, float r, float qx, float qy, float inv_a,
                                            float base, int kt, float wa, float wb, float fsc, float wy, bool iny,
                                            int nd) {
    Geo g;
    const float ux = (md.ex - qx) * inv_a;
    bool in = fabsf(ux) <= 1.0f && (!RANGE || (i >= md.ia && i <= md.ib)) && meta_valid(md);
    float w = window_weight(wa, wb, ux);
    if constexpr (YM == 1) {
        const float uy = (md.ey - qy) * inv_a;
        in = in && fabsf(uy) <= 1.0f;
        w *= window_weight(wa, wb, uy);
    } else if constexpr (YM == 2) {
        in = in && iny;
        w *= wy;
    }
    g.go = true;
    w = in ? w : 0.0f;
    const float num = fmaf(r, md.beta2, md.gamma);
    const float r2 = fmaxf(fmaf(r, r, num), 1e-30f);
    const float den = fmaxf(fmaf(r2, rsqrtf(r2), r), 1e-20f);
    const float s = fmaf(__fdividef(num, den), fsc, base);
    int k;
    const float fl = floor_split(s, k);
#ifdef SUPRA_CHECKED
    const int raw = kt + k - md.ws;
    SUPRA_CHECK(!in || i >= nd || (raw >= 0 && raw + 1 < width_of(meta_widx(md))));
#else
    (void)nd;
#endif
    g.w = w;
    g.w1 = w * (s - fl);
    g.w0 = w - g.w1;
    g.idx = (int)min((unsigned)(kt + k - md.ws), (unsigned)(width_of(kNumWidths - 1) - 2));
    return g;
}

// Frame loop of one element: frame f's row starts at rows + f * FS.
template <int G, int FS>
__device__ __forceinline__ void element_frames(const int16_t *rows, const Geo &g, u64 (&acc2)[G / 2 > 0 ? G / 2 : 1],
                                               float &acc1) {
    const uint16_t *row = reinterpret_cast<const uint16_t *>(rows) + g.idx;
    if constexpr (G == 1) {
        const float x0 = __uint_as_float(biased(row[0])) - kMagic;
        const float x1 = __uint_as_float(biased(row[1])) - kMagic;
        acc1 = fmaf(g.w1, x1, fmaf(g.w0, x0, acc1));   // the frame-pair loop's order
    } else {
        const u64 W0 = pack2(g.w0, g.w0), W1 = pack2(g.w1, g.w1), NB = pack2(-kMagic, -kMagic);
#pragma unroll
        for (int q = 0; q < G / 2; ++q) {
            const uint16_t *ra = row + (2 * q) * FS;
            const uint16_t *rb = row + (2 * q + 1) * FS;
            const u64 f0 = add2(pack2u(biased(ra[0]), biased(rb[0])), NB);
            const u64 f1 = add2(pack2u(biased(ra[1]), biased(rb[1])), NB);
            acc2[q] = fma2(W1, f1, fma2(W0, f0, acc2[q]));
        }
    }
}

template <int G>
__device__ __forceinline__ void element_frames_w(const int16_t *rows, int widx, const Geo &g,
                                                 u64 (&acc2)[G / 2 > 0 ? G / 2 : 1], float &acc1) {
    if constexpr (G == 1) {
        element_frames<1, 0>(rows, g, acc2, acc1);
    } else {
        switch (widx) {
            case 0: element_frames<G, width_of(0)>(rows, g, acc2, acc1); break;
            case 1: element_frames<G, width_of(1)>(rows, g, acc2, acc1); break;
            case 2: element_frames<G, width_of(2)>(rows, g, acc2, acc1); break;
            default: element_frames<G, width_of(3)>(rows, g, acc2, acc1); break;
        }
    }
}

constexpr int kSlotSamples = width_of(kNumWidths - 1);   // samples per frame row reserved in a slot

// One-frame stages (32 slots): groups of four slots, their geometry first (independent
// chains), then their samples; valid slots are a prefix.
template <int YM, bool RANGE>
__device__ __forceinline__ void consume_one_frame(const int16_t *__restrict__ sbuf, const ElemMeta *meta, int i,
                                                  float r, float qx, float qy, float inv_a, float base, int kt,
                                                  float wa, float wb, float fsc, float wy, bool iny, float &acc1,
                                                  float &wsum, int nd) {
    constexpr int kGrp = 4;
    u64 unused[1];
#pragma unroll 1
    for (int e0 = 0; e0 < rows_of(1); e0 += kGrp) {
        if (!meta_valid(meta[e0])) break;
        Geo g[kGrp];
#pragma unroll
        for (int j = 0; j < kGrp; ++j)
            g[j] = element_geo1<YM, RANGE>(meta[e0 + j], i, r, qx, qy, inv_a, base, kt, wa, wb, fsc, wy, iny, nd);
#pragma unroll
        for (int j = 0; j < kGrp; ++j) {
            element_frames<1, 0>(sbuf + (e0 + j) * kSlotSamples, g[j], unused, acc1);
            wsum += g[j].w;
        }
    }
}

template <int G, int SH>
__device__ __forceinline__ void consume_stage(const int16_t *__restrict__ sbuf, const ElemMeta *meta, int i, float r,
                                              float qx, float qy, float inv_a, float base, int kt,
                                              bool use_y, float wa, float wb, float fsc,
                                              u64 (&acc2)[G / 2 > 0 ? G / 2 : 1], float &acc1, float &wsum,
                                              bool halves, int nd) {
    constexpr int E = rows_of(G, SH) / G;
    if constexpr (G == 1) {
        const int f0 = meta[0].flags;
        if (!use_y) {
            if (halves)
                consume_one_frame<0, true>(sbuf, meta, i, r, qx, qy, inv_a, base, kt, wa, wb, fsc, 1.0f, true, acc1,
                                           wsum, nd);
            else
                consume_one_frame<0, false>(sbuf, meta, i, r, qx, qy, inv_a, base, kt, wa, wb, fsc, 1.0f, true, acc1,
                                            wsum, nd);
        } else if (f0 & kRowStage) {   // (row stages only without halves)
            const float uy = (meta[0].ey - qy) * inv_a;
            consume_one_frame<2, false>(sbuf, meta, i, r, qx, qy, inv_a, base, kt, wa, wb, fsc,
                                        window_weight(wa, wb, uy), fabsf(uy) <= 1.0f, acc1, wsum, nd);
        } else if (halves) {
            consume_one_frame<1, true>(sbuf, meta, i, r, qx, qy, inv_a, base, kt, wa, wb, fsc, 1.0f, true, acc1, wsum,
                                       nd);
        } else {
            consume_one_frame<1, false>(sbuf, meta, i, r, qx, qy, inv_a, base, kt, wa, wb, fsc, 1.0f, true, acc1,
                                        wsum, nd);
        }
    } else if constexpr (E <= 4) {
        // geometry of every slot first (independent chains), then the frame loops
        Geo g[E];
        int widx[E];
#pragma unroll
        for (int ej = 0; ej < E; ++ej) {
            const ElemMeta md = meta[ej];
            widx[ej] = meta_widx(md);
            g[ej] = element_geo(md, i, r, qx, qy, inv_a, base, kt, use_y, wa, wb, fsc);
        }
#pragma unroll
        for (int ej = 0; ej < E; ++ej) {
            if (!g[ej].go) continue;
            element_frames_w<G>(sbuf + ej * G * kSlotSamples, widx[ej], g[ej], acc2, acc1);
            wsum += g[ej].w;
        }
    } else {
        // groups of four slots: their geometry first (independent chains), then their samples;
        // valid slots are a prefix, and an invalid slot's `go` is false
        constexpr int kGrp = 4;
        static_assert(E % kGrp == 0, "slot groups");
#pragma unroll 1
        for (int e0 = 0; e0 < E; e0 += kGrp) {
            if (!meta_valid(meta[e0])) break;
            Geo g[kGrp];
            int widx[kGrp];
#pragma unroll
            for (int j = 0; j < kGrp; ++j) {
                const ElemMeta md = meta[e0 + j];
                widx[j] = meta_widx(md);
                g[j] = element_geo(md, i, r, qx, qy, inv_a, base, kt, use_y, wa, wb, fsc);
            }
#pragma unroll
            for (int j = 0; j < kGrp; ++j) {
                if (!g[j].go) continue;
                element_frames_w<G>(sbuf + (e0 + j) * G * kSlotSamples, widx[j], g[j], acc2, acc1);
                wsum += g[j].w;
            }
        }
    }
}

// -------------------------------------------------------------------------------------------------
// Envelope + log compression of one tile (outputs o = i0 - 32 + t, t in [0, kTD)):
// iq = sum_k' g_k' rf(o + 31 - k'), code = floor(a2 log2|iq|^2 + b2) clamped to [0, 255]
// (|iq|^2 = 0 gives -inf and code 0, as env = 0 does).
__device__ __forceinline__ uint32_t code_of(float q, float a2, float b2) {
    // floor with the conversion's saturation at 0 (also for -inf), after clamping at 255
    return __float2uint_rd(fminf(fmaf(a2, __log2f(q), b2), 255.f));
}

// ---- G = 16: the FIR on the tensor cores.  Per 64-output block b of the tile,
// D_b [128 x 32] = A [128 x 128] * ring [positions 64 b .. 64 b + 127][hi, lo of 16 frames].
// Row r of A (lane r of tensor memory): quadrant qd = r / 32, j = r % 32, part
// j / 16 (0: cos taps -> I, 1: sin taps -> Q) of the block's output t = 16 qd +
// j % 16; column u (ring position 64 b + u) holds tap k' = 63 + t - u when
// 0 <= k' < 64, else 0.  A is the same for every block and every tile.  With A
// and the ring each split into FP16 hi + lo parts, two MMAs per K step (A hi and
// A lo, each against the ring's hi and lo columns; FP32 accumulation) leave an
// error of order 2^-22 of each product, as FP32 arithmetic would.  The taps are scaled by kFirTapScale
// (a power of two) so that their lo parts stay normal FP16 numbers; the log
// stage removes the scale exactly.
constexpr float kFirTapScale = 4096.0f;
constexpr float kFirLog2Scale2 = 24.0f;   // log2(kFirTapScale^2)

__device__ __forceinline__ uint32_t half2_bits(__half2 h) { return *reinterpret_cast<const uint32_t *>(&h); }

// (a, b) -> FP16 pairs hi = (a, b) rounded and lo = the remainders rounded.
__device__ __forceinline__ void split_half2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    hi = half2_bits(h);
    lo = half2_bits(__floats2half2_rn(a - hf.x, b - hf.y));
}

// Tap pairs for the fill: entry j of table (part, plane) holds the FP16 (hi or lo)
// pair of the scaled taps k = j - 64 and k - 1 (0 outside 0..63), j < 192; the
// four tables (cos hi, cos lo, sin hi, sin lo) are kFirPairStride words apart
// (200: the sin tables fall 16 banks away from the cos tables).
constexpr int kFirPairStride = 200;
constexpr int kFirPairBytes = 4 * kFirPairStride * 4;
static_assert(kFirPairBytes <= (kRingLen - kTD) / 8 * 512, "tap-pair tables exceed the last ring positions");

__device__ __forceinline__ void fir_tc_build_pairs(const DevPlan *__restrict__ P, uint32_t *tab) {
    for (int e = threadIdx.x; e < 2 * 192; e += blockDim.x) {
        const int part = e / 192, j = e % 192, k = j - 64;
        const float *taps = part ? P->taps_s : P->taps_c;
        const float a = (k >= 0 && k < kTapSlots) ? kFirTapScale * taps[k] : 0.f;
        const float b = (k >= 1 && k - 1 < kTapSlots) ? kFirTapScale * taps[k - 1] : 0.f;
        uint32_t hi, lo;
        split_half2(a, b, hi, lo);
        tab[(2 * part) * kFirPairStride + j] = hi;
        tab[(2 * part + 1) * kFirPairStride + j] = lo;
    }
}

// Warps 0..3 write lanes 32 w .. 32 w + 31 of A hi and A lo (64 columns of FP16
// pairs each): column c of row (part, t) is the pair of taps k' = 63 + t - 2 c, k' - 1.
__device__ __forceinline__ void fir_tc_fill_taps(const uint32_t *tab, uint32_t tbase, int warp, int lane) {
    const int t = 16 * warp + (lane & 15);
    const uint32_t *th = tab + (lane >> 4) * 2 * kFirPairStride + 127 + t;   // j = 63 + t + 64 at c = 0
    const uint32_t *tl = th + kFirPairStride;
    const uint32_t row = tbase + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 16) {
        uint32_t rh[16], rl[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            rh[c] = th[-2 * (c0 + c)];
            rl[c] = tl[-2 * (c0 + c)];
        }
        tc::tmem_st16(row + (uint32_t)c0, rh);
        tc::tmem_st16(row + kFirColLo + (uint32_t)c0, rl);
    }
    tc::tmem_st_wait();
}

// This thread's 16 frames of ring position u, as FP16 hi (columns 0..15) and lo (16..31).
__device__ __forceinline__ void ring16_put(unsigned char *ring16, int u, const float (&v)[16]) {
    uint32_t h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) split_half2(v[2 * k], v[2 * k + 1], h[k], l[k]);
    unsigned char *row = ring16 + (u >> 3) * 512 + (u & 7) * 16;
    *reinterpret_cast<uint4 *>(row) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(row + 128) = make_uint4(h[4], h[5], h[6], h[7]);
    *reinterpret_cast<uint4 *>(row + 256) = make_uint4(l[0], l[1], l[2], l[3]);
    *reinterpret_cast<uint4 *>(row + 384) = make_uint4(l[4], l[5], l[6], l[7]);
}

// One thread: 8 K steps of 16 positions x the 4 blocks x (A hi, A lo), then a commit to `bar`.
__device__ __forceinline__ void fir_tc_issue(uint32_t tbase, uint32_t ring_saddr, uint64_t *bar) {
    constexpr uint32_t idesc = tc::idesc_f16(128, 32, false, true);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t d = tbase + kFirColD + 32u * b;
            const uint64_t bd = tc::smem_desc(ring_saddr + 4096u * b + 1024u * kk, 512, 128);
            tc::mma_f16_ta(d, tbase + 8u * kk, bd, idesc, kk > 0);
            tc::mma_f16_ta(d, tbase + kFirColLo + 8u * kk, bd, idesc, true);
        }
    }
    tc::mma_commit(bar);
}

// The lag tile after a line's last tile has outputs t < 32 only: block 0's products.
__device__ __forceinline__ void fir_tc_issue_block0(uint32_t tbase, uint32_t ring_saddr, uint64_t *bar) {
    constexpr uint32_t idesc = tc::idesc_f16(128, 32, false, true);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint64_t bd = tc::smem_desc(ring_saddr + 1024u * kk, 512, 128);
        tc::mma_f16_ta(tbase + kFirColD, tbase + 8u * kk, bd, idesc, kk > 0);
        tc::mma_f16_ta(tbase + kFirColD, tbase + kFirColLo + 8u * kk, bd, idesc, true);
    }
    tc::mma_commit(bar);
}

// Warp w reads lanes 32 (w % 4) .. of blocks 2 (w / 4) and 2 (w / 4) + 1: lane j
// holds part j / 16 of output t = 64 blk + 16 (w % 4) + j % 16 for the 16 frames
// (the sum of a block's hi and lo columns).
// Lanes j and j ^ 16 swap half of their values, so lane j < 16 finishes |iq|^2
// of frames 0..7 and lane j >= 16 of frames 8..15, and writes their codes.
__device__ __forceinline__ void fir_tc_epilogue(uint32_t tbase, const FrameGroup &fg, int nf, long long row_off,
                                                int i0, int nd, float a2, float b2s) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qd = warp & 3, h = warp >> 2;
    float v[32];
    {
        const uint32_t ta = tbase + ((uint32_t)(32 * qd) << 16) + kFirColD + 64u * h;
        float d[32];
#pragma unroll
        for (int bi = 0; bi < 2; ++bi) {
            tc::tmem_ld32(ta + 32u * bi, d);
#pragma unroll
            for (int f = 0; f < 16; ++f) v[16 * bi + f] = d[f] + d[16 + f];
        }
    }
    const bool hi = lane >= 16;
    const int f0 = hi ? 8 : 0;
#pragma unroll
    for (int bi = 0; bi < 2; ++bi) {
        const int o = i0 - kLag + 64 * (2 * h + bi) + 16 * qd + (lane & 15);
        const bool in = o >= 0 && o < nd;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float a = v[16 * bi + k], b = v[16 * bi + 8 + k];
            const float other = __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
            const float keep = hi ? b : a;
            const float q = fmaf(keep, keep, other * other);
            if (in && f0 + k < nf) static_cast<uint8_t *>(fg.out[f0 + k])[row_off + o] = (uint8_t)code_of(q, a2, b2s);
        }
    }
}

// Wait (bounded) for the products of tile `tile` (phase tile of the FIR
// mbarrier); true for the whole warp when they are complete.  A timeout flags the
// CTA and sets the device status.
__device__ __forceinline__ bool fir_tc_wait(uint64_t *bar, int tile, volatile int *abort_flag, bool &aborted) {
    const bool ok = __all_sync(0xffffffffu, wait_phase(bar, (uint32_t)(tile & 1), abort_flag));
    if (!ok) {
        aborted = true;
        *abort_flag = 1;
        set_status(SUPRA_ETIMEOUT);
    }
    return ok;
}

// Other group sizes: frame pairs with BO = G / 2 outputs per thread (G >= 2), or one
// output per thread (G == 1); addresses computed at run time.
// Outputs t < t_min of the tile are not written (a segment's first outputs, finished from
// the boundary records).
template <int G>
__device__ __forceinline__ void fir_log_tile_generic(const FrameGroup &fg, int nf, int line, int i0, int nd,
                                                     const float *ring, int RS, const float4 *taps4, float a2,
                                                     float b2, int t_min) {
    const int tid = threadIdx.x;
    const long long row_off = (long long)line * nd;
    if constexpr (G == 1) {
        // Two consecutive outputs per thread (threads 0..127): output t + 1 reads at tap k + 1
        // the ring position that output t reads at tap k, so each tap loads one new position.
        // An output's (I, Q) is one f32x2 pair updated with the tap pair (c_k, s_k) (taps4 holds
        // (c, s, c, s) here), tap by tap in the same order as one output per thread.
        const int t0 = 2 * tid;
        if (tid >= kTD / 2 || nf < 1 || t0 + 1 < t_min) return;
        const float2 *cs = reinterpret_cast<const float2 *>(taps4);
        u64 q0 = 0ull, q1 = 0ull;
        float vb = ring[ring_addr(64 + t0)];   // output t0 + 1 at tap 0
#pragma unroll 8
        for (int k = 0; k < kTapSlots; ++k) {
            const float va = ring[ring_addr(63 + t0 - k)];   // output t0 at tap k
            const float2 c = cs[2 * k];
            const u64 C = pack2(c.x, c.y);
            q0 = fma2(C, pack2(va, va), q0);
            q1 = fma2(C, pack2(vb, vb), q1);
            vb = va;
        }
        uint8_t *out = static_cast<uint8_t *>(fg.out[0]) + row_off;
        const int o = i0 - kLag + t0;
        float re, im;
        unpack2(q0, re, im);
        if (o >= 0 && o < nd && t0 >= t_min) out[o] = (uint8_t)code_of(fmaf(re, re, im * im), a2, b2);
        unpack2(q1, re, im);
        if (o + 1 >= 0 && o + 1 < nd) out[o + 1] = (uint8_t)code_of(fmaf(re, re, im * im), a2, b2);
    } else {
        constexpr int NP = G / 2;
        constexpr int TPP = kConsumers / NP;
        constexpr int BO = kTD / TPP;
        const int q = tid / TPP, bq = tid % TPP;
        const int fa = 2 * q, fb = 2 * q + 1;
        const float *ra = ring + fa * RS, *rb = ring + fb * RS;
        u64 re[BO], im[BO];
#pragma unroll
        for (int j = 0; j < BO; ++j) re[j] = im[j] = 0ull;
        for (int k = 0; k < kTapSlots; ++k) {
            const float4 t4 = taps4[k];
            const u64 C = pack2(t4.x, t4.y), S = pack2(t4.z, t4.w);
#pragma unroll
            for (int j = 0; j < BO; ++j) {
                const int a = ring_addr(63 + bq * BO + j - k);
                const u64 v = pack2(ra[a], rb[a]);
                re[j] = fma2(C, v, re[j]);
                im[j] = fma2(S, v, im[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < BO; ++j) {
            const int o = i0 - kLag + bq * BO + j;
            if (o < 0 || o >= nd || bq * BO + j < t_min) continue;
            const u64 qq = fma2(re[j], re[j], mul2(im[j], im[j]));
            float qa, qb;
            unpack2(qq, qa, qb);
            if (fa < nf) static_cast<uint8_t *>(fg.out[fa])[row_off + o] = (uint8_t)code_of(qa, a2, b2);
            if (fb < nf) static_cast<uint8_t *>(fg.out[fb])[row_off + o] = (uint8_t)code_of(qb, a2, b2);
        }
    }
}

// -------------------------------------------------------------------------------------------------
// MODE 0: write RF (float [n_lines][n_depth] per frame).
// MODE 1: envelope + log compression, write uint8 [n_lines][n_depth] per frame.
// MINB: resident CTAs per SM the registers are sized for (3 only for one-frame launches with
// at least three CTAs per SM of work; their shared memory allows it)
// SH: stage shape (rows_of, stages_of).
template <int G, int MODE, bool EXT, int MINB = 2, int SH = 0>
__global__ void __launch_bounds__(das_threads<G, MODE>(), MINB) das_kernel(const __grid_constant__ LaunchGroups L) {
    constexpr int kRows = rows_of(G, SH), kStages = stages_of(G, SH);
    static_assert(kStages <= kMaxStages, "barrier slots");
    constexpr int E = kRows / G;
    constexpr bool kTcFir = (MODE == 1 && G == 16);   // FIR on the tensor cores; whole lines only
    extern __shared__ __align__(128) unsigned char smem[];
    // a boundary kernel launched after this one as a programmatic dependent may be scheduled
    // now: its CTAs are small and wait (griddepcontrol.wait) for this grid's completion
    asm volatile("griddepcontrol.launch_dependents;");
    if constexpr (kTcFir) {
        if (L.n_seg > 1) {   // the host never splits these lines
            if (threadIdx.x == 0) set_status(SUPRA_EINVAL);
            return;
        }
    }
    int gi, line;
    const int n_seg = kTcFir ? 1 : max(L.n_seg, 1);
    const int item = kTcFir ? (int)blockIdx.x : (int)blockIdx.x / n_seg;
    locate_item(L, item, gi, line);
    const FrameGroup &fg = L.g[gi];
    const DevPlan *P = fg.plan;
    const int nf = min(fg.n, G);
    const int NT = P->n_tiles;
    const int nd = P->n_depth;
    // Depth segment: tiles [T0, T1) of the line emit their outputs.  With the envelope, the
    // FIR outputs within kLag of a segment boundary need RF from both sides: either a segment
    // after the first also beamforms the last kHalo depths of tile T0 - 1 (the FIR's leading
    // halo; its outputs belong to the previous segment), or, given boundary records, the
    // segments write the kHalo RF depths on their side of each boundary to its record and
    // leave the 64 outputs around it to boundary_fir_kernel.  The last segment runs the lag
    // tile after the last one.
    const int seg = kTcFir ? 0 : (int)blockIdx.x % n_seg;
    const int T0 = kTcFir ? 0 : seg * NT / n_seg, T1 = kTcFir ? NT : (seg + 1) * NT / n_seg;
    const bool records = !kTcFir && MODE == 1 && n_seg > 1 && L.bnd != nullptr;
    const int tb = (MODE == 1 && T0 > 0 && !records) ? T0 - 1 : T0;
    const int te = T1 + ((MODE == 1 && seg == n_seg - 1) ? 1 : 0);
    const SmemLayout lay(G, MODE, kSlotSamples, SH);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bars);
    uint64_t *empty = full + kMaxStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + lay.bars + 16 * kMaxStages);
    uint64_t *fir_bar = reinterpret_cast<uint64_t *>(smem + lay.bars + 72);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + lay.bars + 80);
    uint64_t *ring_bar = reinterpret_cast<uint64_t *>(smem + lay.bars + 88);
    ElemMeta *metas = reinterpret_cast<ElemMeta *>(smem + lay.meta);
    float4 *taps4 = reinterpret_cast<float4 *>(smem + lay.taps);
    float *ring = reinterpret_cast<float *>(smem + lay.ring);
    int16_t *stages = reinterpret_cast<int16_t *>(smem + lay.stage);
    constexpr int stage_elems = kRows * kSlotSamples;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumers / 32);
        }
        if (kTcFir) {
            mbar_init(fir_bar, 1);
            mbar_init(ring_bar, 1);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if constexpr (kTcFir) {
        if (warp == 0) {
            tc::tmem_alloc(tmem_slot, kFirTmemCols);
            tc::fence_before_sync();
        }
        // zero the halo and the first tile's positions; the tap-pair tables for the fill sit in the
        // last positions' bytes until the first tile's RF overwrites them
        for (int k = tid; k < (kTD / 8) * 512 / 4; k += (int)blockDim.x) reinterpret_cast<uint32_t *>(ring)[k] = 0u;
        fir_tc_build_pairs(P, reinterpret_cast<uint32_t *>(ring) + (kTD / 8) * 512 / 4);
    } else if (MODE == 1) {
        for (int k = tid; k < kTapSlots; k += (int)blockDim.x) {
            const float c = P->taps_c[k], s = P->taps_s[k];
            taps4[k] = G == 1 ? make_float4(c, s, c, s) : make_float4(c, c, s, s);
        }
        for (int k = tid; k < G * lay.ring_stride; k += (int)blockDim.x) ring[k] = 0.f;
    }
    const LineGeo lg = P->lines[line];
    __syncthreads();
    uint32_t tbase = 0;   // tensor memory of the FIR (kTcFir)
    if constexpr (kTcFir) {
        tc::fence_after_sync();
        tbase = *tmem_slot;
        if (warp < 4) {
            fir_tc_fill_taps(reinterpret_cast<const uint32_t *>(ring) + (kTD / 8) * 512 / 4, tbase, warp, tid & 31);
            tc::fence_before_sync();
        }
    }

    if (warp == kConsumers / 32) {
        // ------------------------------------------------------------------ producer warp
        const ProdConst C(P);
        const int lane = tid & 31;
        const float lip = fmaxf(fabsf(lg.dx), fabsf(lg.dy)) + fabsf(lg.dz) * C.inv2f;
        const bool halves = C.a1 > 1.0f + 1e-6f;
        // one-frame tiles of plans with a y window stage each row of the element box as its own
        // stage (when the row fits one), so that the consumers weigh y once per stage
        const bool y_win = G == 1 && !halves && P->row_y && (P->el_ny > 1 || P->ymax > P->ymin);
        bool rows = false;      // the current tile stages row by row
        int n = 0;              // stages issued
        int slot = 0;           // filled slots of stage n
        uint32_t bytes = 0;     // bytes of stage n this lane has put in flight
        bool ok = true;
        auto acquire = [&]() -> bool {   // stage n's buffer is free once consumers released stage n - kStages
            if (n < kStages) return true;
            const int sb = n % kStages;
            return __all_sync(0xffffffffu, wait_phase(&empty[sb], (uint32_t)(((n / kStages) - 1) & 1), abort_flag));
        };
        auto finalize = [&](bool last) {
            const int sb = n % kStages;
            ElemMeta *meta = metas + sb * kRows;
            // unused slots: zero geometry too (one-frame consumers apply every slot with weight 0,
            // and 0 times a delay made from uninitialised bytes could be NaN)
            if (lane >= slot && lane < E) meta[lane] = ElemMeta{};
            __syncwarp();
            if (lane == 0 && (last || rows)) meta[0].flags |= (last ? 8 : 0) | (rows ? kRowStage : 0);
            const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&full[sb], total);
            bytes = 0;
            slot = 0;
            ++n;
        };
        // With compounding, each tile is staged once per transmit of the line (same
        // aperture, that transmit's records and delays), as consecutive (tile, transmit)
        // passes; stages never mix transmits and only the tile's final pass marks its
        // last stage.  Without compounding there is one pass per tile.
        const int n_comp = EXT ? P->n_comp : 1;   // compile-time 1 for plans with a plain transmit model
        for (int vt = tb * n_comp; vt < T1 * n_comp && ok; ++vt) {
            const int tile = vt / n_comp, ci = vt - tile * n_comp;
            const bool final_ci = ci == n_comp - 1;
            const short4 b = __ldg(&C.ap_box[line * C.n_tiles + tile]);
            // a halo tile (before the segment's first) feeds the FIR its last kHalo depths only
            const int i_first = tile * kTD + (tile < T0 ? kTD - kHalo : 0);
            const int nbx = b.y - b.x + 1;
            const int nbox = nbx * (b.w - b.z + 1) * (halves ? 2 : 1);
            rows = y_win && nbx <= E;
            const int step = rows ? nbx : 32;   // items per producer pass: a row, or 32 lanes
            // Stage the active elements, E per stage, and mark the tile's last stage.  With a few
            // elements per stage (G >= 8) a full stage is handed over when the next element
            // needs a slot or the pass ends, so the last stage is known then; with many (a
            // stage of G < 8 frames empties fast) a first pass counts the stages, so that each
            // is handed over as soon as it is full.
            constexpr bool kDefer = G >= 8;
            int nst = 0, emitted = 0;
            if constexpr (!kDefer) {
                int nact = 0, nrows = 0;
                for (int jb = 0; jb < nbox; jb += step) {
                    int e, ia, ib;
                    float4 xe;
                    bool a = lane < step && element_range(C, lg, lip, b, tile, halves, jb + lane, e, xe, ia, ib);
                    if (tile < T0) a = a && ib >= i_first;
                    const int c = __popc(__ballot_sync(0xffffffffu, a));
                    nact += c;
                    nrows += c > 0 ? 1 : 0;
                }
                nst = max(1, rows ? nrows : (nact + E - 1) / E);
            }
            for (int jb = 0; jb < nbox && ok; jb += step) {
                int e, ia, ib;
                float4 xe;
                bool a = lane < step && element_range(C, lg, lip, b, tile, halves, jb + lane, e, xe, ia, ib);
                if (tile < T0) {   // halo tile: only depths from i_first on
                    a = a && ib >= i_first;
                    ia = max(ia, i_first);
                }
                ElemMeta m;
                int tx;
                if constexpr (EXT) {
                    TxTerm tt;
                    if (n_comp > 1) {
                        tt = P->txterms[line * n_comp + ci];
                    } else {
                        tt.b = lg.bt, tt.g = lg.gt, tt.tx = lg.tx, tt.plane = lg.plane;
                    }
                    tx = tt.tx;
                    if (a) element_window(C, lg, tt, ci, tile, ia, ib, xe, m);
                } else {
                    tx = lg.tx;
                    if (a) element_window_line(C, lg, tile, ia, ib, xe, m);
                }
                uint32_t mask = __ballot_sync(0xffffffffu, a);
                while (mask) {
                    if (kDefer && slot == E) finalize(false);   // more elements follow
                    if (slot == 0 && !acquire()) {
                        ok = false;
                        break;
                    }
                    const int take = min(E - slot, __popc(mask));
                    const int rank = __popc(mask & ((1u << lane) - 1u));
                    const bool mine = ((mask >> lane) & 1u) && rank < take;
                    if (mine) {
                        const int sb = n % kStages;
                        ElemMeta *meta = metas + sb * kRows;
                        meta[slot + rank] = m;
                        bytes += stage_element<G>(C, fg, nf, tx, e, m,
                                                  stages + sb * stage_elems + (slot + rank) * G * kSlotSamples,
                                                  &full[sb]);
                    }
                    // drop the `take` lowest lanes of the mask
                    for (int t = 0; t < take; ++t) mask &= mask - 1u;
                    slot += take;
                    if (!kDefer && slot == E) {
                        ++emitted;
                        finalize(final_ci && emitted == nst);
                    }
                }
                if (!kDefer && rows && ok && slot > 0) {   // the row's stage
                    ++emitted;
                    finalize(final_ci && emitted == nst);
                }
            }
            // the pass's last stage (an empty one when the tile's final pass staged nothing)
            if (ok && (slot > 0 || (final_ci && (kDefer || emitted == 0)))) {
                if (slot == 0 && !acquire()) {
                    ok = false;
                } else {
                    finalize(final_ci);
                }
            }
        }
        if (!ok) {
            *abort_flag = 1;
            set_status(SUPRA_ETIMEOUT);
            // let copies in flight land before the CTA's shared memory goes away
            for (int k = max(0, n - kStages); k < n; ++k)
                mbar_wait_bounded(&full[k % kStages], (uint32_t)((k / kStages) & 1), 1LL << 27);
        }
        return;
    }

    if constexpr (kTcFir) {
        if (warp == kConsumers / 32 + 1) {
            // ------------------------------------------------------------ FIR issuer (one lane)
            // tile n's products once the consumers have written its ring (ring_bar phase n)
            if ((tid & 31) == 0) {
                const uint32_t ring_saddr = tc::smem_u32(ring);
                for (int t = 0; t <= NT; ++t) {
                    if (!wait_phase(ring_bar, (uint32_t)(t & 1), abort_flag)) break;
                    tc::fence_after_sync();
                    if (t < NT) fir_tc_issue(tbase, ring_saddr, fir_bar);
                    else fir_tc_issue_block0(tbase, ring_saddr, fir_bar);
                }
            }
            return;
        }
    }

    // ---------------------------------------------------------------------- consumer warps
    const int m = tid;
    const bool use_y = P->el_ny > 1 || P->ymax > P->ymin;
    const bool halves = P->a1 > 1.0f + 1e-6f;   // as the producer decides it
    const float wa = P->win_a, wb = P->win_b;
    const float fsc = P->fsc;
    int sb = 0;                 // stage buffer of the next stage
    uint32_t parity = 0;        // its full-barrier phase parity
    bool aborted = false;
    for (int tile = tb; tile < te; ++tile) {
        const int i0 = tile * kTD;
        const int i = i0 + m;
        u64 acc2[G / 2 > 0 ? G / 2 : 1];
#pragma unroll
        for (int q = 0; q < (G / 2 > 0 ? G / 2 : 1); ++q) acc2[q] = 0ull;
        float acc1 = 0.f, wsum = 0.f;
        if (tile < T1) {
            const float r = P->depth0 + (float)i * P->depth_step;
            const float px = fmaf(r, lg.dx, lg.ox), py = fmaf(r, lg.dy, lg.oy), pz = fmaf(r, lg.dz, lg.oz);
            const float qx = fminf(fmaxf(px, P->xmin), P->xmax);
            const float qy = fminf(fmaxf(py, P->ymin), P->ymax);
            const float inv_a = 1.0f / fmaxf(pz * P->inv2f, P->amin);
            float base = P->tile_f[tile] + P->a1 * (float)m +
                         (EXT ? tx_excess(r, lg.bt, lg.gt, lg.plane) : path_excess(r, lg.bt, lg.gt)) * fsc;
            int cur = 0;   // compounding: transmit whose delay term `base` holds
            const int kt = P->tile_k[tile];
            for (;;) {
                bool ok = !aborted && mbar_try_wait_sleep(&full[sb], parity);
                if (!aborted && !__all_sync(0xffffffffu, ok)) {
                    ok = __all_sync(0xffffffffu, ok || wait_phase(&full[sb], parity, abort_flag));
                    if (!ok) {
                        aborted = true;
                        *abort_flag = 1;
                        set_status(SUPRA_ETIMEOUT);
                    }
                }
                if (aborted) break;
                const ElemMeta *meta = metas + sb * kRows;
                const int last = meta_last(meta[0]);
                if constexpr (EXT) {
                    const int ci = meta_comp(meta[0]);
                    if (ci != cur) {
                        const int nc = P->n_comp;
                        const TxTerm tt = P->txterms[line * nc + ci];
                        base = P->tile_f[tile] + P->a1 * (float)m + tx_excess(r, tt.b, tt.g, tt.plane) * fsc;
                        cur = ci;
                    }
                }
                // a halo tile's depths before its last kHalo are not needed (warp-uniform)
                if (tile >= T0 || warp >= (kTD - kHalo) / 32)
                    consume_stage<G, SH>(stages + sb * stage_elems, meta, i, r, qx, qy, inv_a, base, kt, use_y, wa, wb,
                                     fsc, acc2, acc1, wsum, halves, nd);
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&empty[sb]);
                if (++sb == kStages) {
                    sb = 0;
                    parity ^= 1u;
                }
                if (last) break;
            }
        }
        if (consumer_sync_or(aborted ? 1 : 0)) {
            if constexpr (kTcFir) {
                if (warp == 0) {
                    // the previous tile's products may still be in flight
                    if (tile > 0) mbar_wait_bounded(fir_bar, (uint32_t)((tile - 1) & 1), 1LL << 27);
                    tc::fence_after_sync();
                    tc::tmem_free(tbase, kFirTmemCols);
                }
            }
            return;
        }
        const bool act = (tile < NT) && (i < nd);
        const float inv = wsum > 0.f ? 1.0f / wsum : 0.f;
        float v[G];
        if constexpr (G == 1) {
            v[0] = act ? acc1 * inv : 0.f;
        } else {
#pragma unroll
            for (int q = 0; q < G / 2; ++q) {
                float a, b;
                unpack2(acc2[q], a, b);
                v[2 * q] = act ? a * inv : 0.f;
                v[2 * q + 1] = act ? b * inv : 0.f;
            }
        }
        if (MODE == 0) {
            if (act) {
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (g < nf) static_cast<float *>(fg.out[g])[(long long)line * nd + i] = v[g];
            }
        } else if constexpr (kTcFir) {
            // The FIR of tile n runs on the tensor cores while the consumers beamform tile n + 1;
            // its codes are written after that (one accumulator set suffices: they are read out
            // before the next products are issued).
            unsigned char *ring16 = reinterpret_cast<unsigned char *>(ring);
            bool prev = false;
            if (tile > 0) {
                prev = fir_tc_wait(fir_bar, tile - 1, abort_flag, aborted);
                // keep the last kHalo positions (bytes 512 kTD / 8 ..) as the next tile's leading
                // halo: 4096 B, 16 B per thread
                const uint4 x = *reinterpret_cast<const uint4 *>(ring16 + (kTD / 8) * 512 + 16 * m);
                consumer_sync();   // every thread has read the previous tile's ring
                *reinterpret_cast<uint4 *>(ring16 + 16 * m) = x;
            }
            ring16_put(ring16, kHalo + m, v);
            tc::fence_async_smem();
            if (prev) {
                tc::fence_after_sync();
                fir_tc_epilogue(tbase, fg, nf, (long long)line * nd, i0 - kTD, nd, P->log_a2,
                                P->log_b2 - kFirLog2Scale2 * P->log_a2);
            }
            tc::fence_before_sync();
            consumer_sync();   // ring written, accumulators read out
            if (tid == 0) mbar_arrive(ring_bar);
        } else {
            const int a = ring_addr(kHalo + m);
#pragma unroll
            for (int g = 0; g < G; ++g) ring[g * lay.ring_stride + a] = v[g];
            consumer_sync();
            const bool head = records && tile == T0 && seg > 0;           // RF depths B .. B + 63
            const bool tail = records && tile == T1 - 1 && seg < n_seg - 1; // RF depths B' - 64 .. B' - 1
            if (head || tail) {
                // record of boundary b: slot u holds RF depth B_b - 64 + u (u < 128), as ring
                // position u does in the tile that starts at B_b
                const long long nb = n_seg - 1;
                for (int k = m; k < nf * 2 * kHalo; k += kConsumers) {
                    const int g = k / (2 * kHalo), j = k % (2 * kHalo);
                    const bool hd = j < kHalo;
                    if (hd ? !head : !tail) continue;
                    const long long rec = (((long long)item * G + g) * nb + (hd ? seg - 1 : seg)) * (2 * kHalo);
                    const int u = hd ? kHalo + j : j - kHalo;   // record slot
                    const int p = hd ? kHalo + j : kTD + (j - kHalo);   // ring position
                    if (SUPRA_CHECK(rec + u < L.bnd_floats)) L.bnd[rec + u] = ring[g * lay.ring_stride + ring_addr(p)];
                }
            }
            if (tile >= T0)   // a halo tile's outputs belong to the previous segment
                fir_log_tile_generic<G>(fg, nf, line, i0, nd, ring, lay.ring_stride, taps4, P->log_a2, P->log_b2,
                                        head ? kHalo : 0);
            consumer_sync();
            // keep the last kHalo RF samples as the next tile's leading halo
            for (int k = m; k < G * kHalo; k += kConsumers) {
                const int g = k / kHalo, j = k % kHalo;
                ring[g * lay.ring_stride + ring_addr(j)] = ring[g * lay.ring_stride + ring_addr(kTD + j)];
            }
            consumer_sync();
        }
    }
    if constexpr (kTcFir) {
        // the last tile's FIR
        if (fir_tc_wait(fir_bar, NT, abort_flag, aborted)) {
            tc::fence_after_sync();
            fir_tc_epilogue(tbase, fg, nf, (long long)line * nd, NT * kTD, nd, P->log_a2,
                            P->log_b2 - kFirLog2Scale2 * P->log_a2);
        }
        tc::fence_before_sync();
        consumer_sync();
        if (warp == 0) {
            tc::fence_after_sync();
            tc::tmem_free(tbase, kFirTmemCols);
        }
    }
}

// The 64 outputs around each depth-segment boundary of a B-mode launch with boundary
// records (one CTA of 64 threads per line and boundary, frames in turn): output
// B - kLag + t from record slots 63 + t - k' with the taps, in the order, and the log code
// of fir_log_tile_generic, so that the codes are those of an unsegmented launch bit for bit.
constexpr int kBoundaryThreads = 2 * kLag;
__global__ void __launch_bounds__(kBoundaryThreads) boundary_fir_kernel(const __grid_constant__ LaunchGroups L, int G) {
    __shared__ float rec_s[2 * kHalo];
    __shared__ float2 taps_s[kTapSlots];
    const int nb = L.n_seg - 1;
    if (nb < 1) return;
    const int item = (int)blockIdx.x / nb, b = (int)blockIdx.x % nb;
    int gi, line;
    locate_item(L, item, gi, line);
    const FrameGroup &fg = L.g[gi];
    const DevPlan *P = fg.plan;
    const int nf = min(fg.n, G), nd = P->n_depth;
    const int B = (b + 1) * P->n_tiles / L.n_seg * kTD;   // first depth of segment b + 1
    const int t = threadIdx.x, o = B - kLag + t;
    for (int k = t; k < kTapSlots; k += kBoundaryThreads) taps_s[k] = make_float2(P->taps_c[k], P->taps_s[k]);
    // launched as a programmatic dependent of the beamforming kernel: its records (and its
    // other outputs) are complete and visible after this wait (a no-op in a plain launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int f = 0; f < nf; ++f) {
        const long long rec = (((long long)item * G + f) * nb + b) * (2 * kHalo);
        __syncthreads();
        for (int u = t; u < 2 * kHalo; u += kBoundaryThreads)
            rec_s[u] = SUPRA_CHECK(rec + u < L.bnd_floats) ? L.bnd[rec + u] : 0.0f;
        __syncthreads();
        float re = 0.f, im = 0.f;
#pragma unroll 16
        for (int k = 0; k < kTapSlots; ++k) {
            const float v = rec_s[63 + t - k];
            const float2 c = taps_s[k];
            re = fmaf(c.x, v, re);
            im = fmaf(c.y, v, im);
        }
        if (o < nd)
            static_cast<uint8_t *>(fg.out[f])[(long long)line * nd + o] =
                (uint8_t)code_of(fmaf(re, re, im * im), P->log_a2, P->log_b2);
    }
}

}  // namespace supra
