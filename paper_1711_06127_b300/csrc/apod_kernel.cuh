// apod_kernel.cuh -- learned apodization: a per-pixel network that maps the
// delayed channel samples of the aperture to softmax-normalised element
// weights.  Not in the paper; it stands in for the exact minimum-variance
// beamformer (it is trained on MV outputs) at delay-and-sum cost.
//
//   xh = x / ||x||,  h1 = relu(W1 xh + b1),  h2 = relu(W2 h1 + b2),
//   z = W3 h2 + b3,  w = softmax of z over the aperture,  y = sum_e w_e x_e.
//
// A CTA works on tiles of 128 pixels; pixel p of a tile is TMEM lane p of every
// M = 128 accumulator, and its row is held by the threads p, p + 128, ... (one
// part of its columns each; one warpgroup for the forward pass on stored rows,
// two for training and the fused beamformer, training adding a warp that only
// issues the products).  The three layers and, in training, the two
// activation-gradient products and the three weight-gradient products run as
// BF16 tcgen05 MMAs with FP32 accumulators in tensor memory; ReLU, the masked
// softmax and its backward pass run per thread between them.
// Weight gradients accumulate in tensor memory across all tiles of a CTA and
// are written once, as per-CTA partials (deterministic reduction afterwards).
//
// Bias gradients come from the same MMAs: the B operands of the weight-gradient
// products carry 16 extra columns of ones ([H2 | 1], [H1 | 1], [X | 1]), so the
// accumulator column past the weights is sum over pixels of the output
// gradient.  The 64-row weight-gradient products (dW2, dW1) are issued with
// M = 128; rows 64..127 read the next buffer and are discarded.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "gather.cuh"
#include "tc.cuh"

namespace supra {
namespace apod {

constexpr int kIn = 128, kH1 = 64, kH2 = 64, kTile = 128;
// flat parameter vector: W1 [64][128], b1, W2 [64][64], b2, W3 [128][64], b3
constexpr int kOffW1 = 0, kOffB1 = 8192, kOffW2 = 8256, kOffB2 = 12352, kOffW3 = 12416, kOffB3 = 20608;
constexpr int kParams = 20736;
constexpr int kPartStride = kParams + 4;   // + loss sum, valid-pixel count (rows 16-byte aligned)
enum { kForward = 0, kTrain = 1, kInfer = 2 };

// Shared-memory images, byte offsets.  A "[rows][cols] buffer" keeps 16-byte
// chunks of 8 columns: chunk j of row r at j * 2048 + r * 16 (128 rows).
template <int MODE>
struct Smem {
    static constexpr bool T = MODE == kTrain;
    static constexpr int W1 = 0;        // [hid1][in]:  chunk j of row n at j * 1024 + n * 16
    static constexpr int W2 = 16384;    // [hid2][hid1]: j * 1024 + n * 16
    static constexpr int W3 = 24576;    // [out][hid2]:  j * 2048 + n * 16
    static constexpr int X = 40960;     // [pix][in] (+ 2 chunks of ones when training)
    static constexpr int H1 = X + (T ? 36864 : 32768);   // [pix][hid1] (+ 2 chunks of ones)
    static constexpr int H2 = H1 + (T ? 20480 : 16384);  // [pix][hid2] (+ 2 chunks of ones)
    static constexpr int DZ2 = H2 + (T ? 20480 : 16384); // [pix][hid2]
    static constexpr int DZ1 = DZ2 + (T ? 16384 : 0);    // [pix][hid1]
    static constexpr int DZ3 = DZ1 + (T ? 16384 : 0);    // [pix][out]
    static constexpr int BIAS = DZ3 + (T ? 32768 : 0);   // float b1[64], b2[64], b3[128]
    static constexpr int X2 = BIAS + 256 * 4;            // training: the next tile's [pix][in] (+ ones)
    static constexpr int TOTAL = X2 + (T ? 36864 : 0);
};
static_assert(Smem<kTrain>::TOTAL <= 227 * 1024, "training tile exceeds shared memory");
static_assert(2 * (Smem<kInfer>::TOTAL + 1024) <= 228 * 1024, "two inference CTAs per SM");
// dW2 / dW1 read 128 rows (32 KB) from DZ2 / DZ1: the next buffers must follow
static_assert(Smem<kTrain>::DZ1 == Smem<kTrain>::DZ2 + 16384 && Smem<kTrain>::DZ3 == Smem<kTrain>::DZ1 + 16384,
              "padded weight-gradient operands");

// tensor-memory columns
constexpr uint32_t kT64 = 0, kT128 = 64, kDW3 = 192, kDW2 = 272, kDW1 = 352;

struct Args {
    int rows_tma;          // kTrain: the feature rows come through the kernel's tensor map (else cp.async)
    const float *params;
    // kForward / kTrain: feature rows (bf16 [.][128]), masks (u32 [.][4]), norms, labels
    const uint16_t *feat;
    const uint32_t *mask;
    const float *norm;
    const float *label;
    long long n, stride;   // pixels; rows between consecutive pixels of a tile
    long long tile_stride; // rows between the first pixels of consecutive 128-pixel tiles
    float *y;              // kForward: y = ||x|| * yh per pixel
    float *partial;        // kTrain: [gridDim.x][kPartStride]
    // kInfer
    const DevPlan *plan;
    const int16_t *ch;
    float *rf;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint4 pack8(const float *v) {
    return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}
__device__ __forceinline__ void unpack8(uint4 u, float *v) {
    v[0] = bf_lo(u.x), v[1] = bf_hi(u.x), v[2] = bf_lo(u.y), v[3] = bf_hi(u.y);
    v[4] = bf_lo(u.z), v[5] = bf_hi(u.z), v[6] = bf_lo(u.w), v[7] = bf_hi(u.w);
}
// 2^x (the special-function unit's approximation; exp(z) = 2^(z log2 e))
constexpr float kLog2e = 1.44269504088896341f;
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// mk[i] for a run-time i < 4 by selects (indexing the array at run time would put it in local memory)
__device__ __forceinline__ uint32_t word_of(const uint32_t (&mk)[4], int i) {
    return i == 0 ? mk[0] : i == 1 ? mk[1] : i == 2 ? mk[2] : mk[3];
}
__device__ __forceinline__ uint4 &chunk(unsigned char *sm, int buf, int j, int row) {
    return *reinterpret_cast<uint4 *>(sm + buf + j * 2048 + row * 16);
}
// pack_bf16(max(lo, 0), max(hi, 0)): the conversion's ReLU (rounding keeps the sign, so rounding and
// clamping commute)
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// A layer's activations for this thread's BW columns: relu(v * scale + bias) in BF16 into
// chunks c0.. of row `row` of a buffer, two columns per packed FMA.
template <int BW>
__device__ __forceinline__ void bias_relu_rows(const float (&v)[BW], const float *bias, float scale,
                                               unsigned char *sm, int buf, int c0, int row) {
    const u64 S2 = pack2(scale, scale);
    const float4 *b4 = reinterpret_cast<const float4 *>(bias);
#pragma unroll
    for (int c = 0; c < BW / 8; ++c) {
        const float4 ba = b4[2 * c], bb = b4[2 * c + 1];
        const float bj[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float lo, hi;
            unpack2(fma2(pack2(v[8 * c + 2 * u], v[8 * c + 2 * u + 1]), S2, pack2(bj[2 * u], bj[2 * u + 1])), lo, hi);
            w[u] = pack_bf16_relu(lo, hi);
        }
        chunk(sm, buf, c0 + c, row) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// A ReLU layer's pre-activation gradient for this thread's BW columns: v where the layer's stored
// output h (BF16, >= 0) is positive, else 0, in BF16.  Per BF16 pair of h, bit 15 of each 16-bit
// lane of (h & 0x7fff7fff) + 0x7fff7fff is set exactly when that lane is not zero (no carry
// crosses lanes), and a byte permute replicates it over the lane: a mask for the packed gradient.
template <int BW>
__device__ __forceinline__ void relu_grad_rows(const float (&v)[BW], unsigned char *sm, int hbuf, int dbuf, int c0,
                                               int row) {
#pragma unroll
    for (int c = 0; c < BW / 8; ++c) {
        const uint4 h = chunk(sm, hbuf, c0 + c, row);
        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t nz = (hw[u] & 0x7fff7fffu) + 0x7fff7fffu;
            uint32_t m;
            asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(m) : "r"(nz));
            w[u] = pack_bf16(v[8 * c + 2 * u], v[8 * c + 2 * u + 1]) & m;
        }
        chunk(sm, dbuf, c0 + c, row) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}
// 3D tiled tensor copy global -> shared, completion counted on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
        : "memory");
}

// 16-byte global -> shared copy that completes asynchronously (cp.async), and its waits
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Element range of (line, depth tile): the tile's element box (conservative: elements
// outside it are outside the aperture at every depth of the tile, their samples are 0),
// as the contiguous index range from its first to its last element (e = iy * nx + ix;
// a superset on matrix arrays, whose extra elements fail the per-sample aperture test).
struct ElemBox {
    int lo, hi;
    __device__ __forceinline__ bool has(int e) const { return e >= lo && e <= hi; }
    __device__ __forceinline__ bool any(int e0, int e1) const { return e1 >= lo && e0 <= hi; }
};
__device__ __forceinline__ ElemBox elem_box(const DevPlan *__restrict__ P, int line, int i) {
    const short4 b = __ldg(&P->ap_box[line * P->n_tiles + i / kTD]);
    return ElemBox{b.z * P->el_nx + b.x, b.w * P->el_nx + b.y};
}

// ---- fused beamformer: the tile's sample windows staged in shared memory.
// Per tile (128 depths of one line, inside one 256-depth delay tile), slot j holds samples
// [ws_j, ws_j + kWinW) of the record of element box.lo + j (zero outside the record), ws_j a
// multiple of 8.  The window bounds the two-way delay over the tile's depths as the
// delay-and-sum producer does (the delay at the first and last depth and, where a path has its
// minimum inside, the sum of the paths' minima; one sample before, two after).  Elements past
// the last slot, windows wider than kWinW, plane-wave lines and unaligned records are not
// staged (kNoWin): their samples come from global memory, so the values are the same.
constexpr int kWinW = 144, kWinSlots = 32768 / (kWinW * 2), kNoWin = -0x40000000;

// Also returns the element's receive terms beta = d.(o - x_e), gamma = |o - x_e|^2 (per line and
// element, shared by the tile's pixels).
__device__ __forceinline__ int tile_window(const DevPlan *__restrict__ P, const LineGeo &lg, int e, int i_a, int i_b,
                                           float &beta, float &gamma) {
    const float4 xe = __ldg(&P->elem[e]);
    const float mx = lg.ox - xe.x, my = lg.oy - xe.y, mz = lg.oz - xe.z;
    beta = lg.dx * mx + lg.dy * my + lg.dz * mz;
    gamma = mx * mx + my * my + mz * mz;
    const int tile = i_a / kTD;
    const int kt = __ldg(&P->tile_k[tile]);
    const float ft = __ldg(&P->tile_f[tile]);
    const float r0 = P->depth0 + (float)i_a * P->depth_step, r1 = P->depth0 + (float)i_b * P->depth_step;
    const float s0 = ft + P->a1 * (float)(i_a - tile * kTD) + (path_excess(r0, lg.bt, lg.gt) + path_excess(r0, beta, gamma)) * P->fsc;
    const float s1 = ft + P->a1 * (float)(i_b - tile * kTD) + (path_excess(r1, lg.bt, lg.gt) + path_excess(r1, beta, gamma)) * P->fsc;
    float lo = fminf(s0, s1), hi = fmaxf(s0, s1);
    if ((-beta > r0 && -beta < r1) || (-lg.bt > r0 && -lg.bt < r1)) {
        const float re = fminf(fmaxf(-beta, r0), r1), rt = fminf(fmaxf(-lg.bt, r0), r1);
        const float de = sqrtf(fmaxf(fmaf(re, re + 2.0f * beta, gamma), 0.0f));
        const float dtp = sqrtf(fmaxf(fmaf(rt, rt + 2.0f * lg.bt, lg.gt), 0.0f));
        lo = fminf(lo, (de + dtp) * P->fsc - P->t0fs - (float)kt);
    }
    const int lo_i = kt + (int)floorf(lo) - 1;
    const int ws = (lo_i >> 3) << 3;
    const int need = kt + (int)floorf(hi) + 2 - ws;
    return need <= kWinW ? ws : kNoWin;
}

// element_sample with the element's receive terms given and the two samples read from the
// staged window when it holds them.  The sample is formed for depths outside the aperture too
// (and then weighted 0): the lanes of a warp are consecutive depths of one element, which
// enter the aperture at different depths, and a branch on it would only serialise them.  The
// window covers the delays of every depth of the tile, so those lanes read inside it as well.
// Y: the array has more than one row of elements (else the aperture's y test always passes).
template <bool Y>
__device__ __forceinline__ float element_sample_staged(const DevPlan *__restrict__ P, const PixelGeo &g, int e,
                                                       bool &act, const int16_t *win, int ws, float beta,
                                                       float gamma, float ex, float ey) {
    act = fabsf((ex - g.qx) * g.inv_a) <= 1.0f && (!Y || fabsf((ey - g.qy) * g.inv_a) <= 1.0f);
    const float s = g.base + path_excess(g.r, beta, gamma) * P->fsc;
    int ks;
    const float fl = floor_split(s, ks);   // (|s| is far below 2^22 for the tile's depths)
    const float phi = s - fl;
    const int k = g.kt + ks;               // (sample indices of a record: far below 2^31)
    const int d = k - ws;
    float x0, x1;
    if (d >= 0 && d + 1 < kWinW) {   // int16 -> float exactly, without the conversion pipe
        const uint16_t *w16 = reinterpret_cast<const uint16_t *>(win) + d;
        x0 = __uint_as_float(biased(w16[0])) - kMagic;
        x1 = __uint_as_float(biased(w16[1])) - kMagic;
    } else {
        const int n_s = P->n_s;
        const int16_t *rec = g.rec0 + (long long)e * n_s;
        x0 = (k >= 0 && k < n_s) ? (float)__ldg(rec + k) : 0.0f;
        x1 = (k + 1 >= 0 && k + 1 < n_s) ? (float)__ldg(rec + k + 1) : 0.0f;
    }
    return act ? fmaf(phi, x1 - x0, x0) : 0.0f;
}

// K steps of one MMA chain, issued by one thread (2 core matrices along K per step).
// (The descriptors of successive K steps differ only in their start-address field, by
// 2 * lbo / 16 per step, which stays inside the field for addresses below 256 KB.)
__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a, uint32_t a_lbo, uint32_t a_sbo, uint32_t b,
                                          uint32_t b_lbo, uint32_t b_sbo, uint32_t idesc, int ksteps, bool acc) {
    const uint64_t da = tc::smem_desc(a, a_lbo, a_sbo), db = tc::smem_desc(b, b_lbo, b_sbo);
    const uint64_t ia = (uint64_t)((2u * a_lbo) >> 4), ib = (uint64_t)((2u * b_lbo) >> 4);
#pragma unroll
    for (int s = 0; s < ksteps; ++s) tc::mma_bf16(d, da + s * ia, db + s * ib, idesc, acc || s > 0);
}

// Weights [n][i] (row-major, i fastest) of one matrix into its shared-memory image: element
// (n, i) at img + (i / 8) * jstride + n * 16 + (i % 8) * 2, rounded to BF16.  Four consecutive
// weights per thread and load (16-byte loads, all of a thread's loads in flight at once) when the
// parameter vector is 16-byte aligned, one otherwise.
template <int LOG2_IN>
__device__ __forceinline__ void stage_matrix(const float *__restrict__ w, int count, unsigned char *img, int jstride,
                                             bool vec, int t, int nt) {
    constexpr int kRow = 1 << LOG2_IN;
    if (vec) {
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
#pragma unroll 4
        for (int k4 = t; k4 < count / 4; k4 += nt) {
            const float4 q = __ldg(w4 + k4);
            const int k = 4 * k4, n = k >> LOG2_IN, i = k & (kRow - 1);
            *reinterpret_cast<uint2 *>(img + (i >> 3) * jstride + n * 16 + (i & 7) * 2) =
                make_uint2(pack_bf16(q.x, q.y), pack_bf16(q.z, q.w));
        }
    } else {
#pragma unroll 8
        for (int k = t; k < count; k += nt) {
            const int n = k >> LOG2_IN, i = k & (kRow - 1);
            *reinterpret_cast<__nv_bfloat16 *>(img + (i >> 3) * jstride + n * 16 + (i & 7) * 2) =
                __float2bfloat16_rn(__ldg(w + k));
        }
    }
}

// Threads per CTA: training and the fused beamformer split every pixel row over
// two warpgroups (warps w and w + 4 share TMEM lanes 32 (w % 4).., each takes
// half of every row's columns; in the beamformer each half gathers the elements
// whose weights it computes), so that two warps per scheduler hide each other's
// TMEM, shared-memory and MMA waits; the forward pass on stored rows keeps one
// warpgroup.  The kernel takes any power-of-two number of parts H = compute
// threads / 128 up to 4 (a training split over four measured the same per tile).
// Training adds one warp that only issues the tensor-core products (an MMA
// instruction holds its issuing thread for tens of cycles, which the pixel
// warps would otherwise wait for at the next barrier).
template <int MODE>
__host__ __device__ constexpr int apod_compute_threads() { return MODE == kForward ? 128 : 256; }
template <int MODE>
__host__ __device__ constexpr int apod_threads() { return apod_compute_threads<MODE>() + (MODE == kTrain ? 32 : 0); }

// Barrier of the H warps whose threads hold the parts of the same pixel rows (warps w, w + 4, ...:
// the same tensor-memory lanes); named barriers 1..4, one per lane quarter.
template <int H>
__device__ __forceinline__ void row_parts_sync(int warp) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (warp & 3)), "r"(32 * H) : "memory");
}

// The three matrices staged by the 256 threads of the training kernel with all of a thread's
// 16-byte loads in flight at once (20 per thread), then their BF16 images; the same values as
// stage_matrix.
template <int LOG2_IN, int COUNT, int NT, int N0>
__device__ __forceinline__ void put_matrix(const float4 (&q)[20], unsigned char *img, int jstride, int t) {
    constexpr int kRow = 1 << LOG2_IN;
#pragma unroll
    for (int j = 0; j < COUNT / 4 / NT; ++j) {
        const int k = 4 * (t + j * NT), n = k >> LOG2_IN, i = k & (kRow - 1);
        *reinterpret_cast<uint2 *>(img + (i >> 3) * jstride + n * 16 + (i & 7) * 2) =
            make_uint2(pack_bf16(q[N0 + j].x, q[N0 + j].y), pack_bf16(q[N0 + j].z, q[N0 + j].w));
    }
}

template <int MODE>
__device__ __forceinline__ void stage_weights(const float *__restrict__ prm, unsigned char *sm, int t, int nt) {
    using S = Smem<MODE>;
    // the matrices start at multiples of four floats, so one alignment test covers them
    const bool vec = (reinterpret_cast<uintptr_t>(prm) & 15) == 0;
    constexpr int NT = apod_compute_threads<MODE>();
    if constexpr (MODE == kTrain && NT == 256) {   // (the inference kernel's registers have no room for 20)
        constexpr int n1 = kH1 * kIn / 4 / NT, n2 = kH2 * kH1 / 4 / NT, n3 = kIn * kH2 / 4 / NT;
        static_assert(n1 + n2 + n3 == 20, "loads per thread");
        if (vec && nt == NT) {
            float4 q[20];
            const float4 *w1 = reinterpret_cast<const float4 *>(prm + kOffW1) + t;
            const float4 *w2 = reinterpret_cast<const float4 *>(prm + kOffW2) + t;
            const float4 *w3 = reinterpret_cast<const float4 *>(prm + kOffW3) + t;
#pragma unroll
            for (int j = 0; j < n1; ++j) q[j] = __ldg(w1 + j * NT);
#pragma unroll
            for (int j = 0; j < n2; ++j) q[n1 + j] = __ldg(w2 + j * NT);
#pragma unroll
            for (int j = 0; j < n3; ++j) q[n1 + n2 + j] = __ldg(w3 + j * NT);
            const float bv = t < 64 ? prm[kOffB1 + t] : t < 128 ? prm[kOffB2 + t - 64] : prm[kOffB3 + t - 128];
            put_matrix<7, kH1 * kIn, NT, 0>(q, sm + S::W1, 1024, t);
            put_matrix<6, kH2 * kH1, NT, n1>(q, sm + S::W2, 1024, t);
            put_matrix<6, kIn * kH2, NT, n1 + n2>(q, sm + S::W3, 2048, t);
            reinterpret_cast<float *>(sm + S::BIAS)[t] = bv;
            return;
        }
    }
    stage_matrix<7>(prm + kOffW1, kH1 * kIn, sm + S::W1, 1024, vec, t, nt);
    stage_matrix<6>(prm + kOffW2, kH2 * kH1, sm + S::W2, 1024, vec, t, nt);
    stage_matrix<6>(prm + kOffW3, kIn * kH2, sm + S::W3, 2048, vec, t, nt);
    float *bias = reinterpret_cast<float *>(sm + S::BIAS);
    for (int k = t; k < 256; k += nt)
        bias[k] = k < 64 ? prm[kOffB1 + k] : k < 128 ? prm[kOffB2 + k - 64] : prm[kOffB3 + k - 128];
}

// Wait for the next commit of the MMA barrier; false after ~1 s.
__device__ __forceinline__ bool mma_wait(uint64_t *bar, uint32_t &phase) {
    const bool ok = mbar_wait_bounded(bar, phase & 1u, 1LL << 31);
    ++phase;
    tc::fence_after_sync();
    return ok;
}


// This thread's columns of a 64-wide accumulator: H parts of 64 / H columns, read in blocks of up to 32.
template <int B>
__device__ __forceinline__ void tmem_ld_block(uint32_t taddr, float (&v)[B]) {
    if constexpr (B == 32) tc::tmem_ld32(taddr, v);
    else tc::tmem_ld16(taddr, v);
}

template <int MODE>
__global__ void __launch_bounds__(apod_threads<MODE>(), MODE == kTrain ? 1 : 2) apod_kernel(const Args a, const __grid_constant__ CUtensorMap rows_map) {
    using S = Smem<MODE>;
    // NC threads own the pixel rows (H parts per row); training adds the issuing warp
    constexpr int NT = apod_threads<MODE>(), NC = apod_compute_threads<MODE>(), H = NC / kTile;
    constexpr uint32_t kCols = MODE == kTrain ? 512 : 256;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t bar_dw1;   // training: completion of weight-gradient products (never waited on)
    __shared__ __align__(8) uint64_t bar_rows;  // training with rows_tma: the next tile's feature rows have landed
    __shared__ uint32_t tmem_base;
    __shared__ float red[2][NC / 32];
    __shared__ float xrow[H > 1 ? 3 : 1][H][kTile];   // per-row partials of the softmax (max, sum, weighted sum)
    __shared__ int win_ws[MODE == kInfer ? kWinSlots : 1];   // fused beamformer: staged window starts
    __shared__ float win_bg[MODE == kInfer ? kWinSlots : 1][2];   // and the elements' beta, gamma
    const int t = threadIdx.x, warp = t >> 5;
    const int row = t & (kTile - 1), half = t / kTile;
    const bool issuer = MODE == kTrain && t >= NC;   // the warp that issues the products
    // (training: the issuing warp's lane 0, which then starts the first tile's row copy)
    if (t == (MODE == kTrain ? NC : 0)) {
        mbar_init(&bar, 1);
        mbar_init(&bar_dw1, 1);
        mbar_init(&bar_rows, 1);
        fence_mbar_init();
        if (MODE == kTrain && a.rows_tma)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&rows_map)) : "memory");
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, kCols);
    // Training: the next tile's feature rows are copied into the other X buffer while this
    // tile runs -- by the tensor-copy engine (one 3D copy that the issuing warp starts,
    // completing on bar_rows), else per thread (cp.async); its masks, norms and labels wait in
    // registers.  The copy into a buffer starts once the next Z2 products are complete (the
    // issuing warp: after the barrier that follows their wait): the dW1 products of the tile
    // before, which read that buffer, are issued right after the next Z1 products, so the
    // commit that signals Z2 covers them too (one thread issues all products).  With the copy
    // engine, rows past the pixel count keep whatever lands (real rows or the map's zero fill):
    // they are masked out (no weight, no loss, a zero output gradient), as zeroed rows would be.
    uint32_t nmk[4] = {0u, 0u, 0u, 0u};
    float nnrm = 0.0f, nlab = 0.0f;   // raw loads: nothing uses them before the next tile
    bool nok = false;
    uint32_t rows_phase = 0;          // completions of bar_rows waited for
    bool rows_armed = false;          // a copy engine prefetch is in flight
    auto prefetch = [&](long long tl, int xo) {
        const long long pp = tl * kTile + row;
        nok = pp < a.n;
        const long long rw = tl * a.tile_stride + (long long)row * a.stride;
        if (MODE == kTrain && a.rows_tma) {   // (the issuing warp starts the copy)
            rows_armed = true;
            if (nok) {
                const uint4 m4 = __ldg(reinterpret_cast<const uint4 *>(a.mask) + rw);
                nmk[0] = m4.x, nmk[1] = m4.y, nmk[2] = m4.z, nmk[3] = m4.w;
                nnrm = __ldg(a.norm + rw);
                nlab = __ldg(a.label + rw);
            } else {
                nmk[0] = nmk[1] = nmk[2] = nmk[3] = 0u;
                nnrm = nlab = 0.0f;
            }
            return;
        }
        if (nok) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.feat + rw * kIn);
#pragma unroll
            for (int c = half * (16 / H); c < (half + 1) * (16 / H); ++c) cp_async16(&chunk(sm, xo, c, row), src + c);
            const uint4 m4 = __ldg(reinterpret_cast<const uint4 *>(a.mask) + rw);
            nmk[0] = m4.x, nmk[1] = m4.y, nmk[2] = m4.z, nmk[3] = m4.w;
            nnrm = __ldg(a.norm + rw);
            nlab = __ldg(a.label + rw);
        } else {
#pragma unroll
            for (int c = half * (16 / H); c < (half + 1) * (16 / H); ++c) chunk(sm, xo, c, row) = make_uint4(0u, 0u, 0u, 0u);
            nmk[0] = nmk[1] = nmk[2] = nmk[3] = 0u;
            nnrm = nlab = 0.0f;
        }
        cp_async_commit();
    };
    // one copy of a tile's 128 rows in the chunked layout (the issuing warp's lane 0)
    auto copy_rows = [&](long long tl, int xo) {
        tc::fence_async_smem();   // this buffer's last generic reads precede the copy
        mbar_arrive_expect_tx(&bar_rows, (uint32_t)(kTile * kIn * 2));
        tma_load_3d(&chunk(sm, xo, 0, 0), &rows_map, 0, (int)(tl * a.tile_stride / a.stride), 0, &bar_rows);
    };
    // the first tile's rows are requested before the weights are staged (the two latencies overlap)
    if (MODE == kTrain && (long long)blockIdx.x < (a.n + kTile - 1) / kTile) {
        if (!issuer) prefetch(blockIdx.x, S::X);
        else if (a.rows_tma && (t & 31) == 0) copy_rows(blockIdx.x, S::X);
    }
    if (!issuer) stage_weights<MODE>(a.params, sm, t, NC);
    if (MODE == kTrain && !issuer && half == 0) {
        const uint4 ones = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        chunk(sm, S::X, 16, row) = ones;
        chunk(sm, S::X, 17, row) = ones;
        chunk(sm, S::X2, 16, row) = ones;
        chunk(sm, S::X2, 17, row) = ones;
        chunk(sm, S::H1, 8, row) = ones;
        chunk(sm, S::H1, 9, row) = ones;
        chunk(sm, S::H2, 8, row) = ones;
        chunk(sm, S::H2, 9, row) = ones;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = __shfl_sync(0xffffffffu, tmem_base, 0), lane = (uint32_t)(32 * (warp & 3)) << 16;
    // 64-wide layers: this thread's columns c64 .. c64 + C64, in NB64 blocks of BW64
    constexpr int C64 = 64 / H, BW64 = C64 < 32 ? C64 : 32, NB64 = C64 / BW64;
    const int c64 = C64 * half;
    const uint32_t sb = tc::smem_u32(sm);
    const float *b1 = reinterpret_cast<const float *>(sm + S::BIAS), *b2 = b1 + 64, *b3 = b1 + 128;
    constexpr uint32_t kI64 = tc::idesc_bf16(128, 64, false, false), kI128 = tc::idesc_bf16(128, 128, false, false);
    // this thread's column blocks of 32 of the 128 outputs in the softmax: q = half + H k, k < 4/H --
    // interleaved, so that the parts of a row share its aperture's blocks evenly wherever the
    // aperture lies (a block outside every pixel's aperture of a warp is skipped); the partial
    // gradients are written out by the blocks q4 .. q4 + 4/H - 1
    const int q4 = half * (4 / H);
    auto qb = [&](int k) { return half + H * k; };

    long long n_tiles;
    int nblk = 1, nd = 0;
    if (MODE == kInfer) {
        nd = a.plan->n_depth;
        nblk = (nd + kTile - 1) / kTile;
        n_tiles = (long long)a.plan->n_lines * nblk;
    } else {
        n_tiles = (a.n + kTile - 1) / kTile;
    }
    uint32_t phase = 0;
    bool ok = true, first = true;
    float loss_acc = 0.0f, cnt_acc = 0.0f;
    // The products are issued by one elected lane of a converged warp (training: the issuing
    // warp; else warp 0).  A commit covers the earlier products of the thread that makes it, so
    // every product and commit must come from the same lane: the lowest, which elect.sync picks
    // in a converged warp; another leader is reported as an internal error.  In training the dW1
    // products of a tile wait for the next tile's Z1 products, so that they run while the pixel
    // warps form H1 instead of delaying Z1.
    uint32_t leader = 0, bad_leader = 0;
    auto lead = [&]() {
        const bool e = tc::elect_one(&leader);
        bad_leader |= leader;
        return e;
    };
    int x_prev = S::X;        // the X buffer of the tile whose dW1 products are pending
    bool dw1_acc = false;     // whether they add to earlier tiles' sums
    auto issue_dw1 = [&]() {
        mma_chain(tm + kDW1, sb + S::DZ1, 128, 2048, sb + x_prev, 128, 2048, tc::idesc_bf16(128, 144, true, true), 8,
                  dw1_acc);
        dw1_acc = true;
    };
    // End of a step: the threads' shared-memory operands published to the products that read
    // them (and to the issuing warp, which meets the same barrier); false when some thread failed.
    auto step_end = [&]() -> bool {
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        if (!ok) return false;
        tc::fence_after_sync();
        return true;
    };

    int iter = 0;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++iter) {
        const int xo = (MODE == kTrain && (iter & 1)) ? S::X2 : S::X;   // this tile's X buffer
        if (MODE == kTrain && issuer) {
            // each group of products after the barrier that publishes its operands (the first
            // also the tile before's dZ1, for its dW1 products)
            if (a.rows_tma) {   // (the pixel warps wait for the rows too)
                ok = mbar_wait_bounded(&bar_rows, rows_phase & 1u, 1LL << 31) && ok;
                ++rows_phase;
            }
            if (!step_end()) break;
            if (lead()) {
                mma_chain(tm + kT64, sb + xo, 2048, 128, sb + S::W1, 1024, 128, kI64, 8, false);
                tc::mma_commit(&bar);
                if (!first) {   // the tile before's [dW1 | db1] += dZ1^T [X | 1]
                    issue_dw1();
                    tc::mma_commit(&bar_dw1);
                }
            }
            __syncwarp();
            if (!step_end()) break;
            if (lead()) {
                mma_chain(tm + kT64, sb + S::H1, 2048, 128, sb + S::W2, 1024, 128, kI64, 4, false);
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!step_end()) break;
            if (lead()) {
                mma_chain(tm + kT128, sb + S::H2, 2048, 128, sb + S::W3, 2048, 128, kI128, 4, false);
                tc::mma_commit(&bar);
                // the next tile's rows into the tile before's X buffer (its dW1 products, covered
                // by the Z2 commit that the pixel warps waited for before this barrier, are complete)
                if (a.rows_tma && tile + gridDim.x < n_tiles) copy_rows(tile + gridDim.x, xo == S::X ? S::X2 : S::X);
            }
            __syncwarp();
            if (!step_end()) break;
            if (lead()) {   // dH2 = dZ3 W3 (waited for);  [dW3 | db3] += dZ3^T [H2 | 1]
                mma_chain(tm + kT64, sb + S::DZ3, 2048, 128, sb + S::W3, 128, 2048,
                          tc::idesc_bf16(128, 64, false, true), 8, false);
                tc::mma_commit(&bar);
                mma_chain(tm + kDW3, sb + S::DZ3, 128, 2048, sb + S::H2, 128, 2048,
                          tc::idesc_bf16(128, 80, true, true), 8, !first);
                tc::mma_commit(&bar_dw1);
            }
            __syncwarp();
            if (!step_end()) break;
            if (lead()) {   // dH1 = dZ2 W2 (waited for);  [dW2 | db2] += dZ2^T [H1 | 1]
                mma_chain(tm + kT64, sb + S::DZ2, 2048, 128, sb + S::W2, 128, 1024,
                          tc::idesc_bf16(128, 64, false, true), 4, false);
                tc::mma_commit(&bar);
                mma_chain(tm + kDW2, sb + S::DZ2, 128, 2048, sb + S::H1, 128, 2048,
                          tc::idesc_bf16(128, 80, true, true), 8, !first);
                tc::mma_commit(&bar_dw1);
            }
            __syncwarp();
            x_prev = xo;
            first = false;
            continue;
        }
        // ---- inputs: one row of X per pixel (each half writes its chunks)
        uint32_t mk[4] = {0u, 0u, 0u, 0u};
        float nrm = 0.0f, tgt = 0.0f;
        bool row_ok;
        long long p = 0, rw_out = 0;
        int line = 0, i = 0;
        if (MODE == kInfer) {
            line = (int)(tile / nblk);
            i = (int)(tile % nblk) * kTile + row;
            row_ok = i < nd;
            float n2v[2] = {0.0f, 0.0f};
            const int n_el = a.plan->n_el;
            // the tile's 128 depths lie in one 256-depth delay tile: one element box for the CTA
            const ElemBox box = elem_box(a.plan, line, (int)(tile % nblk) * kTile);
            PixelGeo g;
            if (row_ok) g = pixel_geo(a.plan, a.ch, line, i);
            // stage the box elements' sample windows of this tile in the H1/H2 bytes (free until Z1)
            const LineGeo lgt = a.plan->lines[line];
            const int i_a = (int)(tile % nblk) * kTile, i_b = min(i_a + kTile - 1, nd - 1);
            const int n_slots = min(box.hi - box.lo + 1, kWinSlots);
            const bool staged = a.plan->bulk_ok && (reinterpret_cast<uintptr_t>(a.ch) & 15) == 0 && lgt.plane == 0;
            int16_t *win = reinterpret_cast<int16_t *>(sm + S::H1);
            // the slots' element positions, in the softmax exchange rows (free until the softmax)
            static_assert(MODE != kInfer || (H > 1 && H * kTile >= kWinSlots), "element positions in the exchange rows");
            float *win_x = &xrow[H > 1 ? 1 : 0][0][0], *win_y = &xrow[H > 1 ? 2 : 0][0][0];
            if (staged) {
                if (t < n_slots) {
                    win_ws[t] = tile_window(a.plan, lgt, box.lo + t, i_a, i_b, win_bg[t][0], win_bg[t][1]);
                    const float4 xe = __ldg(&a.plan->elem[box.lo + t]);
                    win_x[t] = xe.x;
                    win_y[t] = xe.y;
                }
                __syncthreads();
                const int n_s = a.plan->n_s;
                const int16_t *rec_base = a.ch + (long long)lgt.tx * n_el * n_s;
                constexpr int kChunks = kWinW / 8;
                for (int q = t; q < n_slots * kChunks; q += NT) {
                    const int j = q / kChunks, c = q - j * kChunks;
                    const int ws = win_ws[j];
                    if (ws == kNoWin) continue;
                    const int s0 = ws + 8 * c;
                    int16_t *dst = win + j * kWinW + 8 * c;
                    const int16_t *src = rec_base + (long long)(box.lo + j) * n_s + s0;
                    if (s0 >= 0 && s0 + 8 <= n_s) {
                        cp_async16(dst, src);
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) dst[u] = (s0 + u >= 0 && s0 + u < n_s) ? src[u] : (int16_t)0;
                    }
                }
                cp_async_commit();
                cp_async_wait_all();
                __syncthreads();
            }
            // The row's 8-element chunks alternate between its H parts, so that each part gathers
            // about the same share of the box's elements wherever the box lies on the array (the
            // aperture of a line near the array's edge fills one end of the row); the mask bits of
            // a part's output blocks that another part found are exchanged after the gather.
            // (one instance per array kind: a single row of elements needs no y test)
            auto gather = [&](auto y_rows) {
                constexpr bool Y = decltype(y_rows)::value;
#pragma unroll 1
                for (int c = half; c < 16; c += H) {
                    if (!box.any(8 * c, 8 * c + 7)) {   // CTA-uniform: the whole chunk is outside the box
                        chunk(sm, S::X, c, row) = make_uint4(0u, 0u, 0u, 0u);
                        continue;
                    }
                    float v[8];
                    uint32_t cb = 0u;   // the chunk's aperture bits (bit j: element 8 c + j)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int e = 8 * c + j;
                        bool act = false;
                        if (row_ok && e < n_el && box.has(e)) {
                            const int jw = e - box.lo;
                            v[j] = (staged && jw < n_slots && win_ws[jw] != kNoWin)
                                       ? element_sample_staged<Y>(a.plan, g, e, act, win + jw * kWinW, win_ws[jw],
                                                                  win_bg[jw][0], win_bg[jw][1], win_x[jw], win_y[jw])
                                       : element_sample(a.plan, g, e, act);
                        } else {
                            v[j] = 0.0f;
                        }
                        n2v[j & 1] = fmaf(v[j], v[j], n2v[j & 1]);
                        cb |= act ? 1u << j : 0u;
                    }
                    // (into word c / 4 by selects: an index computed at run time would put mk in local memory)
#pragma unroll
                    for (int w = 0; w < 4; ++w) mk[w] |= (c >> 2) == w ? cb << (8 * (c & 3)) : 0u;
                    chunk(sm, S::X, c, row) = pack8(v);
                }
            };
            if (a.plan->el_ny > 1 || a.plan->ymax > a.plan->ymin)
                gather(std::true_type{});
            else
                gather(std::false_type{});
            nrm = n2v[0] + n2v[1];   // this half's share of ||x||^2 (square root below)
        } else if (MODE == kTrain) {
            if (rows_armed) {
                ok = mbar_wait_bounded(&bar_rows, rows_phase & 1u, 1LL << 31) && ok;
                ++rows_phase;
                rows_armed = false;
            } else {
                cp_async_wait_all();
            }
            p = tile * kTile + row;
            row_ok = nok;
            mk[0] = nmk[0], mk[1] = nmk[1], mk[2] = nmk[2], mk[3] = nmk[3];
            nrm = nnrm;
            tgt = nnrm > 0.0f ? nlab / nnrm : 0.0f;
        } else {
            p = tile * kTile + row;
            row_ok = p < a.n;
            rw_out = tile * a.tile_stride + (long long)row * a.stride;
            const long long rw = rw_out;
            if (row_ok) {
                const uint4 *src = reinterpret_cast<const uint4 *>(a.feat + rw * kIn);
#pragma unroll
                for (int c = half * (16 / H); c < (half + 1) * (16 / H); ++c) chunk(sm, S::X, c, row) = __ldg(src + c);
                const uint4 m4 = __ldg(reinterpret_cast<const uint4 *>(a.mask) + rw);
                mk[0] = m4.x, mk[1] = m4.y, mk[2] = m4.z, mk[3] = m4.w;
                nrm = __ldg(a.norm + rw);
                if (MODE == kTrain) tgt = nrm > 0.0f ? __ldg(a.label + rw) / nrm : 0.0f;
            } else {
#pragma unroll
                for (int c = half * (16 / H); c < (half + 1) * (16 / H); ++c)
                    chunk(sm, S::X, c, row) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        // (H == 2: mask word w of a row, needed by part w % 2, whose softmax blocks are w and w + 2, is
        // sent by the other part through the softmax exchange rows xrow[1..2]: written after the
        // barrier that ends the gather, since the gather reads the slots' element positions from
        // those rows, and read after the next barrier; the softmax writes them only after the one
        // after that)
        static_assert(MODE != kInfer || H <= 2, "the fused beamformer's mask exchange takes two parts");
        uint32_t *mx = reinterpret_cast<uint32_t *>(&xrow[H > 1 ? 1 : 0][0][0]);
        if constexpr (MODE == kInfer && H > 1) xrow[0][half][row] = nrm;
        if (!step_end()) break;
        if constexpr (MODE == kInfer && H > 1) {
            mx[(1 - half) * kTile + row] = word_of(mk, 1 - half);
            mx[(3 - half) * kTile + row] = word_of(mk, 3 - half);
        }
        if constexpr (MODE == kInfer) nrm = sqrtf(H > 1 ? xrow[0][0][row] + xrow[0][1][row] : nrm);
        const bool valid = row_ok && nrm > 0.0f;

        // ---- Z1 = X W1^T (training: issued by the issuing warp, as all products below)
        if (MODE != kTrain && warp == 0 && lead()) {
            mma_chain(tm + kT64, sb + xo, 2048, 128, sb + S::W1, 1024, 128, kI64, 8, false);
            tc::mma_commit(&bar);
        }
        ok = mma_wait(&bar, phase) && ok;
        const float scale = (MODE == kInfer) ? (nrm > 0.0f ? 1.0f / nrm : 0.0f) : 1.0f;
#pragma unroll
        for (int bk = 0; bk < NB64; ++bk) {
            const int col = c64 + BW64 * bk;
            float v[BW64];
            tmem_ld_block<BW64>(tm + lane + kT64 + col, v);
            bias_relu_rows<BW64>(v, b1 + col, scale, sm, S::H1, col / 8, row);
        }
        if (!step_end()) break;
        if constexpr (MODE == kInfer && H > 1) {   // (the mask words sent above)
            const uint32_t m0 = mx[half * kTile + row], m2 = mx[(half + 2) * kTile + row];
            mk[0] |= half == 0 ? m0 : 0u;
            mk[1] |= half == 1 ? m0 : 0u;
            mk[2] |= half == 0 ? m2 : 0u;
            mk[3] |= half == 1 ? m2 : 0u;
        }

        // ---- Z2 = H1 W2^T
        if (MODE != kTrain && warp == 0 && lead()) {
            mma_chain(tm + kT64, sb + S::H1, 2048, 128, sb + S::W2, 1024, 128, kI64, 4, false);
            tc::mma_commit(&bar);
        }
        ok = mma_wait(&bar, phase) && ok;
        // (the tile before's dW1 products, issued before Z2, are complete: its X buffer is free)
        if (MODE == kTrain && tile + gridDim.x < n_tiles) prefetch(tile + gridDim.x, xo == S::X ? S::X2 : S::X);
#pragma unroll
        for (int bk = 0; bk < NB64; ++bk) {
            const int col = c64 + BW64 * bk;
            float v[BW64];
            tmem_ld_block<BW64>(tm + lane + kT64 + col, v);
            bias_relu_rows<BW64>(v, b2 + col, 1.0f, sm, S::H2, col / 8, row);
        }
        if (!step_end()) break;

        // ---- Z3 = H2 W3^T, masked softmax, output (and its gradient)
        if (MODE != kTrain && warp == 0 && lead()) {
            mma_chain(tm + kT128, sb + S::H2, 2048, 128, sb + S::W3, 2048, 128, kI128, 4, false);
            tc::mma_commit(&bar);
        }
        ok = mma_wait(&bar, phase) && ok;
        // reductions over this thread's outputs in 4 independent partials (latency, not order, matters).
        // Training reads its two 32-column blocks in one tensor-memory round trip and keeps z + b3
        // in registers for the second pass.
        constexpr bool kPair = MODE == kTrain && 4 / H == 2;
        float vv[kPair ? 2 : 1][32];
        auto load_pair = [&]() {
            if constexpr (kPair) tc::tmem_ld32x2(tm + lane + kT128 + 32 * qb(0), tm + lane + kT128 + 32 * qb(1), vv[0], vv[1]);
        };
        float zm4[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        // a 32-output block outside the aperture of all of the warp's 32 pixels (shallow depths)
        // has no weight anywhere: the passes skip it (its exponentials and gradients are 0)
        bool blk[4 / H];
#pragma unroll
        for (int k = 0; k < 4 / H; ++k) blk[k] = __any_sync(0xffffffffu, word_of(mk, qb(k)) != 0u);
        load_pair();
#pragma unroll
        for (int k = 0; k < 4 / H; ++k) {
            const int q = qb(k);
            const uint32_t mq = word_of(mk, q);
            if (!blk[k]) continue;
            float vl[32];
            if constexpr (!kPair) tc::tmem_ld32(tm + lane + kT128 + 32 * q, vl);
            const float *v = kPair ? vv[k] : vl;
            const float4 *b34 = reinterpret_cast<const float4 *>(b3 + 32 * q);
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4) {
                const float4 bq = b34[j4];
                const float bj[4] = {bq.x, bq.y, bq.z, bq.w};
                float zs[4];   // z + b3 (pairs: two outputs per packed add)
                if constexpr (kPair) {
                    unpack2(add2(pack2(v[4 * j4], v[4 * j4 + 1]), pack2(bj[0], bj[1])), zs[0], zs[1]);
                    unpack2(add2(pack2(v[4 * j4 + 2], v[4 * j4 + 3]), pack2(bj[2], bj[3])), zs[2], zs[3]);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) zs[u] = v[4 * j4 + u] + bj[u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = 4 * j4 + u;
                    const bool on = (mq >> j) & 1u;
                    if constexpr (kPair) {   // outputs outside the aperture as -inf: exponential 0 below
                        vv[k][j] = on ? zs[u] : -INFINITY;
                        zm4[u] = fmaxf(zm4[u], vv[k][j]);
                    } else if (on) {
                        zm4[u] = fmaxf(zm4[u], zs[u]);
                    }
                }
            }
        }
        float zmax = fmaxf(fmaxf(zm4[0], zm4[1]), fmaxf(zm4[2], zm4[3]));
        if constexpr (H > 1) {   // the row's maximum over its parts
            xrow[0][half][row] = zmax;
            if constexpr (MODE == kTrain) row_parts_sync<H>(warp);
            else __syncthreads();
            zmax = xrow[0][0][row];
#pragma unroll
            for (int h = 1; h < H; ++h) zmax = fmaxf(zmax, xrow[0][h][row]);
        }
        float se4[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sx4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        // exp(z - zmax) = 2^(z log2 e - zmax log2 e) (a row without any output in the aperture
        // has zmax = -inf and every z = -inf: offset 0 keeps its exponentials 0)
        const float c2 = zmax > -INFINITY ? -zmax * kLog2e : 0.0f;
        // pairs: the partial sums se4 / sx4 [0, 1] and [2, 3] as two packed accumulators each
        u64 se2[2] = {0ull, 0ull}, sx2[2] = {0ull, 0ull};
#pragma unroll
        for (int k = 0; k < 4 / H; ++k) {
            const int q = qb(k);
            const uint32_t mq = word_of(mk, q);
            if (!blk[k]) continue;
            float vl[32], xl[32];
            if constexpr (!kPair) tc::tmem_ld32(tm + lane + kT128 + 32 * q, vl);
            const float *v = kPair ? vv[k] : vl;
            float *x = xl;
#pragma unroll
            for (int c = 0; c < 4; ++c) unpack8(chunk(sm, xo, 4 * q + c, row), x + 8 * c);
            if constexpr (kPair) {   // (masked z + b3 from the first pass), two outputs per packed operation
                const u64 L2 = pack2(kLog2e, kLog2e), C2 = pack2(c2, c2);
#pragma unroll
                for (int j2 = 0; j2 < 16; ++j2) {
                    const int j = 2 * j2;
                    float a0, a1;
                    unpack2(fma2(pack2(v[j], v[j + 1]), L2, C2), a0, a1);
                    vv[k][j] = ex2_approx(a0);   // kept for the output gradient below
                    vv[k][j + 1] = ex2_approx(a1);
                    const u64 ep = pack2(vv[k][j], vv[k][j + 1]);
                    se2[j2 & 1] = add2(se2[j2 & 1], ep);
                    sx2[j2 & 1] = fma2(ep, pack2(x[j], x[j + 1]), sx2[j2 & 1]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float ez = ((mq >> j) & 1u) ? __expf(v[j] + b3[32 * q + j] - zmax) : 0.0f;
                    se4[j & 3] += ez;
                    sx4[j & 3] = fmaf(ez, x[j], sx4[j & 3]);
                }
            }
        }
        if constexpr (kPair) {
            unpack2(se2[0], se4[0], se4[1]);
            unpack2(se2[1], se4[2], se4[3]);
            unpack2(sx2[0], sx4[0], sx4[1]);
            unpack2(sx2[1], sx4[2], sx4[3]);
        }
        float se = (se4[0] + se4[1]) + (se4[2] + se4[3]);
        float sx = (sx4[0] + sx4[1]) + (sx4[2] + sx4[3]);
        if constexpr (H > 1) {   // the row's sums over its parts (pairwise, fixed order)
            xrow[1][half][row] = se;
            xrow[2][half][row] = sx;
            if constexpr (MODE == kTrain) row_parts_sync<H>(warp);
            else __syncthreads();
            if constexpr (H == 2) {
                se = xrow[1][0][row] + xrow[1][1][row];
                sx = xrow[2][0][row] + xrow[2][1][row];
            } else {
                se = (xrow[1][0][row] + xrow[1][1][row]) + (xrow[1][2][row] + xrow[1][3][row]);
                sx = (xrow[2][0][row] + xrow[2][1][row]) + (xrow[2][2][row] + xrow[2][3][row]);
            }
        }
        const float yh = se > 0.0f ? sx / se : 0.0f;
        if (MODE == kForward) {
            if (row_ok && half == 0) a.y[rw_out] = yh * nrm;
        } else if (MODE == kInfer) {
            if (row_ok && half == 0) a.rf[(long long)line * nd + i] = yh;
        } else {
            const float r = valid ? yh - tgt : 0.0f;
            if (half == 0) {
                loss_acc = fmaf(r, r, loss_acc);
                cnt_acc += valid ? 1.0f : 0.0f;
            }
            const float g = 2.0f * r, inv_se = se > 0.0f ? 1.0f / se : 0.0f, gs = g * inv_se;
#pragma unroll
            for (int k = 0; k < 4 / H; ++k) {
                const int q = qb(k);
                const uint32_t mq = word_of(mk, q);
                if (!blk[k]) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) chunk(sm, S::DZ3, 4 * q + c, row) = make_uint4(0u, 0u, 0u, 0u);
                    continue;
                }
                float vl[32], xl[32], dz[32];
                const float *x = xl;
                if constexpr (kPair) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) unpack8(chunk(sm, xo, 4 * q + c, row), xl + 8 * c);
                } else {
                    tc::tmem_ld32(tm + lane + kT128 + 32 * q, vl);
#pragma unroll
                    for (int c = 0; c < 4; ++c) unpack8(chunk(sm, xo, 4 * q + c, row), xl + 8 * c);
                }
                // dz_e = w_e (x_e - yh) g, w_e = exp(z_e - zmax) / sum: pairs reuse the
                // exponentials of the pass above (the same values), two outputs per packed operation
                if constexpr (kPair) {
                    const u64 GS = pack2(gs, gs), NYH = pack2(-yh, -yh);
#pragma unroll
                    for (int j = 0; j < 32; j += 2)
                        unpack2(mul2(mul2(pack2(vv[k][j], vv[k][j + 1]), GS), add2(pack2(x[j], x[j + 1]), NYH)),
                                dz[j], dz[j + 1]);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float pe = ((mq >> j) & 1u) ? __expf(vl[j] + b3[32 * q + j] - zmax) * inv_se : 0.0f;
                        dz[j] = pe * (x[j] - yh) * g;
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) chunk(sm, S::DZ3, 4 * q + c, row) = pack8(dz + 8 * c);
            }
        }
        if (!step_end()) break;
        if (MODE != kTrain) continue;

        // ---- dH2 = dZ3 W3;  [dW3 | db3] += dZ3^T [H2 | 1].  Only dH2 is waited for: the
        // weight-gradient products run while the threads form dZ2 (they read dZ3 and H2, which
        // nothing writes before the next tile's products, issued after them, complete)
        ok = mma_wait(&bar, phase) && ok;
#pragma unroll
        for (int bk = 0; bk < NB64; ++bk) {
            const int col = c64 + BW64 * bk;
            float v[BW64];
            tmem_ld_block<BW64>(tm + lane + kT64 + col, v);
            relu_grad_rows<BW64>(v, sm, S::H2, S::DZ2, col / 8, row);
        }
        if (!step_end()) break;

        // ---- dH1 = dZ2 W2;  [dW2 | db2] += dZ2^T [H1 | 1], dW2 not waited for (as dW3; its
        // discarded rows 64..127 read the DZ1 bytes that the threads write meanwhile)
        ok = mma_wait(&bar, phase) && ok;
#pragma unroll
        for (int bk = 0; bk < NB64; ++bk) {
            const int col = c64 + BW64 * bk;
            float v[BW64];
            tmem_ld_block<BW64>(tm + lane + kT64 + col, v);
            relu_grad_rows<BW64>(v, sm, S::H1, S::DZ1, col / 8, row);
        }
        // ---- [dW1 | db1] += dZ1^T [X | 1]: dZ1 is published by the next tile's first barrier (or
        // the one after the loop); the products are issued after the next tile's Z1 products and
        // covered by the commit of its Z2 (before this X buffer is refilled or DZ1 rewritten); the
        // final commit below covers the last tile's
        first = false;
    }
    if (MODE == kTrain && !first) {   // the last tile's dW1 (unless abandoned), then a commit of all
        const bool done = step_end();    // (publishes the last dZ1)
        if (issuer) {
            if (lead()) {
                if (done) issue_dw1();
                tc::mma_commit(&bar);
            }
            __syncwarp();
        } else {
            ok = mma_wait(&bar, phase) && ok;
        }
    }
    if (MODE == kTrain && rows_armed) {   // a prefetch that no tile waited for (an abort): let it land
        mbar_wait_bounded(&bar_rows, rows_phase & 1u, 1LL << 27);
        rows_armed = false;
    }
    ok = __syncthreads_and(ok);   // the last wait of a tile is not followed by a barrier
    if (!ok && t == 0) set_status(SUPRA_ETIMEOUT);
    if (bad_leader != 0 && (t & 31) == 0) set_status(SUPRA_EINTERNAL);   // (see lead above)

    if (MODE == kTrain) {
        float *part = a.partial + (long long)blockIdx.x * kPartStride;
        // weight and bias gradients (unnormalised sums over this CTA's pixels); lane = row,
        // each half takes half of every accumulator's weight columns.  Weight blocks are stored
        // column by column (see param_of), so that a warp's store covers 32 consecutive floats.
        float v[32], w[16], vb[BW64];
        const bool low = (warp & 3) < 2;   // rows 0..63: the 64-row accumulators dW2, dW1
        if (!issuer && ok && !first) {
            for (int bk = 0; bk < NB64; ++bk) {
                const int col = c64 + BW64 * bk;
                tmem_ld_block<BW64>(tm + lane + kDW3 + col, vb);
#pragma unroll
                for (int j = 0; j < BW64; ++j) part[kOffW3 + (col + j) * 128 + row] = vb[j];
            }
            if (half == 0) {
                tc::tmem_ld16(tm + lane + kDW3 + 64, w);
                part[kOffB3 + row] = w[0];
            }
            if (low) {
                for (int bk = 0; bk < NB64; ++bk) {
                    const int col = c64 + BW64 * bk;
                    tmem_ld_block<BW64>(tm + lane + kDW2 + col, vb);
#pragma unroll
                    for (int j = 0; j < BW64; ++j) part[kOffW2 + (col + j) * 64 + row] = vb[j];
                }
                for (int q = q4; q < q4 + 4 / H; ++q) {
                    tc::tmem_ld32(tm + lane + kDW1 + 32 * q, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) part[kOffW1 + (32 * q + j) * 64 + row] = v[j];
                }
                if (half == 0) {
                    tc::tmem_ld16(tm + lane + kDW2 + 64, w);
                    part[kOffB2 + row] = w[0];
                    tc::tmem_ld16(tm + lane + kDW1 + 128, w);
                    part[kOffB1 + row] = w[0];
                }
            }
        } else if (!issuer) {
            for (int k = t; k < kParams; k += NC) part[k] = 0.0f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
            cnt_acc += __shfl_xor_sync(0xffffffffu, cnt_acc, o);
        }
        if ((t & 31) == 0 && !issuer) red[0][warp] = loss_acc, red[1][warp] = cnt_acc;
        __syncthreads();
        if (t == 0) {
            float ls = 0.0f, cs = 0.0f;
            for (int k = 0; k < NC / 32; ++k) ls += red[0][k], cs += red[1][k];
            part[kParams] = ls;
            part[kParams + 1] = cs;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tm, kCols);
}

// Network inputs of every pixel of a frame: x / ||x|| in BF16 [line * n_depth + i][128],
// aperture mask (bit e of word e / 32) and ||x||.  Two passes over the elements
// (norm, then normalised samples).
__global__ void __launch_bounds__(128) features_kernel(const DevPlan *__restrict__ P, const int16_t *__restrict__ ch,
                                                       uint16_t *__restrict__ feat, uint32_t *__restrict__ mask,
                                                       float *__restrict__ norm) {
    const int line = blockIdx.y, i = blockIdx.x * 128 + threadIdx.x, nd = P->n_depth;
    if (i >= nd) return;
    const PixelGeo g = pixel_geo(P, ch, line, i);
    const ElemBox box = elem_box(P, line, blockIdx.x * 128);
    const int n_el = P->n_el;
    float n2 = 0.0f;
    const int e_end = min(n_el - 1, box.hi);
    for (int e = max(0, box.lo); e <= e_end; ++e) {
        bool act;
        const float x = element_sample(P, g, e, act);
        n2 = fmaf(x, x, n2);
    }
    const float nr = sqrtf(n2), inv = nr > 0.0f ? 1.0f / nr : 0.0f;
    const long long pix = (long long)line * nd + i;
    uint32_t mk[4] = {0u, 0u, 0u, 0u};
    uint4 *dst = reinterpret_cast<uint4 *>(feat + pix * kIn);
#pragma unroll 1
    for (int c = 0; c < 16; ++c) {
        if (!box.any(8 * c, 8 * c + 7)) {
            dst[c] = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = 8 * c + j;
            bool act = false;
            v[j] = (e < n_el && box.has(e)) ? element_sample(P, g, e, act) * inv : 0.0f;
            if (act) mk[e >> 5] |= 1u << (e & 31);
        }
        dst[c] = pack8(v);
    }
    reinterpret_cast<uint4 *>(mask)[pix] = make_uint4(mk[0], mk[1], mk[2], mk[3]);
    norm[pix] = nr;
}

// grad = sum of the per-CTA partials / valid-pixel count; index kParams is the loss.
// Sums in a fixed order, so the result does not depend on scheduling: a block takes 32
// indices, its warp g sums partials g, g + 8, g + 16, ... of each, and the eight warp
// sums are added in warp order.  FP32 (this GPU's FP64 rate is a small fraction of
// its FP32 rate); the error of these short sums stays near 1e-6 of the result.
constexpr int kReduceCols = 32, kReduceGroups = 8;

// Parameter index of entry s of a per-CTA partial gradient: the weight blocks are stored column
// by column (W1 [64][128] as [128][64], W2 [64][64] transposed, W3 [128][64] as [64][128]);
// biases, the loss sum and the pixel count in place.
__device__ __forceinline__ int param_of(int s) {
    if (s < kOffB1) return (s & 63) * 128 + (s >> 6);
    if (s >= kOffW2 && s < kOffB2) {
        const int t = s - kOffW2;
        return kOffW2 + (t & 63) * 64 + (t >> 6);
    }
    if (s >= kOffW3 && s < kOffB3) {
        const int t = s - kOffW3;
        return kOffW3 + (t & 127) * 64 + (t >> 7);
    }
    return s;
}
// Warp g's sums for column j: partials g, g + 8, g + 16, ... added in that order (and, on the
// count lane, their pixel counts); the rows are loaded twenty at a time (all of them for up to
// 160 partials) ahead of the adds.
__device__ __forceinline__ void column_sum(const float *__restrict__ partial, int n_parts, int j, bool count_lane,
                                           int g, float &s, float &cnt) {
    constexpr int U = 20;
    s = 0.0f, cnt = 0.0f;
    const bool col = j <= kParams;
    for (int c = g; c < n_parts; c += U * kReduceGroups) {
        float v[U], w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int cc = c + u * kReduceGroups;
            const float *row = partial + (long long)cc * kPartStride;
            v[u] = (cc < n_parts && col) ? row[j] : 0.0f;
            w[u] = (cc < n_parts && count_lane) ? row[kParams + 1] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c + u * kReduceGroups < n_parts) {
                s += v[u];
                cnt += w[u];
            }
        }
    }
}

__global__ void __launch_bounds__(kReduceCols * kReduceGroups) reduce_kernel(const float *__restrict__ partial,
                                                                            int n_parts, float *__restrict__ grad,
                                                                            float *__restrict__ loss) {
    __shared__ float part_sum[kReduceGroups][kReduceCols + 1];
    __shared__ float part_cnt[kReduceGroups];
    const int lane = threadIdx.x % kReduceCols, g = threadIdx.x / kReduceCols;
    const int j = blockIdx.x * kReduceCols + lane;
    float s, cnt;
    column_sum(partial, n_parts, j, lane == 0, g, s, cnt);
    part_sum[g][lane] = s;
    if (lane == 0) part_cnt[g] = cnt;
    __syncthreads();
    if (g == 0 && j <= kParams) {
        float tot = 0.0f, ct = 0.0f;
        for (int k = 0; k < kReduceGroups; ++k) {
            tot += part_sum[k][lane];
            ct += part_cnt[k];
        }
        const float v = ct > 0.0f ? tot / ct : 0.0f;
        if (j < kParams) grad[param_of(j)] = v;
        else if (loss) *loss = v;
    }
}

// One parameter's Adam update with bias correction (c1 = 1 / (1 - beta1^step), c2 = 1 / (1 - beta2^step))
// from its current p, m, v (pj, mj0, vj0).
__device__ __forceinline__ void adam_store(float *p, float *m, float *v, int j, float gj, float pj, float mj0,
                                           float vj0, float lr, float beta1, float beta2, float eps, float c1,
                                           float c2) {
    const float mj = fmaf(beta1, mj0, (1.0f - beta1) * gj);
    const float vj = fmaf(beta2, vj0, (1.0f - beta2) * gj * gj);
    m[j] = mj;
    v[j] = vj;
    p[j] = pj - lr * (mj * c1) / (sqrtf(vj * c2) + eps);
}
__device__ __forceinline__ void adam_update(float *p, float *m, float *v, int j, float gj, float lr, float beta1,
                                            float beta2, float eps, float c1, float c2) {
    adam_store(p, m, v, j, gj, p[j], m[j], v[j], lr, beta1, beta2, eps, c1, c2);
}

// reduce_kernel followed by the Adam update of each reduced parameter (one kernel for the
// training step's tail); the gradient and the loss are written as reduce_kernel writes them.
__global__ void __launch_bounds__(kReduceCols * kReduceGroups) reduce_adam_kernel(
    const float *__restrict__ partial, int n_parts, float *__restrict__ grad, float *__restrict__ loss,
    float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, float lr, float beta1, float beta2, float eps,
    float c1, float c2) {
    __shared__ float part_sum[kReduceGroups][kReduceCols + 1];
    __shared__ float part_cnt[kReduceGroups];
    const int lane = threadIdx.x % kReduceCols, g = threadIdx.x / kReduceCols;
    const int j = blockIdx.x * kReduceCols + lane;
    // the parameter's current p, m, v are read while the partials load
    const int jp = j < kParams ? param_of(j) : 0;
    float pj = 0.0f, mj = 0.0f, vj = 0.0f;
    if (g == 0 && j < kParams) pj = p[jp], mj = m[jp], vj = v[jp];
    float s, cnt;
    column_sum(partial, n_parts, j, lane == 0, g, s, cnt);
    part_sum[g][lane] = s;
    if (lane == 0) part_cnt[g] = cnt;
    __syncthreads();
    if (g == 0 && j <= kParams) {
        float tot = 0.0f, ct = 0.0f;
        for (int k = 0; k < kReduceGroups; ++k) {
            tot += part_sum[k][lane];
            ct += part_cnt[k];
        }
        const float gj = ct > 0.0f ? tot / ct : 0.0f;
        if (j < kParams) {
            grad[jp] = gj;
            adam_store(p, m, v, jp, gj, pj, mj, vj, lr, beta1, beta2, eps, c1, c2);
        } else if (loss) {
            *loss = gj;
        }
    }
}

// Adam with bias correction (c1 = 1 / (1 - beta1^step), c2 = 1 / (1 - beta2^step)).
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int n, float lr, float beta1, float beta2, float eps, float c1,
                            float c2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    adam_update(p, m, v, j, g[j], lr, beta1, beta2, eps, c1, c2);
}

}  // namespace apod
}  // namespace supra
