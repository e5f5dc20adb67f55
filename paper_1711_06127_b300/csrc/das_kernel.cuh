// das_kernel.cuh -- receive delay-and-sum beamforming (Sec. 1 "receive
// beamforming", Sec. 2 items 1-2, Table 1 "Beamformer") with the envelope and
// log-compression nodes (Sec. 2 items 3-4) fused behind it.
//
// One CTA owns one scanline of a group of G frames that share a plan and
// streams the line's depth axis in tiles of kDepthTile samples.  For every
// tile the aperture's elements are visited in chunks of kChunk: a producer
// (lanes 0..15 of warp 0, one element each) computes the element's sample
// window for the tile and stages that window of all G frames' records into
// shared memory with bulk async copies (TMA engine, cp.async.bulk) that
// complete on the stage's mbarrier; a ring of `stages` buffers keeps
// several chunks in flight while the CTA computes on the oldest.  Each thread
// owns one depth sample and one half of the chunk's elements and computes the
// delay, the linear interpolation weights and the apodization weight once,
// then applies them to all G frames -- frames of one plan share their delays,
// which is what makes a batch cheaper per frame than a single frame.
//
// Delay precision.  The two-way delay in samples reaches a few thousand,
// where the fp32 ulp is ~2.4e-4 samples.  The kernel therefore splits it as
//   s = K_tile + f_tile + a1 (i - i0) + (dt + de) fs / c
// with K_tile/f_tile the fp64-built base of the tile's first depth, and
// dt = |p - o_t| - r, de = |p - x_e| - r evaluated without cancellation as
// (|o - q|^2 + 2 r d.(o - q)) / (|p - q| + r).
#pragma once
#include "common.cuh"

namespace supra {

struct StageMeta {
    float beta, gamma, ex, ey;   // element constants for the CTA's line: d.(o - x_e), |o - x_e|^2, x_e, y_e
    int ws;                      // absolute sample index of the row's first staged sample
    int valid;
    int pad[2];
};

__device__ __forceinline__ float window_weight(int window, float u) {
    if (window == SUPRA_WINDOW_HANN) return 0.5f + 0.5f * __cosf(3.14159265358979f * u);
    if (window == SUPRA_WINDOW_HAMMING) return 0.54f + 0.46f * __cosf(3.14159265358979f * u);
    return 1.0f;
}

// |o + r d - q| - r without cancellation: (gamma + 2 r beta) / (|p - q| + r),
// beta = d.(o - q), gamma = |o - q|^2.
__device__ __forceinline__ float path_excess(float r, float beta, float gamma) {
    float r2 = fmaxf(fmaf(r, r + 2.0f * beta, gamma), 0.0f);
    float dist = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    float den = dist + r;
    float num = fmaf(2.0f * r, beta, gamma);
    return den > 1e-20f ? __fdividef(num, den) : 0.0f;
}

__device__ __forceinline__ int tile_chunks(const DevPlan *P, int line, int tile) {
    short4 b = P->ap_box[line * P->n_tiles + tile];
    int n = (b.y - b.x + 1) * (b.w - b.z + 1);
    return (n + kChunk - 1) / kChunk;
}

// Producer: stage chunk `chunk` of tile `tile` into ring buffer `buf`.
// Called by lanes 0..kChunk-1 of warp 0; each lane stages one element row for all frames.
template <int G>
__device__ __forceinline__ void issue_stage(const DevPlan *P, const FrameGroup &fg, int nf, int line,
                                            const LineGeo &lg, int tile, int chunk, int16_t *ring,
                                            StageMeta *meta, uint64_t *bar, int W) {
    const int lane = threadIdx.x;
    const short4 b = P->ap_box[line * P->n_tiles + tile];
    const int nbx = b.y - b.x + 1, nby = b.w - b.z + 1;
    const int j = chunk * kChunk + lane;
    StageMeta &mt = meta[lane];
    int16_t *rows = ring + lane * W;   // frame g row: rows + g * kChunk * W
    if (j >= nbx * nby) {
        mt.valid = 0;
        mbar_arrive_expect_tx(bar, 0);
        return;
    }
    const int e = (b.z + j / nbx) * P->el_nx + b.x + j % nbx;
    const float4 xe = __ldg(&P->elem[e]);
    const float mx = lg.ox - xe.x, my = lg.oy - xe.y, mz = lg.oz - xe.z;
    const float beta = lg.dx * mx + lg.dy * my + lg.dz * mz;
    const float gamma = mx * mx + my * my + mz * mz;

    const int i0 = tile * kDepthTile;
    const int i1 = min(i0 + kDepthTile - 1, P->n_depth - 1);
    const float r0 = P->depth0 + (float)i0 * P->depth_step;
    const float r1 = P->depth0 + (float)i1 * P->depth_step;
    const int kt = P->tile_k[tile];
    const float ft = P->tile_f[tile];
    float s0 = ft + (path_excess(r0, lg.bt, lg.gt) + path_excess(r0, beta, gamma)) * P->fsc;
    float s1 = ft + P->a1 * (float)(i1 - i0) + (path_excess(r1, lg.bt, lg.gt) + path_excess(r1, beta, gamma)) * P->fsc;
    float lo = fminf(s0, s1), hi = fmaxf(s0, s1);
    // The two-way path is convex in r: its maximum is at an end, its minimum may be
    // inside the tile; bound that minimum by the sum of the two paths' minima.
    if ((-beta > r0 && -beta < r1) || (-lg.bt > r0 && -lg.bt < r1)) {
        float re = fminf(fmaxf(-beta, r0), r1), rt = fminf(fmaxf(-lg.bt, r0), r1);
        float de = sqrtf(fmaxf(fmaf(re, re + 2.0f * beta, gamma), 0.0f));
        float dtp = sqrtf(fmaxf(fmaf(rt, rt + 2.0f * lg.bt, lg.gt), 0.0f));
        float s_abs = (de + dtp) * P->fsc - P->t0fs;
        lo = fminf(lo, s_abs - (float)kt);
    }
    const int lo_i = kt + (int)floorf(lo) - 1;
    const int ws = (lo_i >> 3) << 3;                     // floor to a multiple of 8 samples (16 bytes)
    if (kt + (int)floorf(hi) + 2 > ws + W - 1) set_status(SUPRA_EINTERNAL);
    const int n_s = P->n_s;
    const int c0 = max(ws, 0), c1 = min(ws + W, n_s);
    const long long rec = ((long long)lg.tx * P->n_el + e) * (long long)n_s;
    // zero padding outside the record (generic stores, released by this lane's arrive)
    if (c0 > ws || c1 < ws + W) {
        for (int g = 0; g < nf; ++g) {
            int16_t *dst = rows + g * kChunk * W;
            const int a_end = min(c0, ws + W) - ws;
            for (int k = 0; k < a_end; ++k) dst[k] = 0;
            for (int k = max(c1, c0) - ws; k < W; ++k) dst[k] = 0;
        }
    }
    mt.beta = beta;
    mt.gamma = gamma;
    mt.ex = xe.x;
    mt.ey = xe.y;
    mt.ws = ws;
    mt.valid = 1;
    if (fg.bulk) {
        const uint32_t bytes = c1 > c0 ? (uint32_t)(c1 - c0) * 2u : 0u;
        mbar_arrive_expect_tx(bar, bytes * (uint32_t)nf);
        if (bytes) {
            fence_proxy_async_smem();
            for (int g = 0; g < nf; ++g)
                bulk_g2s(rows + g * kChunk * W + (c0 - ws), fg.ch[g] + rec + c0, bytes, bar);
        }
    } else {
        for (int g = 0; g < nf; ++g) {
            int16_t *dst = rows + g * kChunk * W;
            const int16_t *src = fg.ch[g] + rec;
            for (int k = c0; k < c1; ++k) dst[k - ws] = src[k];
        }
        mbar_arrive_expect_tx(bar, 0);
    }
}

// MODE 0: write RF (float [n_lines][n_depth] per frame).
// MODE 1: envelope + log compression, write uint8 [n_lines][n_depth] per frame.
template <int G, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    das_kernel(const __grid_constant__ LaunchGroups L, int stages, int W, int ring_stride) {
    extern __shared__ __align__(128) unsigned char smem[];
    // ---- which (group, line)
    const int item = blockIdx.x;
    int gi = 0;
    while (gi + 1 < L.n_groups && L.g[gi + 1].line0 <= item) ++gi;
    const FrameGroup &fg = L.g[gi];
    const DevPlan *P = fg.plan;
    const int line = item - fg.line0;
    const int nf = min(fg.n, G);
    const LineGeo lg = P->lines[line];
    const int NT = P->n_tiles;
    const int nd = P->n_depth;

    // ---- shared memory carve-up
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);                     // [kMaxStages]
    StageMeta *metas = reinterpret_cast<StageMeta *>(smem + 64);             // [kMaxStages][kChunk]
    float *red = reinterpret_cast<float *>(smem + 64 + kMaxStages * kChunk * sizeof(StageMeta));  // [G + 1][128]
    float *ring_rf = red + (G + 1) * kDepthTile;                             // MODE 1: [G][ring_stride]
    float *taps = ring_rf + (MODE == 1 ? G * ring_stride : 0);               // MODE 1: [2][kMaxTaps]
    size_t head = 64 + kMaxStages * kChunk * sizeof(StageMeta) + (G + 1) * kDepthTile * 4 +
                  (MODE == 1 ? (G * ring_stride + 2 * kMaxTaps) * 4 : 0);
    head = (head + 127) & ~size_t(127);
    int16_t *stage_buf = reinterpret_cast<int16_t *>(smem + head);
    const int stage_elems = G * kChunk * W;                                  // int16 per stage

    const int tid = threadIdx.x;
    const int m = tid & (kDepthTile - 1);
    const int h = tid >> 7;
    const int H = (P->taps - 1) >> 1;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], kChunk);
        fence_mbar_init();
    }
    if (MODE == 1) {
        for (int k = tid; k < P->taps; k += kThreads) {
            taps[k] = P->taps_c[k];
            taps[kMaxTaps + k] = P->taps_s[k];
        }
        for (int k = tid; k < G * ring_stride; k += kThreads) ring_rf[k] = 0.0f;
    }
    __syncthreads();

    // total stages of this CTA
    int total = 0;
    for (int t = 0; t < NT; ++t) total += tile_chunks(P, line, t);

    // producer cursor (kept by every thread; used by warp 0)
    int p_tile = 0, p_chunk = 0, issued = 0;
    auto advance = [&]() {
        ++p_chunk;
        while (p_tile < NT && p_chunk >= tile_chunks(P, line, p_tile)) {
            p_chunk = 0;
            ++p_tile;
        }
    };
    while (p_tile < NT && tile_chunks(P, line, p_tile) == 0) ++p_tile;
    for (int s = 0; s < stages && issued < total; ++s) {
        if (tid < kChunk)
            issue_stage<G>(P, fg, nf, line, lg, p_tile, p_chunk, stage_buf + s * stage_elems, metas + s * kChunk,
                           &bars[s], W);
        advance();
        ++issued;
    }

    int n = 0;            // stages consumed
    bool failed = false;
    for (int tile = 0; tile <= NT && !failed; ++tile) {
        const int i0 = tile * kDepthTile;
        const int i = i0 + m;
        const bool act = (tile < NT) && (i < nd);
        float acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = 0.0f;
        float wsum = 0.0f;
        if (tile < NT) {
            // per-thread constants of depth sample i
            const float r = P->depth0 + (float)i * P->depth_step;
            const float px = fmaf(r, lg.dx, lg.ox), py = fmaf(r, lg.dy, lg.oy), pz = fmaf(r, lg.dz, lg.oz);
            const float qx = fminf(fmaxf(px, P->xmin), P->xmax);
            const float qy = fminf(fmaxf(py, P->ymin), P->ymax);
            const float a = fmaxf(pz * P->inv2f, P->amin);
            const float inv_a = 1.0f / a;
            const float base = P->tile_f[tile] + P->a1 * (float)m + path_excess(r, lg.bt, lg.gt) * P->fsc;
            const int kt = P->tile_k[tile];
            const int nch = tile_chunks(P, line, tile);
            const int window = P->window;
            const float fsc = P->fsc;
            for (int c = 0; c < nch; ++c, ++n) {
                const int sb = n % stages;
                bool ok = mbar_wait_bounded(&bars[sb], (uint32_t)((n / stages) & 1), 1LL << 31);
                if (ok && act) {
                    const StageMeta *mt = metas + sb * kChunk;
                    const int16_t *buf = stage_buf + sb * stage_elems;
#pragma unroll 2
                    for (int jj = 0; jj < kChunk / 2; ++jj) {
                        const int slot = h * (kChunk / 2) + jj;
                        const StageMeta md = mt[slot];
                        if (!md.valid) break;
                        const float ux = (md.ex - qx) * inv_a, uy = (md.ey - qy) * inv_a;
                        if (fabsf(ux) > 1.0f || fabsf(uy) > 1.0f) continue;
                        const float w = window_weight(window, ux) * window_weight(window, uy);
                        const float s = base + path_excess(r, md.beta, md.gamma) * fsc;
                        const float fl = floorf(s);
                        const float phi = s - fl;
                        int idx = kt + (int)fl - md.ws;
                        idx = min(max(idx, 0), W - 2);
                        const int16_t *row = buf + slot * W + idx;
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const float x0 = (float)row[g * kChunk * W];
                            const float x1 = (float)row[g * kChunk * W + 1];
                            acc[g] = fmaf(w, fmaf(phi, x1 - x0, x0), acc[g]);
                        }
                        wsum += w;
                    }
                }
                failed = __syncthreads_or(!ok);
                if (failed) break;
                // refill the buffer just consumed with stage n + stages
                if (issued < total) {
                    if (tid < kChunk)
                        issue_stage<G>(P, fg, nf, line, lg, p_tile, p_chunk, stage_buf + sb * stage_elems,
                                       metas + sb * kChunk, &bars[sb], W);
                    advance();
                    ++issued;
                }
            }
            if (failed) break;
            // combine the two element halves
            if (h == 1) {
#pragma unroll
                for (int g = 0; g < G; ++g) red[g * kDepthTile + m] = acc[g];
                red[G * kDepthTile + m] = wsum;
            }
            __syncthreads();
            if (h == 0) {
                wsum += red[G * kDepthTile + m];
                const float inv = wsum > 0.0f ? 1.0f / wsum : 0.0f;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const float v = act ? (acc[g] + red[g * kDepthTile + m]) * inv : 0.0f;
                    if (MODE == 0) {
                        if (act && g < nf)
                            static_cast<float *>(fg.out[g])[(long long)line * nd + i] = v;
                    } else {
                        ring_rf[g * ring_stride + 2 * H + m] = v;
                    }
                }
            }
        } else if (MODE == 1) {
            // the tile past the end: zero padding feeds the last H outputs
            for (int k = tid; k < G * kDepthTile; k += kThreads)
                ring_rf[(k / kDepthTile) * ring_stride + 2 * H + (k % kDepthTile)] = 0.0f;
        }
        if (MODE == 1) {
            __syncthreads();
            // envelope of depth o = i0 - H + m: 2 |sum_k g_k rf(o + H - k)|, g_k = h_k e^{j w (k - H)}
            const int o = i0 - H + m;
            if (o >= 0 && o < nd) {
                for (int g = h; g < nf; g += 2) {
                    const float *x = ring_rf + g * ring_stride + 2 * H + m;
                    float re = 0.0f, im = 0.0f;
                    for (int k = 0; k < 2 * H + 1; ++k) {
                        const float v = x[-k];
                        re = fmaf(taps[k], v, re);
                        im = fmaf(taps[kMaxTaps + k], v, im);
                    }
                    const float env = 2.0f * sqrtf(fmaf(re, re, im * im));
                    float code = 0.0f;
                    if (env > 0.0f) code = fminf(fmaxf(floorf(fmaf(P->log_a, __log2f(env), P->log_b)), 0.0f), 255.0f);
                    static_cast<uint8_t *>(fg.out[g])[(long long)line * nd + o] = (uint8_t)code;
                }
            }
            __syncthreads();
            // keep the last 2H RF samples for the next tile's halo
            for (int k = tid; k < G * 2 * H; k += kThreads) {
                const int g = k / (2 * H), j = k % (2 * H);
                ring_rf[g * ring_stride + j] = ring_rf[g * ring_stride + kDepthTile + j];
            }
            __syncthreads();
        }
    }
    if (failed) {
        set_status(SUPRA_ETIMEOUT);
        // let copies still in flight land before the CTA's shared memory goes away
        if (tid == 0)
            for (int k = n; k < issued; ++k)
                mbar_wait_bounded(&bars[k % stages], (uint32_t)((k / stages) & 1), 1LL << 27);
        __syncthreads();
    }
}

}  // namespace supra
