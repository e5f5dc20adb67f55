// post_kernels.cuh -- the unfused envelope and log-compression nodes and the
// scan-conversion node (Sec. 1 step list; Sec. 2 items 3-5; Table 1 columns
// "Envelope", "Log comp.", "Scan conv.").
#pragma once
#include "common.cuh"

namespace supra {

constexpr int kEnvTile = 256;
constexpr float kInsideEps = 1e-3f;   // grid points this close (in index units) to the scanned region's edge are inside

// IQ demodulation + low-pass + |.|: env(i) = 2 |sum_k' g_k' rf(i + 31 - k')| over the
// plan's centred 63-slot taps, with the demodulation phase folded into the taps
// (g_k' = h e^{j w (k' - 31)}; the remaining factor e^{-j w i} has unit modulus).
// Frequency compounding (Sec. 2 item 3): one such sum per band of the plan's bank,
// env = (2 / K) sum_k |iq_k|.
__global__ void __launch_bounds__(kEnvTile) envelope_kernel(const DevPlan *__restrict__ P, const float *__restrict__ rf,
                                                            float *__restrict__ env) {
    __shared__ float x[kEnvTile + kTapSlots];
    __shared__ float tc[kMaxBands][kTapSlots], ts[kMaxBands][kTapSlots];
    const int line = blockIdx.y;
    const int nd = P->n_depth;
    const int i0 = blockIdx.x * kEnvTile;
    const int nb = P->n_bands;
    const float *src = rf + (long long)line * nd;
    for (int k = threadIdx.x; k < kTapSlots; k += kEnvTile) {
        if (nb == 1) {
            tc[0][k] = P->taps_c[k];
            ts[0][k] = P->taps_s[k];
        } else {
            for (int b = 0; b < nb; ++b) {
                tc[b][k] = P->bank_c[b][k];
                ts[b][k] = P->bank_s[b][k];
            }
        }
    }
    for (int k = threadIdx.x; k < kEnvTile + kTapSlots - 1; k += kEnvTile) {
        const int i = i0 - kTapSlots / 2 + k;   // x[k] = rf(i0 - 32 + k)
        x[k] = (i >= 0 && i < nd) ? src[i] : 0.0f;
    }
    __syncthreads();
    const int i = i0 + threadIdx.x;
    if (i >= nd) return;
    const float *xp = x + threadIdx.x + kTapSlots - 1;   // rf(i + 31)
    float mag = 0.0f;
    for (int b = 0; b < nb; ++b) {
        float re = 0.0f, im = 0.0f;
#pragma unroll 8
        for (int k = 0; k < kTapSlots; ++k) {
            re = fmaf(tc[b][k], xp[-k], re);
            im = fmaf(ts[b][k], xp[-k], im);
        }
        mag += sqrtf(fmaf(re, re, im * im));
    }
    env[(long long)line * nd + i] = nb == 1 ? 2.0f * mag : (2.0f / (float)nb) * mag;
}

__device__ __forceinline__ uint8_t log_code(const DevPlan *P, float env) {
    if (!(env > 0.0f)) return 0;
    return (uint8_t)fminf(fmaxf(floorf(fmaf(P->log_a, __log2f(env), P->log_b)), 0.0f), 255.0f);
}

__global__ void logcompress_kernel(const DevPlan *__restrict__ P, const float *__restrict__ env,
                                   uint8_t *__restrict__ bm, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        bm[k] = log_code(P, env[k]);
}

// One scan-converted frame of a launch.
struct ScanFrame {
    const DevPlan *plan;
    const uint8_t *bm;
    uint8_t *img;
};

constexpr int kMaxScanFrames = 256;
constexpr int kScanGroup = 4;   // frames of one plan per CTA of the linear kernel
struct ScanLaunch {
    int n;
    ScanFrame f[kMaxScanFrames];
    // linear kernel: blockIdx.y = group of gn[g] <= kScanGroup consecutive frames from g0[g], one plan
    int n_groups;
    short g0[kMaxScanFrames], gn[kMaxScanFrames];
};

// Fractional line / depth coordinates of point (x, y, z) and the inside test.
__device__ __forceinline__ bool scan_coords(const DevPlan *P, float x, float y, float z, float &u, float &w,
                                            float &v) {
    const float rx = x - P->apx, ry = y - P->apy, rz = z - P->apz;
    if (P->geometry == SUPRA_GEOM_LINEAR) {
        u = (x - P->u0) * P->du_inv;
        w = 0.0f;
        v = (rz - P->v0) * P->dv_inv;
    } else if (P->geometry == SUPRA_GEOM_SECTOR) {
        u = (atan2f(rx, rz) - P->u0) * P->du_inv;
        w = 0.0f;
        v = (sqrtf(fmaf(rx, rx, rz * rz)) - P->v0) * P->dv_inv;
    } else {
        if (!(rz > 0.0f)) return false;
        u = (atanf(rx / rz) - P->u0) * P->du_inv;
        w = (atanf(ry / rz) - P->w0) * P->dw_inv;
        v = (sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz))) - P->v0) * P->dv_inv;
        if (!(w >= -kInsideEps && w <= (float)(P->lines_y - 1) + kInsideEps)) return false;
    }
    return u >= -kInsideEps && u <= (float)(P->lines_x - 1) + kInsideEps && v >= -kInsideEps &&
           v <= (float)(P->n_depth - 1) + kInsideEps;
}

// The scan conversion's floors and byte conversions stay off the conversion pipe (the kernels
// are bound by it otherwise): x + 1.5 * 2^23 rounded toward -inf is floor(x) + 1.5 * 2^23
// exactly for |x| < 2^22, whose bits give the integer; a byte placed in the mantissa of 2^23
// is that byte plus 2^23 exactly.
constexpr float kScanMagic = 12582912.0f;   // 1.5 * 2^23
__device__ __forceinline__ float scan_floor(float x, int &k) {
    const float t = __fadd_rd(x, kScanMagic);
    k = __float_as_int(t) - __float_as_int(kScanMagic);
    return t - kScanMagic;
}
__device__ __forceinline__ float byte_f(uint32_t b) { return __uint_as_float(0x4B000000u | b) - 8388608.0f; }
// floor(y) clamped to [0, 255] (y finite, within the interpolated bytes' range)
__device__ __forceinline__ uint8_t floor_byte(float y) {
    int k;
    scan_floor(y, k);
    return (uint8_t)min(max(k, 0), 255);
}

// u clamped to [0, n - 1] -> cell i0 <= max(n - 2, 0) and the fraction f = u - i0 (f = 1 at u = n - 1)
__device__ __forceinline__ void lerp_axis(float u, int n, int &i0, float &f) {
    u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
    int k;
    const float fl = scan_floor(u, k);
    const int top = max(n - 2, 0);
    i0 = min(k, top);
    f = u - (k > top ? fl - 1.0f : fl);   // (k > top only at u = n - 1: i0 = k - 1)
}

// Scan conversion of one output tile per CTA: 2D tiles are 64 (x) x 32 (z) pixels,
// 3D tiles 16 x 16 x 8 voxels; each thread owns 4 consecutive x at 2 z.  The
// tile's pixels are mapped back to (line, depth) coordinates, the bounding box
// of the lines and depths they interpolate is staged into shared memory with
// coalesced loads, and the interpolation reads shared memory.  A box that does
// not fit falls back to reading the lines in global memory.
constexpr int kScanBox = 24576;   // bytes of staged lines per tile

__device__ __forceinline__ uint8_t lerp_lines(const DevPlan *P, const uint8_t *src, int sx, int sy, int sv, float u,
                                              float w, float v) {
    // src addresses line (ix, iy) depth iv at ix * sx + iy * sy + iv * sv
    const int nlx = P->lines_x, nd = P->n_depth;
    int ix, iv;
    float fx, fv;
    lerp_axis(u, nlx, ix, fx);
    lerp_axis(v, nd, iv, fv);
    const int dx = ix + 1 < nlx ? sx : 0, dv = iv + 1 < nd ? sv : 0;
    float val;
    if (P->geometry == SUPRA_GEOM_PYRAMID) {
        int iy;
        float fy;
        lerp_axis(w, P->lines_y, iy, fy);
        const int dy = iy + 1 < P->lines_y ? sy : 0;
        const uint8_t *b = src + ix * sx + iy * sy + iv * sv;
        const float c00 = fmaf(fv, byte_f(b[dv]) - byte_f(b[0]), byte_f(b[0]));
        const float c01 = fmaf(fv, byte_f(b[dx + dv]) - byte_f(b[dx]), byte_f(b[dx]));
        const float c10 = fmaf(fv, byte_f(b[dy + dv]) - byte_f(b[dy]), byte_f(b[dy]));
        const float c11 = fmaf(fv, byte_f(b[dy + dx + dv]) - byte_f(b[dy + dx]), byte_f(b[dy + dx]));
        const float c0 = fmaf(fx, c01 - c00, c00), c1 = fmaf(fx, c11 - c10, c10);
        val = fmaf(fy, c1 - c0, c0);
    } else {
        const uint8_t *b = src + ix * sx + iv * sv;
        const float c0 = fmaf(fv, byte_f(b[dv]) - byte_f(b[0]), byte_f(b[0]));
        const float c1 = fmaf(fv, byte_f(b[dx + dv]) - byte_f(b[dx]), byte_f(b[dx]));
        val = fmaf(fx, c1 - c0, c0);
    }
    return floor_byte(val + 0.5f);
}

__global__ void __launch_bounds__(256) scanconvert_kernel(const __grid_constant__ ScanLaunch L) {
    __shared__ __align__(16) uint8_t box[kScanBox];
    __shared__ int red[6][8];
    const ScanFrame &F = L.f[blockIdx.y];
    const DevPlan *P = F.plan;
    const bool is3d = P->geometry == SUPRA_GEOM_PYRAMID;
    const int TX = is3d ? 16 : 64, TY = is3d ? 16 : 1, TZ = is3d ? 8 : 32;
    const int nx = P->gnx, ny = P->gny, nz = P->gnz;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY, ntz = (nz + TZ - 1) / TZ;
    const int t = threadIdx.x;
    const int nlx = P->lines_x, nly = P->lines_y, nd = P->n_depth;
    for (int tile = blockIdx.x; tile < ntx * nty * ntz; tile += gridDim.x) {
        const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
        // this thread: x = x0 .. x0 + 3, y, z = z0 and z0 + TZ / 2
        const int x0 = tx * TX + (t % (TX / 4)) * 4;
        const int y = ty * TY + (is3d ? (t / 4) % 16 : 0);
        const int zr = is3d ? t / 64 : t / 16;
        float pu[8], pw[8], pv[8];
        bool pin[8];
        int lo_x = 1 << 30, hi_x = -1, lo_y = 1 << 30, hi_y = -1, lo_v = 1 << 30, hi_v = -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + (k & 3), z = tz * TZ + zr + (k >> 2) * (TZ / 2);
            pin[k] = false;
            pu[k] = pw[k] = pv[k] = 0.f;
            if (x < nx && y < ny && z < nz) {
                pin[k] = scan_coords(P, fmaf((float)x, P->gsx, P->gox), fmaf((float)y, P->gsy, P->goy),
                                     fmaf((float)z, P->gsz, P->goz), pu[k], pw[k], pv[k]);
            }
            if (pin[k]) {
                int i0;
                float f;
                lerp_axis(pu[k], nlx, i0, f);
                lo_x = min(lo_x, i0);
                hi_x = max(hi_x, min(i0 + 1, nlx - 1));
                lerp_axis(pv[k], nd, i0, f);
                lo_v = min(lo_v, i0);
                hi_v = max(hi_v, min(i0 + 1, nd - 1));
                if (is3d) {
                    lerp_axis(pw[k], nly, i0, f);
                    lo_y = min(lo_y, i0);
                    hi_y = max(hi_y, min(i0 + 1, nly - 1));
                }
            }
        }
        if (!is3d) lo_y = hi_y = 0;
        // block-wide bounding box
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo_x = min(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
            hi_x = max(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
            lo_y = min(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
            hi_y = max(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
            lo_v = min(lo_v, __shfl_xor_sync(0xffffffffu, lo_v, o));
            hi_v = max(hi_v, __shfl_xor_sync(0xffffffffu, hi_v, o));
        }
        if ((t & 31) == 0) {
            red[0][t >> 5] = lo_x;
            red[1][t >> 5] = hi_x;
            red[2][t >> 5] = lo_y;
            red[3][t >> 5] = hi_y;
            red[4][t >> 5] = lo_v;
            red[5][t >> 5] = hi_v;
        }
        __syncthreads();
        int bx0 = red[0][0], bx1 = red[1][0], by0 = red[2][0], by1 = red[3][0], bv0 = red[4][0], bv1 = red[5][0];
        for (int w8 = 1; w8 < 8; ++w8) {
            bx0 = min(bx0, red[0][w8]);
            bx1 = max(bx1, red[1][w8]);
            by0 = min(by0, red[2][w8]);
            by1 = max(by1, red[3][w8]);
            bv0 = min(bv0, red[4][w8]);
            bv1 = max(bv1, red[5][w8]);
        }
        const bool any = bx1 >= bx0;
        // depth runs are contiguous in bm: stage whole 4-byte words when lines start 4-byte aligned
        const bool words = (nd & 3) == 0 && (reinterpret_cast<uintptr_t>(F.bm) & 3) == 0;
        if (words) bv0 &= ~3;
        const int nbx = bx1 - bx0 + 1, nby = by1 - by0 + 1;
        const int nbv = words ? ((bv1 - bv0) | 3) + 1 : bv1 - bv0 + 1;   // staged depths per line
        const bool staged = any && (long long)nbx * nby * nbv <= kScanBox;
        if (staged) {
            // box[(iy - by0) * nbx * nbv + (ix - bx0) * nbv + (iv - bv0)]
            const int rows = nbx * nby;
            if (words) {
                const int nw = nbv >> 2, total = rows * nw;
                for (int base = 0; base < total; base += 256 * 4) {
                    uint32_t r[4];
                    int dsti[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {   // all loads in flight before the stores
                        const int id = base + t + 256 * u;
                        dsti[u] = -1;
                        if (id < total) {
                            const int row = id / nw, wi = id - row * nw;
                            const int iy = by0 + row / nbx, ix = bx0 + row % nbx;
                            r[u] = __ldg(reinterpret_cast<const uint32_t *>(F.bm + ((long long)iy * nlx + ix) * nd + bv0) + wi);
                            dsti[u] = id;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (dsti[u] >= 0) reinterpret_cast<uint32_t *>(box)[dsti[u]] = r[u];
                }
            } else {
                for (int rrow = t / 32; rrow < rows; rrow += 8) {
                    const int iy = by0 + rrow / nbx, ix = bx0 + rrow % nbx;
                    const uint8_t *src = F.bm + ((long long)iy * nlx + ix) * nd + bv0;
                    uint8_t *dst = box + rrow * nbv;
                    for (int k = t & 31; k < nbv; k += 32) dst[k] = src[k];
                }
            }
        }
        __syncthreads();
        uint8_t outv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            outv[k] = 0;
            if (!pin[k]) continue;
            if (staged)
                outv[k] = lerp_lines(P, box - (bx0 * nbv + by0 * nbx * nbv + bv0), nbv, nbx * nbv, 1, pu[k], pw[k],
                                     pv[k]);
            else
                outv[k] = lerp_lines(P, F.bm, nd, nlx * nd, 1, pu[k], pw[k], pv[k]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int z = tz * TZ + zr + h * (TZ / 2);
            if (y >= ny || z >= nz || x0 >= nx) continue;
            uint8_t *dst = F.img + ((long long)z * ny + y) * nx + x0;
            if (x0 + 4 <= nx && (reinterpret_cast<uintptr_t>(dst) & 3) == 0) {
                *reinterpret_cast<uint32_t *>(dst) = (uint32_t)outv[4 * h] | ((uint32_t)outv[4 * h + 1] << 8) |
                                                      ((uint32_t)outv[4 * h + 2] << 16) |
                                                      ((uint32_t)outv[4 * h + 3] << 24);
            } else {
                for (int k = 0; k < 4; ++k)
                    if (x0 + k < nx) dst[k] = outv[4 * h + k];
            }
        }
        __syncthreads();
    }
}

// Linear layouts: the inverse map is separable (u from x, v from z).  A CTA
// covers 32 columns x 64 rows of up to kScanGroup frames of one plan: the
// coordinates are computed once and the frames' loads issue together.  Each
// warp takes 4 columns; its lanes walk 32 consecutive rows of one column at a
// time, so both lines it interpolates are read within one or two cache lines per
// load; the tiles go through shared memory so that rows are written out
// coalesced.  Same arithmetic as scan_coords / lerp_lines.
// When the tile's lines and depths fit (kLinStageLines lines, kLinStageRow bytes a line), the
// CTA first copies them from every frame into shared memory with 16-byte loads (each line's
// bytes from the 16-byte boundary at or below its first depth) and interpolates from there.
constexpr int kLinStageLines = 20, kLinStageRow = 288;
__global__ void __launch_bounds__(256) scanconvert_linear_kernel(const __grid_constant__ ScanLaunch L) {
    __shared__ uint8_t tile[kScanGroup][64][33];
    __shared__ __align__(16) uint8_t stg[kScanGroup][kLinStageLines][kLinStageRow];
    const int f0 = L.g0[blockIdx.y], nf = L.gn[blockIdx.y];
    const DevPlan *P = L.f[f0].plan;
    const int nx = P->gnx, nz = P->gnz, nlx = P->lines_x, nd = P->n_depth;
    const int cols = (nx + 31) >> 5;
    const int xb = (blockIdx.x % cols) * 32, zb = (blockIdx.x / cols) * 64;
    if (zb >= nz) return;
    const uint8_t *bm[kScanGroup];
#pragma unroll
    for (int f = 0; f < kScanGroup; ++f) bm[f] = L.f[f0 + (f < nf ? f : 0)].bm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the lines and depths this tile reads (the clamped maps are monotonic in x and z)
    int lo_l, hi_l, lo_d, hi_d;
    {
        int ia, ib, da, db;
        float fr;
        lerp_axis((fmaf((float)xb, P->gsx, P->gox) - P->u0) * P->du_inv, nlx, ia, fr);
        lerp_axis((fmaf((float)min(xb + 31, nx - 1), P->gsx, P->gox) - P->u0) * P->du_inv, nlx, ib, fr);
        lerp_axis((fmaf((float)zb, P->gsz, P->goz) - P->apz - P->v0) * P->dv_inv, nd, da, fr);
        lerp_axis((fmaf((float)min(zb + 63, nz - 1), P->gsz, P->goz) - P->apz - P->v0) * P->dv_inv, nd, db, fr);
        lo_l = min(ia, ib), hi_l = min(max(ia, ib) + 1, nlx - 1);
        lo_d = min(da, db), hi_d = min(max(da, db) + 1, nd - 1);
    }
    const long long frame_bytes = (long long)nlx * nd;
    bool staged = hi_l - lo_l + 1 <= kLinStageLines && hi_d - lo_d + 1 + 15 <= kLinStageRow && (frame_bytes & 15) == 0;
#pragma unroll
    for (int f = 0; f < kScanGroup; ++f) staged = staged && (reinterpret_cast<uintptr_t>(bm[f]) & 15) == 0;
    if (staged) {
        const int nL = hi_l - lo_l + 1, nC = (hi_d - lo_d + 1 + 15 + 15) >> 4;   // 16-byte chunks a line
        for (int k = threadIdx.x; k < nf * nL * nC; k += blockDim.x) {
            const int f = k / (nL * nC), r = k - f * (nL * nC), l = r / nC, c = r - l * nC;
            const long long a = (((long long)(lo_l + l) * nd + lo_d) & ~15LL) + 16 * c;
            static_assert(kScanGroup == 4, "frame pointer by selects");   // (a run-time index: local memory)
            const uint8_t *src = f == 0 ? bm[0] : f == 1 ? bm[1] : f == 2 ? bm[2] : bm[3];
            if (a < frame_bytes)   // chunks past the frame's last byte are never read
                *reinterpret_cast<uint4 *>(&stg[f][l][16 * c]) = __ldg(reinterpret_cast<const uint4 *>(src + a));
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int xl = warp * 4 + c, x = xb + xl;
            const float u = (fmaf((float)x, P->gsx, P->gox) - P->u0) * P->du_inv;
            const bool in_u = x < nx && u >= -kInsideEps && u <= (float)(nlx - 1) + kInsideEps;
            int ix;
            float fx;
            lerp_axis(u, nlx, ix, fx);
            const int ix1 = ix + 1 < nlx ? ix + 1 : ix;
            // byte of depth lo_d of line l in its staged row: (l nd + lo_d) mod 16
            const int o0 = (int)(((long long)ix * nd + lo_d) & 15) - lo_d;
            const int o1 = (int)(((long long)ix1 * nd + lo_d) & 15) - lo_d;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int zl = h * 32 + lane, z = zb + zl;
                const float rz = fmaf((float)z, P->gsz, P->goz) - P->apz;
                const float v = (rz - P->v0) * P->dv_inv;
                const bool in = in_u && z < nz && v >= -kInsideEps && v <= (float)(nd - 1) + kInsideEps;
                int iv;
                float fv;
                lerp_axis(v, nd, iv, fv);
                const int dv = iv + 1 < nd ? 1 : 0;
#pragma unroll
                for (int f = 0; f < kScanGroup; ++f) {
                    uint8_t out = 0;
                    if (in && f < nf &&
                        SUPRA_CHECK(ix >= lo_l && ix1 - lo_l < kLinStageLines && o0 + iv >= 0 && o1 + iv >= 0 &&
                                    o0 + iv + dv < kLinStageRow && o1 + iv + dv < kLinStageRow)) {
                        const uint8_t *b0 = &stg[f][ix - lo_l][o0 + iv];
                        const uint8_t *b1 = &stg[f][ix1 - lo_l][o1 + iv];
                        const float c0 = fmaf(fv, byte_f(b0[dv]) - byte_f(b0[0]), byte_f(b0[0]));
                        const float c1 = fmaf(fv, byte_f(b1[dv]) - byte_f(b1[0]), byte_f(b1[0]));
                        out = floor_byte(fmaf(fx, c1 - c0, c0) + 0.5f);
                    }
                    tile[f][zl][xl] = out;
                }
            }
        }
    } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int xl = warp * 4 + c, x = xb + xl;
        const float u = (fmaf((float)x, P->gsx, P->gox) - P->u0) * P->du_inv;
        const bool in_u = x < nx && u >= -kInsideEps && u <= (float)(nlx - 1) + kInsideEps;
        int ix;
        float fx;
        lerp_axis(u, nlx, ix, fx);
        const int dx = ix + 1 < nlx ? nd : 0;
        const long long lo = (long long)ix * nd;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int zl = h * 32 + lane, z = zb + zl;
            const float rz = fmaf((float)z, P->gsz, P->goz) - P->apz;
            const float v = (rz - P->v0) * P->dv_inv;
            const bool in = in_u && z < nz && v >= -kInsideEps && v <= (float)(nd - 1) + kInsideEps;
            int iv;
            float fv;
            lerp_axis(v, nd, iv, fv);
            const int dv = iv + 1 < nd ? 1 : 0;
#pragma unroll
            for (int f = 0; f < kScanGroup; ++f) {
                uint8_t out = 0;
                if (in && f < nf) {
                    const uint8_t *b = bm[f] + lo + iv;
                    const float c0 = fmaf(fv, byte_f(b[dv]) - byte_f(b[0]), byte_f(b[0]));
                    const float c1 = fmaf(fv, byte_f(b[dx + dv]) - byte_f(b[dx]), byte_f(b[dx]));
                    out = floor_byte(fmaf(fx, c1 - c0, c0) + 0.5f);
                }
                tile[f][zl][xl] = out;
            }
        }
    }
    }
    __syncthreads();
    // per frame, 64 rows x 32 bytes: thread -> (row, 8-byte chunk)
    const int row = threadIdx.x >> 2, ch = (threadIdx.x & 3) * 8, z = zb + row;
    if (z < nz) {
        for (int f = 0; f < nf; ++f) {
            uint8_t *dst = L.f[f0 + f].img + (long long)z * nx + xb + ch;
            if (xb + ch + 8 <= nx && (reinterpret_cast<uintptr_t>(dst) & 7) == 0) {
                uint2 w;
                w.x = (uint32_t)tile[f][row][ch] | ((uint32_t)tile[f][row][ch + 1] << 8) |
                      ((uint32_t)tile[f][row][ch + 2] << 16) | ((uint32_t)tile[f][row][ch + 3] << 24);
                w.y = (uint32_t)tile[f][row][ch + 4] | ((uint32_t)tile[f][row][ch + 5] << 8) |
                      ((uint32_t)tile[f][row][ch + 6] << 16) | ((uint32_t)tile[f][row][ch + 7] << 24);
                *reinterpret_cast<uint2 *>(dst) = w;
            } else {
                for (int k = 0; k < 8; ++k)
                    if (xb + ch + k < nx) dst[k] = tile[f][row][ch + k];
            }
        }
    }
}

}  // namespace supra
