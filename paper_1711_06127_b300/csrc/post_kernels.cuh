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
__global__ void __launch_bounds__(kEnvTile) envelope_kernel(const DevPlan *__restrict__ P, const float *__restrict__ rf,
                                                            float *__restrict__ env) {
    __shared__ float x[kEnvTile + kTapSlots];
    __shared__ float tc[kTapSlots], ts[kTapSlots];
    const int line = blockIdx.y;
    const int nd = P->n_depth;
    const int i0 = blockIdx.x * kEnvTile;
    const float *src = rf + (long long)line * nd;
    for (int k = threadIdx.x; k < kTapSlots; k += kEnvTile) {
        tc[k] = P->taps_c[k];
        ts[k] = P->taps_s[k];
    }
    for (int k = threadIdx.x; k < kEnvTile + kTapSlots - 1; k += kEnvTile) {
        const int i = i0 - kTapSlots / 2 + k;   // x[k] = rf(i0 - 32 + k)
        x[k] = (i >= 0 && i < nd) ? src[i] : 0.0f;
    }
    __syncthreads();
    const int i = i0 + threadIdx.x;
    if (i >= nd) return;
    float re = 0.0f, im = 0.0f;
    const float *xp = x + threadIdx.x + kTapSlots - 1;   // rf(i + 31)
#pragma unroll 8
    for (int k = 0; k < kTapSlots; ++k) {
        re = fmaf(tc[k], xp[-k], re);
        im = fmaf(ts[k], xp[-k], im);
    }
    env[(long long)line * nd + i] = 2.0f * sqrtf(fmaf(re, re, im * im));
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
struct ScanLaunch {
    int n;
    ScanFrame f[kMaxScanFrames];
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

__device__ __forceinline__ void lerp_axis(float u, int n, int &i0, float &f) {
    u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
    i0 = min((int)floorf(u), max(n - 2, 0));
    f = u - (float)i0;
}

__device__ __forceinline__ uint8_t scan_point(const DevPlan *P, const uint8_t *__restrict__ bm, float x, float y,
                                              float z) {
    float u, w, v;
    if (!scan_coords(P, x, y, z, u, w, v)) return 0;
    const int nlx = P->lines_x, nd = P->n_depth;
    int ix, iv;
    float fx, fv;
    lerp_axis(u, nlx, ix, fx);
    lerp_axis(v, nd, iv, fv);
    const int ix1 = min(ix + 1, nlx - 1), iv1 = min(iv + 1, nd - 1);
    float val;
    if (P->geometry == SUPRA_GEOM_PYRAMID) {
        int iy;
        float fy;
        lerp_axis(w, P->lines_y, iy, fy);
        const int iy1 = min(iy + 1, P->lines_y - 1);
        const uint8_t *b00 = bm + ((long long)iy * nlx + ix) * nd;
        const uint8_t *b01 = bm + ((long long)iy * nlx + ix1) * nd;
        const uint8_t *b10 = bm + ((long long)iy1 * nlx + ix) * nd;
        const uint8_t *b11 = bm + ((long long)iy1 * nlx + ix1) * nd;
        const float c00 = fmaf(fv, (float)b00[iv1] - (float)b00[iv], (float)b00[iv]);
        const float c01 = fmaf(fv, (float)b01[iv1] - (float)b01[iv], (float)b01[iv]);
        const float c10 = fmaf(fv, (float)b10[iv1] - (float)b10[iv], (float)b10[iv]);
        const float c11 = fmaf(fv, (float)b11[iv1] - (float)b11[iv], (float)b11[iv]);
        const float c0 = fmaf(fx, c01 - c00, c00), c1 = fmaf(fx, c11 - c10, c10);
        val = fmaf(fy, c1 - c0, c0);
    } else {
        const uint8_t *b0 = bm + (long long)ix * nd;
        const uint8_t *b1 = bm + (long long)ix1 * nd;
        const float c0 = fmaf(fv, (float)b0[iv1] - (float)b0[iv], (float)b0[iv]);
        const float c1 = fmaf(fv, (float)b1[iv1] - (float)b1[iv], (float)b1[iv]);
        val = fmaf(fx, c1 - c0, c0);
    }
    return (uint8_t)fminf(fmaxf(floorf(val + 0.5f), 0.0f), 255.0f);
}

// Scan conversion: blockIdx.y selects the frame; each thread writes 4 consecutive x.
__global__ void __launch_bounds__(256) scanconvert_kernel(const __grid_constant__ ScanLaunch L) {
    const ScanFrame &F = L.f[blockIdx.y];
    const DevPlan *P = F.plan;
    const int nx = P->gnx, ny = P->gny, nz = P->gnz;
    const int qx = (nx + 3) >> 2;
    const long long nquads = (long long)qx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nquads;
         q += (long long)gridDim.x * blockDim.x) {
        const int xq = (int)(q % qx);
        const long long rest = q / qx;
        const int iy = (int)(rest % ny), iz = (int)(rest / ny);
        const float y = fmaf((float)iy, P->gsy, P->goy), z = fmaf((float)iz, P->gsz, P->goz);
        uint8_t out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ix = xq * 4 + k;
            out[k] = ix < nx ? scan_point(P, F.bm, fmaf((float)ix, P->gsx, P->gox), y, z) : 0;
        }
        uint8_t *dst = F.img + (rest * nx) + xq * 4;
        if ((nx & 3) == 0 && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
            *reinterpret_cast<uint32_t *>(dst) =
                (uint32_t)out[0] | ((uint32_t)out[1] << 8) | ((uint32_t)out[2] << 16) | ((uint32_t)out[3] << 24);
        } else {
            for (int k = 0; k < 4; ++k)
                if (xq * 4 + k < nx) dst[k] = out[k];
        }
    }
}

}  // namespace supra
