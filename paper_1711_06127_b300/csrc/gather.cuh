// gather.cuh -- delayed, interpolated samples of single elements at one pixel,
// for the per-pixel beamformers (minimum variance, learned apodization).  Same
// receive delays, linear interpolation, zero padding and F-number aperture as
// the delay-and-sum kernel (Sec. 2 item 1), evaluated one element at a time.
#pragma once
#include "common.cuh"
#include "das_kernel.cuh"

namespace supra {

struct PixelGeo {
    LineGeo lg;
    float r, qx, qy, inv_a, base;
    int kt;
    const int16_t *rec0;
};

// Image point, aperture centre and half-width, and the delay base of depth i
// (< n_depth) on `line`.
__device__ __forceinline__ PixelGeo pixel_geo(const DevPlan *__restrict__ P, const int16_t *__restrict__ ch, int line,
                                              int i) {
    PixelGeo g;
    g.lg = P->lines[line];
    const int tile = i / kTD;
    g.r = P->depth0 + (float)i * P->depth_step;
    const float px = fmaf(g.r, g.lg.dx, g.lg.ox), py = fmaf(g.r, g.lg.dy, g.lg.oy), pz = fmaf(g.r, g.lg.dz, g.lg.oz);
    g.qx = fminf(fmaxf(px, P->xmin), P->xmax);
    g.qy = fminf(fmaxf(py, P->ymin), P->ymax);
    g.inv_a = 1.0f / fmaxf(pz * P->inv2f, P->amin);
    g.base = P->tile_f[tile] + P->a1 * (float)(i - tile * kTD) + tx_excess(g.r, g.lg.bt, g.lg.gt, g.lg.plane) * P->fsc;
    g.kt = P->tile_k[tile];
    g.rec0 = ch + (long long)g.lg.tx * P->n_el * P->n_s;
    return g;
}

// Sample of element e (< n_el); act = inside the aperture (x = 0 outside).
__device__ __forceinline__ float element_sample(const DevPlan *__restrict__ P, const PixelGeo &g, int e, bool &act) {
    const float4 xe = __ldg(&P->elem[e]);
    act = fabsf((xe.x - g.qx) * g.inv_a) <= 1.0f && fabsf((xe.y - g.qy) * g.inv_a) <= 1.0f;
    if (!act) return 0.0f;
    const float mx = g.lg.ox - xe.x, my = g.lg.oy - xe.y, mz = g.lg.oz - xe.z;
    const float beta = g.lg.dx * mx + g.lg.dy * my + g.lg.dz * mz;
    const float gamma = mx * mx + my * my + mz * mz;
    const float s = g.base + path_excess(g.r, beta, gamma) * P->fsc;
    const float fl = floorf(s);
    const float phi = s - fl;
    const long long k = (long long)g.kt + (long long)fl;
    const int n_s = P->n_s;
    const int16_t *rec = g.rec0 + (long long)e * n_s;
    const float x0 = (k >= 0 && k < n_s) ? (float)__ldg(rec + k) : 0.0f;
    const float x1 = (k + 1 >= 0 && k + 1 < n_s) ? (float)__ldg(rec + k + 1) : 0.0f;
    return fmaf(phi, x1 - x0, x0);
}

}  // namespace supra
