// render_kernel.cuh -- headless volume rendering of a scan-converted volume
// (the paper shows rendered volumes of its 3D output, Fig. 4b; this is the
// textbook orthographic ray march into a device buffer, no graphics API).
//
// Pixel (px, py), sample k sits at voxel coordinates
//   u = base + px R + py D + k S
// (camera mapped to voxel space on the host in FP64).  Samples are trilinear
// in the uint8 volume, 0 outside [0, n - 1] on any axis.  MIP keeps the
// maximum; emission-absorption composites front to back with a linear ramp
// transfer function: a = clamp((v - lo) / (hi - lo), 0, 1) alpha, c = v / 255,
// C += T a c, T *= 1 - a (no early termination).
#pragma once
#include <cstdint>

namespace supra {

struct RenderArgs {
    const uint8_t *vol;
    int nx, ny, nz;
    float bx, by, bz;   // base
    float rx, ry, rz;   // R: one pixel right
    float dx, dy, dz;   // D: one pixel down
    float sx, sy, sz;   // S: one sample along the ray
    int n_steps, W, H, mode;
    float lo, inv_range, alpha;
    float *image;       // [H][W]
};

constexpr int kRenderTile = 16;

__device__ __forceinline__ float voxel(const uint8_t *__restrict__ v, int nx, int nxy, int x, int y, int z) {
    return (float)__ldg(v + (long long)z * nxy + y * nx + x);
}

__global__ void __launch_bounds__(kRenderTile *kRenderTile) render_kernel(const RenderArgs a) {
    const int px = blockIdx.x * kRenderTile + threadIdx.x, py = blockIdx.y * kRenderTile + threadIdx.y;
    if (px >= a.W || py >= a.H) return;
    const float ox = fmaf((float)py, a.dx, fmaf((float)px, a.rx, a.bx));
    const float oy = fmaf((float)py, a.dy, fmaf((float)px, a.ry, a.by));
    const float oz = fmaf((float)py, a.dz, fmaf((float)px, a.rz, a.bz));
    const float mx = (float)(a.nx - 1), my = (float)(a.ny - 1), mz = (float)(a.nz - 1);
    const int nxy = a.nx * a.ny;
    const int xm = max(a.nx - 2, 0), ym = max(a.ny - 2, 0), zm = max(a.nz - 2, 0);
    float best = 0.0f, col = 0.0f, T = 1.0f;
    for (int k = 0; k < a.n_steps; ++k) {
        const float fk = (float)k;
        const float ux = fmaf(fk, a.sx, ox), uy = fmaf(fk, a.sy, oy), uz = fmaf(fk, a.sz, oz);
        float v = 0.0f;
        if (ux >= 0.0f && ux <= mx && uy >= 0.0f && uy <= my && uz >= 0.0f && uz <= mz) {
            const int x0 = min((int)ux, xm), y0 = min((int)uy, ym), z0 = min((int)uz, zm);
            const float fx = ux - (float)x0, fy = uy - (float)y0, fz = uz - (float)z0;
            const int x1 = min(x0 + 1, a.nx - 1), y1 = min(y0 + 1, a.ny - 1), z1 = min(z0 + 1, a.nz - 1);
            const float c000 = voxel(a.vol, a.nx, nxy, x0, y0, z0), c100 = voxel(a.vol, a.nx, nxy, x1, y0, z0);
            const float c010 = voxel(a.vol, a.nx, nxy, x0, y1, z0), c110 = voxel(a.vol, a.nx, nxy, x1, y1, z0);
            const float c001 = voxel(a.vol, a.nx, nxy, x0, y0, z1), c101 = voxel(a.vol, a.nx, nxy, x1, y0, z1);
            const float c011 = voxel(a.vol, a.nx, nxy, x0, y1, z1), c111 = voxel(a.vol, a.nx, nxy, x1, y1, z1);
            const float c00 = fmaf(fx, c100 - c000, c000), c10 = fmaf(fx, c110 - c010, c010);
            const float c01 = fmaf(fx, c101 - c001, c001), c11 = fmaf(fx, c111 - c011, c011);
            const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
            v = fmaf(fz, c1 - c0, c0);
        }
        if (a.mode == 0) {
            best = fmaxf(best, v);
        } else {
            const float al = fminf(fmaxf((v - a.lo) * a.inv_range, 0.0f), 1.0f) * a.alpha;
            col = fmaf(T * al, v * (1.0f / 255.0f), col);
            T *= 1.0f - al;
        }
    }
    a.image[(long long)py * a.W + px] = a.mode == 0 ? best : col;
}

}  // namespace supra
