// mv_kernel.cuh -- exact minimum-variance (Capon) beamformer.  Not in the
// paper: it labels the data the learned apodization is trained on, is the
// fallback beamformer and the yardstick for the learned weights' error.
//
// Per pixel (one warp): the delayed, interpolated samples x of the active
// aperture (same delays and aperture rule as delay-and-sum, no apodization),
// subapertures x_l = x[l : l + L] (K = M - L + 1 of them), spatially smoothed
// covariance R = sum_l x_l x_l^T (the 1/K factor cancels in the weights),
// diagonal loading relative to the mean eigenvalue, R + loading * (trace(R) / L) * I,
// w = R^{-1} 1 / (1^T R^{-1} 1),
// y = w^T xbar with xbar = (1/K) sum_l x_l.  Fewer than two active elements:
// the delay-and-sum value.
//
// The loading bounds the condition number by 1 + L/loading; FP32 is used when
// that bound is at most 1e4, FP64 otherwise.
#pragma once
#include "common.cuh"
#include "das_kernel.cuh"

namespace supra {

constexpr int kMvMaxM = 256;   // active elements per pixel
template <typename T>
__host__ __device__ constexpr int mv_warps() { return sizeof(T) == 8 ? 4 : 8; }   // pixels per CTA (one per warp); static smem < 48 KB
constexpr int kMvMaxL = 32;

__device__ __forceinline__ float inv_sqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double inv_sqrt(double v) { return 1.0 / sqrt(v); }
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}

// FP32: four CTAs per SM (registers capped at 64; the factorisation is a chain of dependent
// steps per warp, so resident warps, not registers, bound it)
template <typename T>
__global__ void __launch_bounds__(mv_warps<T>() * 32, sizeof(T) == 8 ? 1 : 4) mv_kernel(const DevPlan *__restrict__ P,
                                                                const int16_t *__restrict__ ch, float *__restrict__ rf,
                                                                int Lreq, float loading) {
    constexpr int kMvWarps = mv_warps<T>();
    __shared__ float xs[kMvWarps][kMvMaxM];
    __shared__ T Rm[kMvWarps][kMvMaxL][kMvMaxL + 1];
    __shared__ __align__(16) T Cb[kMvWarps][2][kMvMaxL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = blockIdx.y;
    const int i = blockIdx.x * kMvWarps + warp;
    const int nd = P->n_depth;
    if (i >= nd) return;   // warp-uniform
    const LineGeo lg = P->lines[line];
    const int n_el = P->n_el, n_s = P->n_s;
    // image point, aperture, delay base (as in das_kernel)
    const int tile = i / kTD;
    const float r = P->depth0 + (float)i * P->depth_step;
    const float px = fmaf(r, lg.dx, lg.ox), py = fmaf(r, lg.dy, lg.oy), pz = fmaf(r, lg.dz, lg.oz);
    const float qx = fminf(fmaxf(px, P->xmin), P->xmax), qy = fminf(fmaxf(py, P->ymin), P->ymax);
    const float inv_a = 1.0f / fmaxf(pz * P->inv2f, P->amin);
    const float base = P->tile_f[tile] + P->a1 * (float)(i - tile * kTD) + tx_excess(r, lg.bt, lg.gt, lg.plane) * P->fsc;
    const int kt = P->tile_k[tile];
    const int16_t *rec0 = ch + (long long)lg.tx * n_el * n_s;
    // delayed samples of the active elements, compacted in element order
    int M = 0;
    for (int e0 = 0; e0 < n_el; e0 += 32) {
        const int e = e0 + lane;
        bool act = false;
        float x = 0.0f;
        if (e < n_el) {
            const float4 xe = __ldg(&P->elem[e]);
            act = fabsf((xe.x - qx) * inv_a) <= 1.0f && fabsf((xe.y - qy) * inv_a) <= 1.0f;
            if (act) {
                const float mx = lg.ox - xe.x, my = lg.oy - xe.y, mz = lg.oz - xe.z;
                const float beta = lg.dx * mx + lg.dy * my + lg.dz * mz;
                const float gamma = mx * mx + my * my + mz * mz;
                const float s = base + path_excess(r, beta, gamma) * P->fsc;
                const float fl = floorf(s);
                const float phi = s - fl;
                const long long k = (long long)kt + (long long)fl;
                const int16_t *rec = rec0 + (long long)e * n_s;
                const float x0 = (k >= 0 && k < n_s) ? (float)rec[k] : 0.0f;
                const float x1 = (k + 1 >= 0 && k + 1 < n_s) ? (float)rec[k + 1] : 0.0f;
                x = fmaf(phi, x1 - x0, x0);
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, act);
        const int pos = M + __popc(mask & ((1u << lane) - 1u));
        if (act && pos < kMvMaxM) xs[warp][pos] = x;
        M += __popc(mask);
    }
    __syncwarp();
    float *out = rf + (long long)line * nd + i;
    if (M > kMvMaxM) {
        if (lane == 0) {
            *out = 0.0f;
            set_status(SUPRA_EINTERNAL);
        }
        return;
    }
    if (M < 2) {
        if (lane == 0) *out = M == 1 ? xs[warp][0] : 0.0f;
        return;
    }
    const int L = min(Lreq, M), K = M - L + 1;
    const float *x = xs[warp];
    T(*R)[kMvMaxL + 1] = Rm[warp];
    // covariance: lane d walks the d-th diagonal, R[a][a+d] = R[a-1][a-1+d] + x[a-1+K] x[a-1+K+d] - x[a-1] x[a-1+d];
    // its first pass also sums lane d's entry of the averaged subaperture (sum_l x[l + d])
    T xb = 0;
    if (lane < L) {
        const int d = lane;
        T acc = 0;
        for (int l = 0; l < K; ++l) {
            const T xd = (T)x[l + d];
            acc += (T)x[l] * xd;
            xb += xd;
        }
        R[0][d] = acc;
        R[d][0] = acc;
        for (int a = 1; a + d < L; ++a) {
            acc += (T)x[a - 1 + K] * (T)x[a - 1 + K + d] - (T)x[a - 1] * (T)x[a - 1 + d];
            R[a][a + d] = acc;
            R[a + d][a] = acc;
        }
    }
    __syncwarp();
    // trace and loading; dimensions past L become an identity block
    T tr = lane < L ? R[lane][lane] : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (tr == (T)0) {   // all samples zero (e.g. delays past the record): R = 0, output 0
        if (lane == 0) *out = 0.0f;
        return;
    }
    const T delta = (T)loading * tr / (T)L;
    T rr[kMvMaxL];
#pragma unroll
    for (int j = 0; j < kMvMaxL; ++j) {
        if (lane < L && j < L) rr[j] = R[lane][j] + (j == lane ? delta : (T)0);
        else rr[j] = (j == lane) ? (T)1 : (T)0;
    }
    // Cholesky R = G G^T, lane i keeps row i of G in rr[0..i] and lane k the reciprocal
    // 1 / G[k][k] (multiplications instead of divisions in the factorisation and both
    // solves).  Column k reaches the lanes through a per-warp shared buffer (double
    // buffered), read four entries at a time.
    bool bad = false;
    T dinv = (T)1;
    T *colbuf = Cb[warp][0];
#pragma unroll
    for (int k = 0; k < kMvMaxL; ++k) {
        const T dkk = __shfl_sync(0xffffffffu, rr[k], k);
        bad |= !(dkk > (T)0);
        const T ginv = inv_sqrt(dkk > (T)0 ? dkk : (T)1);
        if (lane == k) {
            rr[k] = dkk * ginv;
            dinv = ginv;
        } else if (lane > k) {
            rr[k] *= ginv;
        }
        if (k + 1 < kMvMaxL) {
            T *col = colbuf + (k & 1) * kMvMaxL;
            col[lane] = rr[k];
            __syncwarp();
#pragma unroll
            for (int jb = (k + 1) & ~3; jb < kMvMaxL; jb += 4) {
                T g4[4];
                load4(col + jb, g4);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = jb + t;
                    if (j > k && lane >= j) rr[j] -= rr[k] * g4[t];
                }
            }
        }
    }
    // forward G y = b (b = 1 on the first L dimensions)
    T yv = 0, sacc = 0;
#pragma unroll
    for (int j = 0; j < kMvMaxL; ++j) {
        if (lane == j) yv = ((j < L ? (T)1 : (T)0) - sacc) * dinv;
        const T yj = __shfl_sync(0xffffffffu, yv, j);
        if (lane > j) sacc += rr[j] * yj;
    }
    // backward G^T z = y with G from shared memory (the diagonal as its reciprocal)
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kMvMaxL; ++j)
        if (j <= lane) R[lane][j] = j == lane ? dinv : rr[j];
    __syncwarp();
    T zv = 0, tacc = 0;
#pragma unroll
    for (int j = kMvMaxL - 1; j >= 0; --j) {
        if (lane == j) zv = (yv - tacc) * R[j][j];
        const T zj = __shfl_sync(0xffffffffu, zv, j);
        if (lane < j) tacc += R[j][lane] * zj;
    }
    // weights, averaged subaperture, output
    T zs = lane < L ? zv : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(0xffffffffu, zs, o);
    T part = 0;
    if (lane < L) part = (zv / zs) * (xb / (T)K);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) {
        *out = (float)part;
        if (bad) set_status(SUPRA_EINTERNAL);
    }
}

}  // namespace supra
