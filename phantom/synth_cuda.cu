// synth_cuda.cu -- GPU twin of phantom.synth_channels' echo accumulation (the
// forward acquisition model only: where each scatterer's echo arrives on each
// element).  Input generation for the tests and the benchmark; no part of the
// beamforming chain lives here.
//
// For transmit t and element e the noise-free record is
//   sum over (scatterer p, transmit t) pairs of
//     a_p * exp(-(k/fs - T)^2 / (2 s^2)) * cos(2 pi fc (k/fs - T)),  |k/fs - T| <= half,
//   T = (|p - o_t| + |p - x_e|) / c  (a plane-wave transmit of direction n: n.(p - o_t) + |p - x_e|),
// with a_p already including the transmit-beam weight.  One CTA accumulates 4
// elements of one transmit in shared memory, in 32.32 fixed point with integer
// atomics: each term is rounded to a multiple of 2^-32 and integer sums do not
// depend on the order the threads add them in, so the records are the same bits
// on every run.
#include <cuda_runtime.h>
#include <math.h>

namespace {

constexpr int kElems = 4;
constexpr float kFix = 4294967296.0f;   // 2^32

__global__ void __launch_bounds__(256) echo_kernel(int n_el, int n_s, const float *__restrict__ elem,
                                                   const float *__restrict__ tx_origin,
                                                   const float *__restrict__ tx_dir, const int *__restrict__ start,
                                                   const float4 *__restrict__ pairs, float c, float fs, float fc,
                                                   float sig, float half, int J, float *__restrict__ out) {
    extern __shared__ unsigned long long acc[];   // [kElems][n_s], two's complement 32.32 fixed point
    const int t = blockIdx.x, e0 = blockIdx.y * kElems;
    for (int k = threadIdx.x; k < kElems * n_s; k += blockDim.x) acc[k] = 0ull;
    __syncthreads();
    const float ox = tx_origin[3 * t], oy = tx_origin[3 * t + 1], oz = tx_origin[3 * t + 2];
    // plane-wave transmit (unit direction, zero for a spherical wave from the origin)
    const float nx = tx_dir[3 * t], ny = tx_dir[3 * t + 1], nz = tx_dir[3 * t + 2];
    const bool plane = nx != 0.0f || ny != 0.0f || nz != 0.0f;
    const float inv2s2 = 1.0f / (2.0f * sig * sig), w = 6.283185307179586f * fc;
    const int p0 = start[t], p1 = start[t + 1];
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const float4 q = pairs[p];
        const float dtx = plane ? nx * (q.x - ox) + ny * (q.y - oy) + nz * (q.z - oz)
                                : sqrtf((q.x - ox) * (q.x - ox) + (q.y - oy) * (q.y - oy) + (q.z - oz) * (q.z - oz));
        for (int j = 0; j < kElems && e0 + j < n_el; ++j) {
            const float *x = elem + 3 * (e0 + j);
            const float drx = sqrtf((q.x - x[0]) * (q.x - x[0]) + (q.y - x[1]) * (q.y - x[1]) + (q.z - x[2]) * (q.z - x[2]));
            const float T = (dtx + drx) / c;
            const int k0 = (int)ceilf((T - half) * fs);
            for (int i = 0; i < J; ++i) {
                const int k = k0 + i;
                if (k < 0 || k >= n_s) continue;
                const float dt = (float)k / fs - T;
                if (fabsf(dt) > half) continue;
                const float v = q.w * expf(-dt * dt * inv2s2) * cosf(w * dt);
                atomicAdd(&acc[j * n_s + k], (unsigned long long)llrintf(v * kFix));
            }
        }
    }
    __syncthreads();
    for (int j = 0; j < kElems && e0 + j < n_el; ++j) {
        float *dst = out + ((long long)t * n_el + e0 + j) * n_s;
        for (int k = threadIdx.x; k < n_s; k += blockDim.x)
            dst[k] = (float)((double)(long long)acc[j * n_s + k] * (1.0 / 4294967296.0));
    }
}

}  // namespace

// Accumulates the noise-free records float [n_tx][n_el][n_s] (device pointers).
// pairs: float4 (x, y, z, amplitude) grouped by transmit, start[t]..start[t+1].
// Returns 0 or a CUDA error code.
extern "C" __attribute__((visibility("default"))) int phantom_echoes(int n_tx, int n_el, int n_s, const float *elem,
                                                                     const float *tx_origin, const float *tx_dir,
                                                                     const int *start,
                                                                     const float *pairs, float c, float fs, float fc,
                                                                     float sig, float half, int J, float *out,
                                                                     void *stream) {
    const size_t smem = sizeof(unsigned long long) * kElems * (size_t)n_s;
    if (smem > 200 * 1024) return (int)cudaErrorInvalidValue;
    cudaFuncSetAttribute(echo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(n_tx, (n_el + kElems - 1) / kElems);
    echo_kernel<<<grid, 256, smem, static_cast<cudaStream_t>(stream)>>>(
        n_el, n_s, elem, tx_origin, tx_dir, start, reinterpret_cast<const float4 *>(pairs), c, fs, fc, sig, half, J, out);
    return (int)cudaGetLastError();
}
