// tiDAS row-wise lateral convolution (Eq. (2.13)) and its transpose, FP32 on
// CUDA cores.  One block per (row, group of frames).  The row's kernel and
// input lines are staged in shared memory, zero padded; every thread makes
// kV consecutive outputs from a register window of 2 kV inputs, so each
// shared-memory word feeds kV / 2 multiply-adds.  Lines are stored
// column-blocked (element j at (j % kV) * W + j / kV, W odd) so that the 32
// lanes of a warp, whose windows start kV elements apart, read 32
// consecutive words: no bank conflicts.
#include "common.cuh"

namespace tidas {

constexpr int kV = 16;      // outputs per thread
constexpr int kFB = 4;      // frames per block
constexpr int kThreads = 128;

// y[x] = sum_s hr[s] * rp[x + s], rp[j] = in[j - off] (zero outside [0, nx)).
__global__ void __launch_bounds__(kThreads) tidas_direct_kernel(
    const float* __restrict__ kern, int taps, int off, bool reverse, int nz, int nx,
    const float* __restrict__ in, float* __restrict__ out, int nf) {
    extern __shared__ float sm[];
    const int tpad = (taps + kV - 1) / kV * kV;
    const int len = nx + tpad + 2 * kV;          // staged line length
    const int W = ((len + kV - 1) / kV) | 1;     // column height, odd
    float* hr = sm;                              // [tpad]
    float* lines = sm + tpad;                    // [kFB][kV][W]
    const int iz = blockIdx.x;
    const int f0 = blockIdx.y * kFB;
    const int nfb = min(kFB, nf - f0);

    for (int s = threadIdx.x; s < tpad; s += blockDim.x) {
        float v = 0.f;
        if (s < taps) v = kern[(size_t)iz * taps + (reverse ? taps - 1 - s : s)];
        hr[s] = v;
    }
    for (int fb = 0; fb < nfb; ++fb) {
        const float* src = in + ((size_t)(f0 + fb) * nz + iz) * nx;
        float* ln = lines + fb * kV * W;
        for (int j = threadIdx.x; j < kV * W; j += blockDim.x) {
            const int x = j - off;
            ln[(j % kV) * W + j / kV] = (x >= 0 && x < nx) ? __ldg(src + x) : 0.f;
        }
    }
    __syncthreads();

    const int chunks = (nx + kV - 1) / kV;
    const bool vec = (nx % 4) == 0;
    for (int item = threadIdx.x; item < nfb * chunks; item += blockDim.x) {
        const int fb = item / chunks;
        const int c = item % chunks;
        const float* ln = lines + fb * kV * W + c;
        float y[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) y[v] = 0.f;
        for (int s = 0; s < tpad; s += kV) {
            const int sb = s / kV;
            float a[2 * kV], h[kV];
#pragma unroll
            for (int k = 0; k < 2 * kV; ++k) a[k] = ln[(k % kV) * W + sb + k / kV];
#pragma unroll
            for (int k = 0; k < kV; k += 4) {
                const float4 t = *reinterpret_cast<const float4*>(hr + s + k);
                h[k] = t.x;
                h[k + 1] = t.y;
                h[k + 2] = t.z;
                h[k + 3] = t.w;
            }
#pragma unroll
            for (int k = 0; k < kV; ++k)
#pragma unroll
                for (int v = 0; v < kV; ++v) y[v] = fmaf(h[k], a[v + k], y[v]);
        }
        const int x0 = c * kV;
        float* dst = out + ((size_t)(f0 + fb) * nz + iz) * nx + x0;
        if (vec && x0 + kV <= nx) {
#pragma unroll
            for (int v = 0; v < kV; v += 4)
                *reinterpret_cast<float4*>(dst + v) = make_float4(y[v], y[v + 1], y[v + 2], y[v + 3]);
        } else {
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (x0 + v < nx) dst[v] = y[v];
        }
    }
}

int launch_tidas_direct(const float* kern, int taps, int center, bool adjoint, int nz, int nx,
                        const float* in, float* out, int nf, cudaStream_t st) {
    const int tpad = (taps + kV - 1) / kV * kV;
    const int len = nx + tpad + 2 * kV;
    const int W = ((len + kV - 1) / kV) | 1;
    size_t smem = (size_t)(tpad + kFB * kV * W) * sizeof(float);
    if (smem > 220 * 1024) return set_error(TIDAS_ERR_UNSUPPORTED, "tidas direct: row too long");
    if (nx % 4 == 0 && ((uintptr_t)out % 16) != 0)
        return set_error(TIDAS_ERR_ARG, "tidas direct: output must be 16-byte aligned");
    cudaFuncSetAttribute(tidas_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    // forward: hr[s] = h[taps-1-s], off = taps-1-center; adjoint: hr = h, off = center
    const int off = adjoint ? center : taps - 1 - center;
    dim3 grid(nz, (nf + kFB - 1) / kFB);
    tidas_direct_kernel<<<grid, kThreads, smem, st>>>(kern, taps, off, !adjoint, nz, nx, in, out,
                                                     nf);
    return check_launch("tidas_direct_kernel");
}

}  // namespace tidas
