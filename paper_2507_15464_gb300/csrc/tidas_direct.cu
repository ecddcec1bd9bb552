// tiDAS row-wise lateral convolution (Eq. (2.13)) and its transpose, FP32 on
// CUDA cores.  One block per (row, run of frame groups); the row's kernel is
// staged once, and the input lines of kFB frames at a time are fetched with
// cp.async into one of two shared-memory buffers while the block computes
// the previous group from the other, so that loads and multiply-adds
// overlap.  Every thread makes kV consecutive outputs from a register window
// of 2 kV inputs, so each shared-memory word feeds kV / 2 multiply-adds.
// Lines are stored column-blocked (element j at (j % kV) * W + j / kV, W odd)
// so that the 32 lanes of a warp, whose windows start kV elements apart,
// read 32 consecutive words, and the 32 consecutive elements a warp fetches
// land in 32 distinct banks: no bank conflicts either way.
#include "common.cuh"

namespace tidas {

constexpr int kV = 16;      // outputs per thread
constexpr int kFB = 4;      // frames per group
constexpr int kThreads = 128;

// 4-byte global -> shared copy; src_bytes 0 writes a zero
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// y[x] = sum_s hr[s] * rp[x + s], rp[j] = in[j - off] (zero outside [0, nx)).
// WC > 0: lines are stored with the compile-time column height WC (>= the
// needed one, odd), so that every shared-memory read of the multiply-add loop
// is a base register plus an immediate offset, and a line fits kSlots
// staging slots per thread whose offsets are computed once per block.
// WC == 0: the column height is computed at run time (long rows).
constexpr int kSlots = 9;
template <int WC>
__global__ void __launch_bounds__(kThreads, 4) tidas_direct_kernel(
    const float* __restrict__ kern, int taps, int off, bool reverse, int nz, int nx,
    const float* __restrict__ in, float* __restrict__ out, int nf, int groups_per_block) {
    extern __shared__ float sm[];
    const int tpad = (taps + kV - 1) / kV * kV;
    const int len = nx + tpad + 2 * kV;          // staged line length
    const int W = WC > 0 ? WC : ((len + kV - 1) / kV) | 1;  // column height, odd
    constexpr bool PRE = WC > 0;
    float* hr = sm;                              // [tpad]
    float* bufs = sm + tpad;                     // [2][kFB][kV][W]
    const int buf_len = kFB * kV * W;
    const int iz = blockIdx.x;
    const int ngroups = (nf + kFB - 1) / kFB;
    const int g0 = blockIdx.y * groups_per_block;
    const int g1 = min(ngroups, g0 + groups_per_block);

    for (int s = threadIdx.x; s < tpad; s += blockDim.x) {
        float v = 0.f;
        if (s < taps) v = kern[(size_t)iz * taps + (reverse ? taps - 1 - s : s)];
        hr[s] = v;
    }
    // this thread's staging slots j = threadIdx.x + i * kThreads of a line:
    // destination (column-blocked) and source column, -1 outside [0, nx)
    int dsto[kSlots], srcx[kSlots];
#pragma unroll
    for (int i = 0; i < kSlots; ++i) {
        const int j = threadIdx.x + i * kThreads;
        const int x = j - off;
        dsto[i] = j < kV * W ? (j % kV) * W + j / kV : -1;
        srcx[i] = (x >= 0 && x < nx) ? x : -1;
    }
    // stage the kFB lines of group g into buffer b (one commit group)
    auto stage = [&](int g, int b) {
        float* dstb = bufs + b * buf_len;
#pragma unroll
        for (int fb = 0; fb < kFB; ++fb) {
            const int f = g * kFB + fb;
            const float* src = in + ((size_t)min(f, nf - 1) * nz + iz) * nx;
            float* ln = dstb + fb * kV * W;
            const bool live = f < nf;
            if (PRE) {
#pragma unroll
                for (int i = 0; i < kSlots; ++i) {
                    if (dsto[i] < 0) continue;
                    const bool inside = live && srcx[i] >= 0;
                    cp_async4(ln + dsto[i], src + (inside ? srcx[i] : 0), inside ? 4 : 0);
                }
            } else {
                for (int j = threadIdx.x; j < kV * W; j += blockDim.x) {
                    const int x = j - off;
                    const bool inside = live && x >= 0 && x < nx;
                    cp_async4(ln + (j % kV) * W + j / kV, src + (inside ? x : 0), inside ? 4 : 0);
                }
            }
        }
        cp_async_commit();
    };

    const int chunks = (nx + kV - 1) / kV;
    const bool vec = (nx % 4) == 0;
    if (g0 < g1) stage(g0, 0);
    for (int g = g0; g < g1; ++g) {
        const int b = (g - g0) & 1;
        if (g + 1 < g1) {
            stage(g + 1, b ^ 1);
            cp_async_wait<1>();  // this group's lines have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int nfb = min(kFB, nf - g * kFB);
        const float* lines = bufs + b * buf_len;
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
                    const float4 q = *reinterpret_cast<const float4*>(hr + s + k);
                    h[k] = q.x;
                    h[k + 1] = q.y;
                    h[k + 2] = q.z;
                    h[k + 3] = q.w;
                }
#pragma unroll
                for (int k = 0; k < kV; ++k)
#pragma unroll
                    for (int v = 0; v < kV; ++v) y[v] = fmaf(h[k], a[v + k], y[v]);
            }
            const int x0 = c * kV;
            float* dst = out + ((size_t)(g * kFB + fb) * nz + iz) * nx + x0;
            if (vec && x0 + kV <= nx) {
#pragma unroll
                for (int v = 0; v < kV; v += 4)
                    *reinterpret_cast<float4*>(dst + v) =
                        make_float4(y[v], y[v + 1], y[v + 2], y[v + 3]);
            } else {
#pragma unroll
                for (int v = 0; v < kV; ++v)
                    if (x0 + v < nx) dst[v] = y[v];
            }
        }
        __syncthreads();  // buffer b is refilled two groups later
    }
}

int launch_tidas_direct(const float* kern, int taps, int center, bool adjoint, int nz, int nx,
                        const float* in, float* out, int nf, cudaStream_t st) {
    const int tpad = (taps + kV - 1) / kV * kV;
    const int len = nx + tpad + 2 * kV;
    const int W = ((len + kV - 1) / kV) | 1;
    size_t smem = (size_t)(tpad + 2 * kFB * kV * W) * sizeof(float);
    if (smem > 220 * 1024) return set_error(TIDAS_ERR_UNSUPPORTED, "tidas direct: row too long");
    if (nx % 4 == 0 && ((uintptr_t)out % 16) != 0)
        return set_error(TIDAS_ERR_ARG, "tidas direct: output must be 16-byte aligned");
    constexpr int kWC = 65;  // kV * kWC <= kSlots * kThreads
    static_assert(kV * kWC <= kSlots * kThreads, "staging slots");
    const bool fixed = W <= kWC;
    if (fixed) smem = (size_t)(tpad + 2 * kFB * kV * kWC) * sizeof(float);
    auto kernel = fixed ? tidas_direct_kernel<kWC> : tidas_direct_kernel<0>;
    TIDAS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // forward: hr[s] = h[taps-1-s], off = taps-1-center; adjoint: hr = h, off = center
    const int off = adjoint ? center : taps - 1 - center;
    // rows x runs of frame groups: enough blocks for a few waves of 152 SMs
    const int ngroups = (nf + kFB - 1) / kFB;
    int runs = 1;
    while (runs < ngroups && (long long)nz * runs < 4LL * 152 * 4) runs *= 2;
    const int per = (ngroups + runs - 1) / runs;
    dim3 grid(nz, (ngroups + per - 1) / per);
    kernel<<<grid, kThreads, smem, st>>>(kern, taps, off, !adjoint, nz, nx, in, out, nf, per);
    return check_launch("tidas_direct_kernel");
}

// 2D band kernels (the PSF's axial extent): kernels [nz][kz][taps], slice u of
// row j = the image of a unit scatterer on row j at output row j + u - kz/2.
//   forward:  y[i][x]  = sum_u sum_t h[j][u][t] r[j][x - t + c],  j = i - u + kz/2
//   adjoint:  r[j][x'] = sum_u sum_t h[j][u][t] y[i][x' + t - c], i = j + u - kz/2
// Same block structure as the row-wise kernel, with a staging sequence over
// (frame group, u): every step stages the input lines of row i - u + kz/2
// (forward) or i + u - kz/2 (adjoint) and the kernel slice it needs, and the
// output registers accumulate over the valid u of a group before the store.
// A group holds nfg <= kFB frames, so that nfg * (nx / kV) outputs fit one
// per thread.
template <int WC>
__global__ void __launch_bounds__(kThreads, 4) tidas_direct2d_kernel(
    const float* __restrict__ kern, int kz, int taps, int off, bool adjoint, int nz, int nx,
    const float* __restrict__ in, float* __restrict__ out, int nf, int nfg, int groups_per_block) {
    extern __shared__ float sm[];
    const int tpad = (taps + kV - 1) / kV * kV;
    const int len = nx + tpad + 2 * kV;
    const int W = WC > 0 ? WC : ((len + kV - 1) / kV) | 1;
    const int step_len = tpad + nfg * kV * W;    // kernel slice + nfg lines
    float* bufs = sm;                             // [2][step_len]
    const int io = blockIdx.x;                    // output row
    const int cz = kz / 2;
    const int ngroups = (nf + nfg - 1) / nfg;
    const int g0 = blockIdx.y * groups_per_block;
    const int g1 = min(ngroups, g0 + groups_per_block);
    // valid u: input rows inside [0, nz)
    const int u_lo = adjoint ? max(0, cz - io) : max(0, io + cz - (nz - 1));
    const int u_hi = adjoint ? min(kz - 1, nz - 1 - io + cz) : min(kz - 1, io + cz);
    const int nu = u_hi >= u_lo ? u_hi - u_lo + 1 : 0;
    const int nsteps = (g1 - g0) * (nu > 0 ? nu : 1);

    // step k: group g0 + k / nu, slice u_lo + k % nu
    auto stage = [&](int k, int b) {
        float* hr = bufs + b * step_len;
        float* lines = hr + tpad;
        const int g = g0 + k / max(nu, 1), u = u_lo + k % max(nu, 1);
        const int irow = adjoint ? io + u - cz : io - u + cz;   // input row
        const int krow = adjoint ? io : irow;                   // kernel row
        const float* ks = kern + ((size_t)krow * kz + u) * taps;
        for (int s = threadIdx.x; s < tpad; s += blockDim.x) {
            float v = 0.f;
            if (nu > 0 && s < taps) v = __ldg(ks + (adjoint ? s : taps - 1 - s));
            hr[s] = v;
        }
        for (int fb = 0; fb < nfg; ++fb) {
            const int f = g * nfg + fb;
            const float* src = in + ((size_t)min(f, nf - 1) * nz + (nu > 0 ? irow : 0)) * nx;
            float* ln = lines + fb * kV * W;
            const bool live = nu > 0 && f < nf;
            for (int j = threadIdx.x; j < kV * W; j += blockDim.x) {
                const int x = j - off;
                const bool inside = live && x >= 0 && x < nx;
                cp_async4(ln + (j % kV) * W + j / kV, src + (inside ? x : 0), inside ? 4 : 0);
            }
        }
        cp_async_commit();
    };

    const int chunks = (nx + kV - 1) / kV;
    const bool vec = (nx % 4) == 0;
    // one output item per thread and group: nfg frames x chunks of kV columns
    const int item = threadIdx.x;
    const int fb = item / chunks, c = item % chunks;
    float y[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) y[v] = 0.f;
    if (nsteps > 0) stage(0, 0);
    for (int k = 0; k < nsteps; ++k) {
        const int b = k & 1;
        if (k + 1 < nsteps) {
            stage(k + 1, b ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int g = g0 + k / max(nu, 1);
        const int nfb = min(nfg, nf - g * nfg);
        const float* hr = bufs + b * step_len;
        if (item < nfb * chunks && nu > 0) {
            const float* ln = hr + tpad + fb * kV * W + c;
            for (int s = 0; s < tpad; s += kV) {
                const int sb = s / kV;
                float a[2 * kV], h[kV];
#pragma unroll
                for (int q = 0; q < 2 * kV; ++q) a[q] = ln[(q % kV) * W + sb + q / kV];
#pragma unroll
                for (int q = 0; q < kV; q += 4) {
                    const float4 t4 = *reinterpret_cast<const float4*>(hr + s + q);
                    h[q] = t4.x;
                    h[q + 1] = t4.y;
                    h[q + 2] = t4.z;
                    h[q + 3] = t4.w;
                }
#pragma unroll
                for (int q = 0; q < kV; ++q)
#pragma unroll
                    for (int v = 0; v < kV; ++v) y[v] = fmaf(h[q], a[v + q], y[v]);
            }
        }
        if (nu == 0 || k % nu == nu - 1) {  // the group's last slice: store, restart
            if (item < nfb * chunks) {
                const int x0 = c * kV;
                float* dst = out + ((size_t)(g * nfg + fb) * nz + io) * nx + x0;
                if (vec && x0 + kV <= nx) {
#pragma unroll
                    for (int v = 0; v < kV; v += 4)
                        *reinterpret_cast<float4*>(dst + v) =
                            make_float4(y[v], y[v + 1], y[v + 2], y[v + 3]);
                } else {
#pragma unroll
                    for (int v = 0; v < kV; ++v)
                        if (x0 + v < nx) dst[v] = y[v];
                }
            }
#pragma unroll
            for (int v = 0; v < kV; ++v) y[v] = 0.f;
        }
        __syncthreads();  // buffer b is refilled two steps later
    }
}

int launch_tidas_direct2d(const float* kern, int kz, int taps, bool adjoint, int nz, int nx,
                          const float* in, float* out, int nf, cudaStream_t st) {
    const int tpad = (taps + kV - 1) / kV * kV;
    const int len = nx + tpad + 2 * kV;
    const int W = ((len + kV - 1) / kV) | 1;
    const int chunks = (nx + kV - 1) / kV;
    if (chunks > kThreads)
        return set_error(TIDAS_ERR_UNSUPPORTED, "tidas 2D direct: rows up to %d columns",
                         kThreads * kV);
    const int nfg = min(kFB, kThreads / chunks);
    constexpr int kWC = 65;
    const bool fixed = W <= kWC;
    const size_t smem = (size_t)2 * (tpad + nfg * kV * (fixed ? kWC : W)) * sizeof(float);
    if (smem > 220 * 1024) return set_error(TIDAS_ERR_UNSUPPORTED, "tidas 2D direct: row too long");
    if (nx % 4 == 0 && ((uintptr_t)out % 16) != 0)
        return set_error(TIDAS_ERR_ARG, "tidas 2D direct: output must be 16-byte aligned");
    auto kernel = fixed ? tidas_direct2d_kernel<kWC> : tidas_direct2d_kernel<0>;
    TIDAS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // forward: taps reversed, off = taps-1-c; adjoint: taps as stored, off = c
    const int center = taps / 2;
    const int off = adjoint ? center : taps - 1 - center;
    const int ngroups = (nf + nfg - 1) / nfg;
    int runs = 1;
    while (runs < ngroups && (long long)nz * runs < 4LL * 152 * 4) runs *= 2;
    const int per = (ngroups + runs - 1) / runs;
    dim3 grid(nz, (ngroups + per - 1) / per);
    kernel<<<grid, kThreads, smem, st>>>(kern, kz, taps, off, adjoint, nz, nx, in, out, nf, nfg,
                                         per);
    return check_launch("tidas_direct2d_kernel");
}

}  // namespace tidas
