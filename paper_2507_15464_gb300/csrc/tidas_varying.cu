// Spatially varying tiDAS: Eq. (2.13) with a kernel per pixel.  Kernel
// (j, s) is the single-scatterer image (Eq. (2.6)-(2.7)) of pixel (row j,
// column s): kz rows x taps columns centred on the pixel (kz = 1: the
// row-wise lateral form).  Eq. (2.1) and (2.2) are linear in the
// reflectivity, so the image of a map is the superposition of its pixels'
// images, each scaled by its reflectivity:
//   forward  y[f][i][x] = sum_{u,t} K[j][s][u][t] r[f][j][s],
//                         j = i - u + kz/2, s = x - t + taps/2
//   adjoint  r[f][j][s] = sum_{u,t} K[j][s][u][t] y[f][j + u - kz/2][s + t - taps/2]
// Kernels are the INPUT pixel's (the scatterer's), stored [nz][nx][kz][ld].
//
// The tcgen05 form of the forward map (BF16 operands, FP32 sums) is in
// tidas_gemm.cu; this file holds the FP32 CUDA-core form and the entry
// points.  One block per (128-column tile, row, frame chunk); per band
// slice u the block stages the kernels its tile needs (odd row
// stride, so a warp's lanes, which read kernels of consecutive pixels, hit
// distinct banks) and the matching input line of 8 frames, then each thread
// accumulates one output column for 8 frames in registers.
#include "common.cuh"

namespace tidas {
namespace {

constexpr int kVTX = 128;       // columns per block (one per thread)
constexpr int kVF = 8;          // frames per register group
constexpr int kVGroups = 8;     // register groups per block (64 frames)
constexpr int kVMaxTaps = 64;
constexpr int kVMaxKz = 64;

__host__ __device__ constexpr int varying_ldk(int taps) { return (taps & 1) ? taps : taps + 1; }

// ADJ = false: forward (kernels of input columns s = x - t + cx, indexed by
// sl = tid - t + taps - 1 from base x0 - (taps - 1 - cx)).
// ADJ = true: adjoint (the thread's own pixel's kernel, window over output
// columns x = s + t - cx, indexed by tid + t from base s0 - cx).
template <bool ADJ>
__global__ void __launch_bounds__(kVTX) tidas_varying_direct_kernel(
    const float* __restrict__ kern, int ld, int kz, int taps, int nz, int nx,
    const float* __restrict__ in, float* __restrict__ out, int nf) {
    extern __shared__ float vsm[];
    const int ldk = varying_ldk(taps);
    const int nk = ADJ ? kVTX : kVTX + taps - 1;  // kernels staged per slice
    const int nl = kVTX + taps - 1;               // line samples staged per frame
    const int nlp = nl | 1;
    float* Ks = vsm;                               // [nk][ldk]
    float* Ls = vsm + (size_t)nk * ldk;            // [kVF][nlp]
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kVTX;              // first column of the tile
    const int row = blockIdx.y;                    // output row (forward) / input row (adjoint)
    const int cz = kz / 2, cx = taps / 2;
    // first column of the staged kernels and of the staged line
    const int kb = ADJ ? x0 : x0 - (taps - 1 - cx);
    const int lb = ADJ ? x0 - cx : x0 - (taps - 1 - cx);
    const int f_first = blockIdx.z * kVF * kVGroups;
    const int f_end = min(nf, f_first + kVF * kVGroups);
    const bool once = (kz == 1);  // one slice: stage the kernels once for all frames

    auto stage_kernels = [&](int krow, int u) {
        for (int idx = tid; idx < nk * taps; idx += kVTX) {
            const int sl = idx / taps, t = idx - sl * taps;
            const int s = kb + sl;
            Ks[sl * ldk + t] = (s >= 0 && s < nx)
                                   ? __ldg(kern + (((size_t)krow * nx + s) * kz + u) * ld + t)
                                   : 0.f;
        }
    };
    if (once) {
        stage_kernels(row, 0);
    }
    for (int fg = f_first; fg < f_end; fg += kVF) {
        float acc[kVF];
#pragma unroll
        for (int f = 0; f < kVF; ++f) acc[f] = 0.f;
        for (int u = 0; u < kz; ++u) {
            // forward: input row j feeding output row `row`; adjoint: output
            // row i read by input row `row`
            const int lrow = ADJ ? row + u - cz : row - u + cz;
            if (lrow < 0 || lrow >= nz) continue;  // uniform across the block
            __syncthreads();
            if (!once) stage_kernels(ADJ ? row : lrow, u);
            for (int idx = tid; idx < kVF * nl; idx += kVTX) {
                const int f = idx / nl, l = idx - f * nl;
                const int x = lb + l;
                const int ff = fg + f;
                Ls[f * nlp + l] = (ff < f_end && x >= 0 && x < nx)
                                      ? __ldg(in + ((size_t)ff * nz + lrow) * nx + x)
                                      : 0.f;
            }
            __syncthreads();
            for (int t = 0; t < taps; ++t) {
                const int kl = ADJ ? tid : tid - t + taps - 1;
                const int ll = ADJ ? tid + t : kl;
                const float kv = Ks[kl * ldk + t];
#pragma unroll
                for (int f = 0; f < kVF; ++f) acc[f] = fmaf(kv, Ls[f * nlp + ll], acc[f]);
            }
        }
        const int x = x0 + tid;
        if (x < nx) {
#pragma unroll
            for (int f = 0; f < kVF; ++f)
                if (fg + f < f_end) out[((size_t)(fg + f) * nz + row) * nx + x] = acc[f];
        }
    }
}

size_t varying_smem(int taps, bool adj) {
    const int nk = adj ? kVTX : kVTX + taps - 1;
    const int nl = kVTX + taps - 1;
    return sizeof(float) * ((size_t)nk * varying_ldk(taps) + (size_t)kVF * (nl | 1));
}

int launch_varying_direct(bool adj, const float* kern, int ld, int kz, int taps, int nz, int nx,
                          const float* in, float* out, int nf, cudaStream_t st) {
    const size_t smem = varying_smem(taps, adj);
    dim3 grid((nx + kVTX - 1) / kVTX, nz, (nf + kVF * kVGroups - 1) / (kVF * kVGroups));
    if (adj) {
        TIDAS_CUDA(cudaFuncSetAttribute(tidas_varying_direct_kernel<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tidas_varying_direct_kernel<true>
            <<<grid, kVTX, smem, st>>>(kern, ld, kz, taps, nz, nx, in, out, nf);
    } else {
        TIDAS_CUDA(cudaFuncSetAttribute(tidas_varying_direct_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tidas_varying_direct_kernel<false>
            <<<grid, kVTX, smem, st>>>(kern, ld, kz, taps, nz, nx, in, out, nf);
    }
    return check_launch("tidas_varying_direct_kernel");
}

int varying_args(const char* who, const float* kern, int ld, int kz, int taps, int nz, int nx,
                 const void* in, const void* out, int nf, int variant, bool gemm_ok) {
    TIDAS_REQUIRE(kern && in && out, "%s: null pointer", who);
    TIDAS_REQUIRE(taps >= 1 && taps <= kVMaxTaps && kz >= 1 && kz <= kVMaxKz && ld >= taps,
                  "%s: need 1 <= taps <= %d, 1 <= kz <= %d, ld >= taps (taps=%d kz=%d ld=%d)", who,
                  kVMaxTaps, kVMaxKz, taps, kz, ld);
    TIDAS_REQUIRE(nz >= 1 && nx >= 1 && nf >= 1 && nz <= 65535,
                  "%s: need nz, nx, n_frames >= 1 and nz <= 65535", who);
    if (variant == TIDAS_VARIANT_GEMM_BF16 && gemm_ok) {
        if (nx % 8 != 0)
            return set_error(TIDAS_ERR_UNSUPPORTED, "%s: the GEMM variant needs nx %% 8 == 0", who);
        TIDAS_REQUIRE(((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0 &&
                          ((uintptr_t)kern % 16) == 0,
                      "%s: the GEMM variant needs 16-byte aligned arrays", who);
        return 0;
    }
    if (variant != TIDAS_VARIANT_DIRECT)
        return set_error(TIDAS_ERR_UNSUPPORTED, "%s: variant %d not available", who, variant);
    return 0;
}

}  // namespace

// tcgen05 form of the forward map (tidas_gemm.cu); kern FP32 or (k16) BF16
int launch_tidas_varying_gemm(const void* kern, bool k16, int ld, int kz, int taps, int nz, int nx,
                              const void* in, float* out, int nf, cudaStream_t st);
}  // namespace tidas

using namespace tidas;

extern "C" int tidas_forward_varying(const float* kernels, int32_t ld, int32_t taps, int32_t nz,
                                     int32_t nx, const float* refl, float* img, int32_t n_frames,
                                     void* stream) {
    if (int rc = varying_args("tidas_forward_varying", kernels, ld, 1, taps, nz, nx, refl, img,
                              n_frames, TIDAS_VARIANT_DIRECT, false))
        return rc;
    return launch_varying_direct(false, kernels, ld, 1, taps, nz, nx, refl, img, n_frames,
                                 (cudaStream_t)stream);
}

extern "C" int tidas_forward_varying_2d(const float* kernels, int32_t ld, int32_t kz, int32_t taps,
                                        int32_t nz, int32_t nx, const void* refl, float* img,
                                        int32_t n_frames, int32_t variant, void* stream) {
    if (int rc = varying_args("tidas_forward_varying_2d", kernels, ld, kz, taps, nz, nx, refl,
                              img, n_frames, variant, true))
        return rc;
    if (variant == TIDAS_VARIANT_GEMM_BF16)
        return launch_tidas_varying_gemm(kernels, false, ld, kz, taps, nz, nx, refl, img, n_frames,
                                         (cudaStream_t)stream);
    return launch_varying_direct(false, kernels, ld, kz, taps, nz, nx, (const float*)refl, img,
                                 n_frames, (cudaStream_t)stream);
}

extern "C" int tidas_forward_varying_2d_bf16k(const void* kernels16, int32_t ld, int32_t kz,
                                              int32_t taps, int32_t nz, int32_t nx,
                                              const void* refl, float* img, int32_t n_frames,
                                              void* stream) {
    if (int rc = varying_args("tidas_forward_varying_2d_bf16k", (const float*)kernels16, ld, kz, taps,
                              nz, nx, refl, img, n_frames, TIDAS_VARIANT_GEMM_BF16, true))
        return rc;
    return launch_tidas_varying_gemm(kernels16, true, ld, kz, taps, nz, nx, refl, img, n_frames,
                                     (cudaStream_t)stream);
}

extern "C" int tidas_adjoint_varying_2d(const float* kernels, int32_t ld, int32_t kz, int32_t taps,
                                        int32_t nz, int32_t nx, const void* img, float* refl,
                                        int32_t n_frames, int32_t variant, void* stream) {
    if (int rc = varying_args("tidas_adjoint_varying_2d", kernels, ld, kz, taps, nz, nx, img,
                              refl, n_frames, variant, false))
        return rc;
    return launch_varying_direct(true, kernels, ld, kz, taps, nz, nx, (const float*)img, refl,
                                 n_frames, (cudaStream_t)stream);
}
