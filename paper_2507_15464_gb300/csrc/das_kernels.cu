// Delay-and-Sum family on CUDA cores (sm_103a): forward DAS (Eq. (2.2)), its
// transpose, channel-data synthesis (Eq. (2.1)) and its transpose, and the
// exact single-scatterer PSF rows that define the tiDAS kernels.
#include <climits>

#include "common.cuh"

namespace tidas {

// ---------------------------------------------------------------- DAS
// One thread per pixel; a warp covers 32 neighbouring columns of one row so
// that the 32 gathers of one tap fall inside ~32 consecutive samples.  The
// per-(pixel, element) receive correction and apodization are computed once
// and reused for every angle; the per-(pixel, element, angle) delay and
// interpolation weights are reused for the FB frames a thread accumulates.
// Serves FP32 batches of seven or more frames; FP16 batches take
// das_forward_fi_kernel below (or the tensor cores), smaller batches
// das_coeff_kernel.
template <typename RF, int INTERP, int FB, bool CHECK>
__global__ void __launch_bounds__(256, 2)
    das_forward_kernel(DasDev d, const RF* __restrict__ rf, float* __restrict__ img, int nf) {
    // per-thread transmit delay split of every angle
    __shared__ int s_bi[kMaxAngles][256];
    __shared__ float s_bf[kMaxAngles][256];
    const int lane = threadIdx.x;
    const int tid = threadIdx.y * 32 + lane;
    const int ix = blockIdx.x * 32 + lane;
    // deepest rows first (widest apertures), so the last blocks are the cheap ones
    const int iz = (gridDim.y - 1 - blockIdx.y) * blockDim.y + threadIdx.y;
    if (iz >= d.nz) return;  // uniform per warp; no block-wide barrier follows
    const int f0 = blockIdx.z * FB;
    const int A = d.n_angles, NE = d.n_elem, S = d.n_samples, NX = d.nx;
    const bool xin = ix < NX;
    const int ixc = xin ? ix : NX - 1;
    const float zs = __ldg(d.zs + iz);

    for (int a = 0; a < A; ++a) {
        s_bi[a][tid] = __ldg(d.bxi + a * NX + ixc) + __ldg(d.bzi + a * d.nz + iz);
        s_bf[a][tid] = __ldg(d.bxf + a * NX + ixc) + __ldg(d.bzf + a * d.nz + iz);
    }
    __syncwarp();

    // element range of the warp's aperture union (one element of margin)
    int n_lo = 0, n_hi = NE - 1;
    if (d.fnum > 0.f) {
        const int ix_first = blockIdx.x * 32;
        const int ix_last = min(ix_first + 31, NX - 1);
        const float h = zs / (2.f * d.fnum);
        float lo = (__ldg(d.xs + ix_first) - h - d.elem0_s) / d.pitch_s;
        float hi = (__ldg(d.xs + ix_last) + h - d.elem0_s) / d.pitch_s;
        n_lo = max(0, (int)floorf(lo) - 1);
        n_hi = min(NE - 1, (int)ceilf(hi) + 1);
    }

    float acc[FB];
#pragma unroll
    for (int f = 0; f < FB; ++f) acc[f] = 0.f;
    const size_t fstride = (size_t)A * NE * S;

    for (int n = n_lo; n <= n_hi; ++n) {
        const float dxs = __ldg(d.dxs + (size_t)n * NX + ixc);
        const float w = xin ? apod_weight(dxs, zs, d.fnum) : 0.f;
        if (__ballot_sync(0xffffffffu, w != 0.f) == 0u) continue;
        const float exc = rx_excess(dxs, zs);
        // apodized Keys weights as polynomials in phi with w folded into the
        // coefficients (Horner form): w w0 = phi (phi (ca phi + w) + ca),
        // w w1 = phi^2 (cc phi + cd) + w, w w2 = phi (phi (cf - cc phi) + ch),
        // w w3 = phi^2 (ch phi - ch); (w0, w2) and the inner terms of (w1, w3)
        // are evaluated as packed pairs
        const float ca = -0.5f * w, cc = 1.5f * w, cd = -2.5f * w, cf = 2.f * w, ch = 0.5f * w;
        const uint64_t k02a = f2(ca, -cc), k02b = f2(w, cf), k02c = f2(ca, ch);
        const uint64_t k13a = f2(cc, ch), k13b = f2(cd, -ch);
        // element n's record of angle 0 in frame f0; angle a adds a NE S
        const RF* rown = rf + ((size_t)f0 * A * NE + n) * S;
        const size_t astride = (size_t)NE * S;
#pragma unroll 2
        for (int a = 0; a < A; ++a) {
            const float uf = s_bf[a][tid] + exc;
            const float fl = floorf(uf);
            const float phi = uf - fl;
            const int i = s_bi[a][tid] + (int)fl;
            const RF* row = rown + a * astride;
            const int nfb = FB > 1 ? min(FB, nf - f0) : 1;
            if (!CHECK) {
                // every tap inside the record: one pointer, stepped frame by frame
                if (INTERP == TIDAS_INTERP_CUBIC) {
                    const float p2 = phi * phi;
                    const uint64_t P = f2(phi, phi);
                    const uint64_t t02 = f2_mul(f2_fma(f2_fma(k02a, P, k02b), P, k02c), P);
                    const uint64_t t13 = f2_fma(k13a, P, k13b);
                    const float v0 = f2_lo(t02), v2 = f2_hi(t02);
                    const float v1 = fmaf(f2_lo(t13), p2, w), v3 = f2_hi(t13) * p2;
                    const RF* p = row + (i - 1);
                    if (nfb == FB) {
#pragma unroll
                        for (int f = 0; f < FB; ++f) {
                            float v = fmaf(v0, load_rf(p), acc[f]);
                            v = fmaf(v1, load_rf(p + 1), v);
                            v = fmaf(v2, load_rf(p + 2), v);
                            acc[f] = fmaf(v3, load_rf(p + 3), v);
                            p += fstride;
                        }
                    } else {
#pragma unroll
                        for (int f = 0; f < FB; ++f) {
                            if (f >= nfb) break;
                            float v = fmaf(v0, load_rf(p), acc[f]);
                            v = fmaf(v1, load_rf(p + 1), v);
                            v = fmaf(v2, load_rf(p + 2), v);
                            acc[f] = fmaf(v3, load_rf(p + 3), v);
                            p += fstride;
                        }
                    }
                } else {
                    // apodized linear weights w (1 - phi), w phi
                    const float v0 = fmaf(-w, phi, w), v1 = w * phi;
                    const RF* p = row + i;
#pragma unroll
                    for (int f = 0; f < FB; ++f) {
                        if (f >= nfb) break;
                        acc[f] = fmaf(v1, load_rf(p + 1), fmaf(v0, load_rf(p), acc[f]));
                        p += fstride;
                    }
                }
                continue;
            }
            if (INTERP == TIDAS_INTERP_CUBIC) {
                float w0, w1, w2, w3;
                keys_weights(phi, w0, w1, w2, w3);
                int m0 = i - 1, m1 = i, m2 = i + 1, m3 = i + 2;
                if (CHECK) {
                    if ((unsigned)m0 >= (unsigned)S) { w0 = 0.f; m0 = 0; }
                    if ((unsigned)m1 >= (unsigned)S) { w1 = 0.f; m1 = 0; }
                    if ((unsigned)m2 >= (unsigned)S) { w2 = 0.f; m2 = 0; }
                    if ((unsigned)m3 >= (unsigned)S) { w3 = 0.f; m3 = 0; }
                }
#pragma unroll
                for (int f = 0; f < FB; ++f) {
                    if (FB > 1 && f0 + f >= nf) break;
                    const RF* r = row + f * fstride;
                    float v = w0 * load_rf(r + m0);
                    v = fmaf(w1, load_rf(r + m1), v);
                    v = fmaf(w2, load_rf(r + m2), v);
                    v = fmaf(w3, load_rf(r + m3), v);
                    acc[f] = fmaf(w, v, acc[f]);
                }
            } else {
                float w0 = 1.f - phi, w1 = phi;
                int m0 = i, m1 = i + 1;
                if (CHECK) {
                    if ((unsigned)m0 >= (unsigned)S) { w0 = 0.f; m0 = 0; }
                    if ((unsigned)m1 >= (unsigned)S) { w1 = 0.f; m1 = 0; }
                }
#pragma unroll
                for (int f = 0; f < FB; ++f) {
                    if (FB > 1 && f0 + f >= nf) break;
                    const RF* r = row + f * fstride;
                    float v = w0 * load_rf(r + m0);
                    v = fmaf(w1, load_rf(r + m1), v);
                    acc[f] = fmaf(w, v, acc[f]);
                }
            }
        }
    }
    if (xin) {
#pragma unroll
        for (int f = 0; f < FB; ++f)
            if (f0 + f < nf) img[((size_t)(f0 + f) * d.nz + iz) * NX + ix] = acc[f];
    }
}

template <typename RF, int INTERP, bool CHECK>
static void das_forward_dispatch_fb(const DasDev& d, const void* rf, float* img, int nf,
                                    cudaStream_t st) {
    dim3 block(32, 8);
    int fb = nf >= 16 ? 16 : (nf >= 8 ? 8 : (nf >= 4 ? 4 : 2));
    dim3 grid((d.nx + 31) / 32, (d.nz + 7) / 8, (nf + fb - 1) / fb);
    const RF* r = (const RF*)rf;
    switch (fb) {
        case 16: das_forward_kernel<RF, INTERP, 16, CHECK><<<grid, block, 0, st>>>(d, r, img, nf); break;
        case 8: das_forward_kernel<RF, INTERP, 8, CHECK><<<grid, block, 0, st>>>(d, r, img, nf); break;
        case 4: das_forward_kernel<RF, INTERP, 4, CHECK><<<grid, block, 0, st>>>(d, r, img, nf); break;
        default: das_forward_kernel<RF, INTERP, 2, CHECK><<<grid, block, 0, st>>>(d, r, img, nf); break;
    }
}

template <typename RF>
static void das_forward_dispatch(const Plan& P, const void* rf, float* img, int nf,
                                 cudaStream_t st) {
    const DasDev& d = P.dev;
    bool check = !P.taps_in_range;
    if (d.interp == TIDAS_INTERP_CUBIC) {
        if (check) das_forward_dispatch_fb<RF, 1, true>(d, rf, img, nf, st);
        else das_forward_dispatch_fb<RF, 1, false>(d, rf, img, nf, st);
    } else {
        if (check) das_forward_dispatch_fb<RF, 0, true>(d, rf, img, nf, st);
        else das_forward_dispatch_fb<RF, 0, false>(d, rf, img, nf, st);
    }
}

// ------------------------------------------------ DAS, frames innermost
// FP16 batches of 5 or more frames that do not take the tensor cores
// (5 .. 15 frames, or the tensor cores switched off).  The batch is first
// restaged as [frame tile][angle, element][sample][NFP frames] (frames past
// nf zero), so that one tap of one pixel reads the NFP frames of its frame
// tile as 16-byte vectors instead of NFP scalar gathers.  The delay, the
// Keys weights and the apodization (folded into the tap weights) are
// computed once per (pixel, angle, element) and serve all NFP frames.

// [nf][R][S] -> [FT][R][S][NFP]: one block per (frame tile, row, 64 samples)
template <typename RF>
__global__ void __launch_bounds__(256) frames_inner_pack_kernel(const RF* __restrict__ rf,
                                                                RF* __restrict__ out, int nf,
                                                                int R, int S, int NFP) {
    __shared__ RF t[16][65];  // [frame][sample]
    const int nsb = (S + 63) / 64;
    const int sb = blockIdx.x % nsb;
    const int r = (blockIdx.x / nsb) % R;
    const int ft = blockIdx.x / (nsb * R);
    const int s0 = sb * 64;
    for (int i = threadIdx.x; i < NFP * 64; i += blockDim.x) {
        const int f = i >> 6, k = i & 63;
        const int ff = ft * NFP + f, sidx = s0 + k;
        t[f][k] = (ff < nf && sidx < S) ? rf[((size_t)ff * R + r) * S + sidx] : RF(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * NFP; i += blockDim.x) {
        const int k = i / NFP, f = i - k * NFP;
        const int sidx = s0 + k;
        if (sidx < S) out[(((size_t)ft * R + r) * S + sidx) * NFP + f] = t[f][k];
    }
}

// the NFP frames of one (row, sample) of the restaged FP16 batch, as floats
template <int NFP>
__device__ __forceinline__ void load_frames(const __half* __restrict__ p, float (&v)[NFP]) {
    static_assert(NFP % 8 == 0, "frame vectors of 16 bytes");
    uint32_t w[NFP / 2];
#pragma unroll
    for (int j = 0; j < NFP / 8; ++j) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(p) + j);
        w[4 * j] = q.x;
        w[4 * j + 1] = q.y;
        w[4 * j + 2] = q.z;
        w[4 * j + 3] = q.w;
    }
#pragma unroll
    for (int j = 0; j < NFP / 2; ++j) {
        const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&w[j]));
        v[2 * j] = f2.x;
        v[2 * j + 1] = f2.y;
    }
}

template <typename RF, int INTERP, int NFP, bool CHECK>
__global__ void __launch_bounds__(256, 2) das_forward_fi_kernel(DasDev d, const RF* __restrict__ rfi,
                                                                float* __restrict__ img, int nf) {
    __shared__ int s_bi[kMaxAngles][256];
    __shared__ float s_bf[kMaxAngles][256];
    const int lane = threadIdx.x;
    const int tid = threadIdx.y * 32 + lane;
    const int ix = blockIdx.x * 32 + lane;
    const int iz = (gridDim.y - 1 - blockIdx.y) * blockDim.y + threadIdx.y;
    if (iz >= d.nz) return;  // uniform per warp; no block-wide barrier follows
    const int ft = blockIdx.z;
    const int A = d.n_angles, NE = d.n_elem, S = d.n_samples, NX = d.nx;
    const bool xin = ix < NX;
    const int ixc = xin ? ix : NX - 1;
    const float zs = __ldg(d.zs + iz);
    for (int a = 0; a < A; ++a) {
        s_bi[a][tid] = __ldg(d.bxi + a * NX + ixc) + __ldg(d.bzi + a * d.nz + iz);
        s_bf[a][tid] = __ldg(d.bxf + a * NX + ixc) + __ldg(d.bzf + a * d.nz + iz);
    }
    __syncwarp();
    int n_lo = 0, n_hi = NE - 1;
    if (d.fnum > 0.f) {
        const int ix_first = blockIdx.x * 32;
        const int ix_last = min(ix_first + 31, NX - 1);
        const float h = zs / (2.f * d.fnum);
        float lo = (__ldg(d.xs + ix_first) - h - d.elem0_s) / d.pitch_s;
        float hi = (__ldg(d.xs + ix_last) + h - d.elem0_s) / d.pitch_s;
        n_lo = max(0, (int)floorf(lo) - 1);
        n_hi = min(NE - 1, (int)ceilf(hi) + 1);
    }
    float acc[NFP];
#pragma unroll
    for (int f = 0; f < NFP; ++f) acc[f] = 0.f;
    const RF* tile = rfi + (size_t)ft * A * NE * S * NFP;
    for (int n = n_lo; n <= n_hi; ++n) {
        const float dxs = __ldg(d.dxs + (size_t)n * NX + ixc);
        const float w = xin ? apod_weight(dxs, zs, d.fnum) : 0.f;
        if (__ballot_sync(0xffffffffu, w != 0.f) == 0u) continue;
        const float exc = rx_excess(dxs, zs);
        // apodized Keys weights in Horner form with w folded into the
        // coefficients, (w0, w2) and the inner terms of (w1, w3) as packed
        // pairs (as in das_forward_kernel)
        const float ca = -0.5f * w, cc = 1.5f * w, cd = -2.5f * w, cf = 2.f * w, ch = 0.5f * w;
        const uint64_t k02a = f2(ca, -cc), k02b = f2(w, cf), k02c = f2(ca, ch);
        const uint64_t k13a = f2(cc, ch), k13b = f2(cd, -ch);
        const RF* rown = tile + (size_t)n * S * NFP;  // element n's record of angle 0
        const size_t astride = (size_t)NE * S * NFP;
#pragma unroll 2
        for (int a = 0; a < A; ++a) {
            const float uf = s_bf[a][tid] + exc;
            const float fl = floorf(uf);
            const float phi = uf - fl;
            const int i = s_bi[a][tid] + (int)fl;
            const RF* row = rown + a * astride;
            constexpr int T = INTERP == TIDAS_INTERP_CUBIC ? 4 : 2;
            float wt[T];
            int m[T];
            if (INTERP == TIDAS_INTERP_CUBIC) {
                const float p2 = phi * phi;
                const uint64_t P = f2(phi, phi);
                const uint64_t t02 = f2_mul(f2_fma(f2_fma(k02a, P, k02b), P, k02c), P);
                const uint64_t t13 = f2_fma(k13a, P, k13b);
                wt[0] = f2_lo(t02);
                wt[1] = fmaf(f2_lo(t13), p2, w);
                wt[T > 2 ? 2 : 0] = f2_hi(t02);
                wt[T > 3 ? 3 : 0] = f2_hi(t13) * p2;
                m[0] = i - 1;
            } else {
                wt[0] = fmaf(-w, phi, w);
                wt[1] = w * phi;
                m[0] = i;
            }
#pragma unroll
            for (int k = 1; k < T; ++k) m[k] = m[0] + k;
            if (CHECK) {
#pragma unroll
                for (int k = 0; k < T; ++k)
                    if ((unsigned)m[k] >= (unsigned)S) {
                        wt[k] = 0.f;
                        m[k] = 0;
                    }
            }
#pragma unroll
            for (int k = 0; k < T; ++k) {
                float v[NFP];
                load_frames<NFP>(row + (size_t)m[k] * NFP, v);
#pragma unroll
                for (int f = 0; f < NFP; ++f) acc[f] = fmaf(wt[k], v[f], acc[f]);
            }
        }
    }
    if (xin) {
#pragma unroll
        for (int f = 0; f < NFP; ++f) {
            const int ff = ft * NFP + f;
            if (ff < nf) img[((size_t)ff * d.nz + iz) * NX + ix] = acc[f];
        }
    }
}

template <typename RF, int INTERP, bool CHECK>
static void das_forward_fi_dispatch(const DasDev& d, const RF* rfi, float* img, int nf, int NFP,
                                    cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((d.nx + 31) / 32, (d.nz + 7) / 8, (nf + NFP - 1) / NFP);
    switch (NFP) {
        case 8: das_forward_fi_kernel<RF, INTERP, 8, CHECK><<<grid, block, 0, st>>>(d, rfi, img, nf); break;
        default: das_forward_fi_kernel<RF, INTERP, 16, CHECK><<<grid, block, 0, st>>>(d, rfi, img, nf); break;
    }
}

template <typename RF>
static int das_forward_frames_inner(const Plan& P, const void* rf, float* img, int nf,
                                    cudaStream_t st) {
    const DasDev& d = P.dev;
    const int NFP = nf <= 8 ? 8 : 16;  // batches of 5 .. 15 frames reach here
    const int R = d.n_angles * d.n_elem, S = d.n_samples;
    const int FT = (nf + NFP - 1) / NFP;
    const size_t need = (size_t)FT * R * S * NFP * sizeof(RF);
    void* ws = nullptr;
    bool fresh = false;  // every sample of this layout is written below
    if (int rc = plan_staging(P, need, &ws, 1, &fresh)) return rc;
    const size_t blocks = (size_t)FT * R * ((S + 63) / 64);
    if (blocks > (size_t)INT_MAX) return set_error(TIDAS_ERR_UNSUPPORTED, "das_forward: batch too large");
    frames_inner_pack_kernel<RF><<<(unsigned)blocks, 256, 0, st>>>((const RF*)rf, (RF*)ws, nf, R,
                                                                   S, NFP);
    if (int rc = check_launch("frames_inner_pack_kernel")) return rc;
    const bool check = !P.taps_in_range;
    if (d.interp == TIDAS_INTERP_CUBIC) {
        if (check) das_forward_fi_dispatch<RF, 1, true>(d, (const RF*)ws, img, nf, NFP, st);
        else das_forward_fi_dispatch<RF, 1, false>(d, (const RF*)ws, img, nf, NFP, st);
    } else {
        if (check) das_forward_fi_dispatch<RF, 0, true>(d, (const RF*)ws, img, nf, NFP, st);
        else das_forward_fi_dispatch<RF, 0, false>(d, (const RF*)ws, img, nf, NFP, st);
    }
    return check_launch("das_forward_fi_kernel");
}

int launch_das_forward(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st) {
    // batches of FP16 channel data go to the tensor cores (frames are the
    // MMA's N dimension); smaller FP16 batches are restaged with the frames
    // innermost (16-byte frame vectors per tap: 1.4x faster at 8 frames).
    // FP32 batches read the batch in place: for FP32 the frame vectors
    // measured no faster at 8 frames and slower at 64, where the kernel's 16
    // FP32 accumulators and vectors cost its occupancy.  Single frames and
    // small batches read per-interval interpolation coefficients
    // (das_coeff.cu).
    if (P.dev.rf_dtype == TIDAS_RF_F16 && P.tc_ok && P.tc_mode == 1 && nf >= 16 &&
        ((uintptr_t)rf % 16) == 0)
        return launch_das_tc(P, rf, img, nf, st);
    // (measured per batch size: the coefficient path up to 6 FP32 / 4 FP16
    // frames, the sample gathers above)
    if (nf <= (P.dev.rf_dtype == TIDAS_RF_F16 ? 4 : 6)) return launch_das_coeff(P, rf, img, nf, st);
    if (P.dev.rf_dtype == TIDAS_RF_F16)
        return das_forward_frames_inner<__half>(P, rf, img, nf, st);
    das_forward_dispatch<float>(P, rf, img, nf, st);
    return check_launch("das_forward_kernel");
}

// ------------------------------------------------------------ DAS^T
// One block per (element, group of ag <= kAG angles, frame): the group's channel
// rows are accumulated in shared memory.  Threads walk the rows of each
// column (their delays are ~3 samples apart, so taps of neighbouring lanes
// rarely collide); the apodization and receive delay of a (pixel, element)
// are computed once for the group's angles, and each angle adds
// w * (interpolation weight) * img into the samples the forward pass read.
constexpr int kAG = 4;
template <int INTERP>
__global__ void __launch_bounds__(256) das_adjoint_kernel(DasDev d, const float* __restrict__ img,
                                                          float* __restrict__ rf, int ag) {
    extern __shared__ float acc[];  // [ag][S]
    const int n = blockIdx.x, a0 = blockIdx.y * ag, f = blockIdx.z;
    const int S = d.n_samples, NX = d.nx, NZ = d.nz;
    const int na = min(ag, d.n_angles - a0);
    for (int k = threadIdx.x; k < na * S; k += blockDim.x) acc[k] = 0.f;
    __syncthreads();
    const float* im = img + (size_t)f * NZ * NX;
    for (int ix = 0; ix < NX; ++ix) {
        const float dxs = __ldg(d.dxs + (size_t)n * NX + ix);
        for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
            const float zs = __ldg(d.zs + iz);
            const float w = apod_weight(dxs, zs, d.fnum);
            if (w == 0.f) continue;
            const float exc = rx_excess(dxs, zs);
            const float v = w * __ldg(im + (size_t)iz * NX + ix);
            for (int q = 0; q < na; ++q) {
                int i;
                float phi;
                pixel_delay(d, a0 + q, ix, iz, exc, i, phi);
                float* ac = acc + q * S;
                if (INTERP == TIDAS_INTERP_CUBIC) {
                    float w0, w1, w2, w3;
                    keys_weights(phi, w0, w1, w2, w3);
                    if ((unsigned)(i - 1) < (unsigned)S) atomicAdd(ac + i - 1, w0 * v);
                    if ((unsigned)(i) < (unsigned)S) atomicAdd(ac + i, w1 * v);
                    if ((unsigned)(i + 1) < (unsigned)S) atomicAdd(ac + i + 1, w2 * v);
                    if ((unsigned)(i + 2) < (unsigned)S) atomicAdd(ac + i + 2, w3 * v);
                } else {
                    if ((unsigned)(i) < (unsigned)S) atomicAdd(ac + i, (1.f - phi) * v);
                    if ((unsigned)(i + 1) < (unsigned)S) atomicAdd(ac + i + 1, phi * v);
                }
            }
        }
    }
    __syncthreads();
    for (int q = 0; q < na; ++q) {
        float* out = rf + ((size_t)(f * d.n_angles + a0 + q) * d.n_elem + n) * S;
        for (int k = threadIdx.x; k < S; k += blockDim.x) out[k] = acc[q * S + k];
    }
}

int launch_das_adjoint(const Plan& P, const float* img, float* rf, int nf, cudaStream_t st) {
    const DasDev& d = P.dev;
    // as many angles per block as kAG rows of accumulators allow (at least one)
    const size_t row = (size_t)d.n_samples * sizeof(float);
    int ag = (int)min((size_t)kAG, (size_t)(200 * 1024) / row);
    if (ag < 1) ag = 1;
    const size_t smem = (size_t)ag * row;
    dim3 grid(d.n_elem, (d.n_angles + ag - 1) / ag, nf);
    if (d.interp == TIDAS_INTERP_CUBIC) {
        TIDAS_CUDA(cudaFuncSetAttribute(das_adjoint_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
        das_adjoint_kernel<1><<<grid, 256, smem, st>>>(d, img, rf, ag);
    } else {
        TIDAS_CUDA(cudaFuncSetAttribute(das_adjoint_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
        das_adjoint_kernel<0><<<grid, 256, smem, st>>>(d, img, rf, ag);
    }
    return check_launch("das_adjoint_kernel");
}

// --------------------------------------------------------------- pulse
// Taps of the pulse delayed by a fractional sample phi: p(j - phi) for the
// integers j with |j - phi| <= thalf, p(t) = exp(-beta t^2) cos(pi wcar t).
// Written as exp(-beta phi^2) * Q_j * G^j * (C_j cos(pi wcar phi) +
// S_j sin(pi wcar phi)) with Q_j = exp(-beta j^2), G = exp(2 beta phi),
// C_j + i S_j = exp(i pi wcar j): one exp pair and one sincos per delay,
// then a few multiplies per tap.  Tables live in shared memory (index j + kJ).
struct PulseSmem {
    float q[2 * kJ + 1], c[2 * kJ + 1], s[2 * kJ + 1];
};

__device__ void load_pulse_tables(const DasDev& d, PulseSmem& t) {
    for (int j = threadIdx.x + threadIdx.y * blockDim.x; j <= 2 * kJ;
         j += blockDim.x * blockDim.y) {
        t.q[j] = __ldg(d.ptab + j);
        t.c[j] = __ldg(d.ptab + (2 * kJ + 1) + j);
        t.s[j] = __ldg(d.ptab + 2 * (2 * kJ + 1) + j);
    }
}

struct PulseAt {
    float e0, g, ginv, cph, sph;
    int jlo, jhi;
};

__device__ __forceinline__ PulseAt pulse_at(const DasDev& d, float phi) {
    PulseAt p;
    p.e0 = expf(-d.beta * phi * phi);
    p.g = expf(2.f * d.beta * phi);
    p.ginv = expf(-2.f * d.beta * phi);
    sincospif(d.wcar * phi, &p.sph, &p.cph);
    p.jlo = (int)ceilf(phi - d.thalf);
    p.jhi = (int)floorf(phi + d.thalf);
    return p;
}

// ------------------------------------------------- synthesis, point list
// One block per (element, angle, frame) channel row; scatterers are spread
// over the threads; samples accumulate in shared memory.  Delays in FP64.
template <typename RF>
__global__ void __launch_bounds__(256) synth_points_kernel(DasDev d, const double* __restrict__ pos,
                                                           const float* __restrict__ amp, int n_scat,
                                                           const double* __restrict__ sncs,
                                                           RF* __restrict__ rf, double c, double t0,
                                                           double fs, double pitch) {
    extern __shared__ float acc[];
    const int n = blockIdx.x, a = blockIdx.y, f = blockIdx.z;
    const int S = d.n_samples;
    for (int k = threadIdx.x; k < S; k += blockDim.x) acc[k] = 0.f;
    __syncthreads();
    const double sa = sncs[2 * a], ca = sncs[2 * a + 1];
    const double xn = __dmul_rn(__dsub_rn((double)n, 0.5 * (double)(d.n_elem - 1)), pitch);
    const double* ps = pos + (size_t)f * n_scat * 2;
    const float* am = amp + (size_t)f * n_scat * 2;
    for (int j = threadIdx.x; j < n_scat; j += blockDim.x) {
        const double x = ps[2 * j], z = ps[2 * j + 1];
        const double ddx = __dsub_rn(x, xn);
        const double tx = __dadd_rn(__dmul_rn(x, sa), __dmul_rn(z, ca));
        const double rx = __dsqrt_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(z, z)));
        const double u = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tx, rx), c), t0), fs);
        const double fl = floor(u);
        const int i0 = (int)fl;
        const float phi = (float)(u - fl);
        const float are = am[2 * j], aim = am[2 * j + 1];
        const int jlo = (int)ceilf(phi - d.thalf), jhi = (int)floorf(phi + d.thalf);
        for (int jj = jlo; jj <= jhi; ++jj) {
            const int m = i0 + jj;
            if ((unsigned)m >= (unsigned)S) continue;
            const float t = (float)jj - phi;
            float sv, cv;
            sincospif(d.wcar * t, &sv, &cv);
            const float env = expf(-d.beta * t * t);
            atomicAdd(acc + m, env * (are * cv - aim * sv));
        }
    }
    __syncthreads();
    RF* out = rf + ((size_t)(f * d.n_angles + a) * d.n_elem + n) * S;
    for (int k = threadIdx.x; k < S; k += blockDim.x) store_rf(out + k, acc[k]);
}

int launch_synthesize(const Plan& P, const double* pos, const float* amp, int n_scat, int nf,
                      void* rf, cudaStream_t st) {
    const DasDev& d = P.dev;
    size_t smem = (size_t)d.n_samples * sizeof(float);
    dim3 grid(d.n_elem, d.n_angles, nf);
    if (d.rf_dtype == TIDAS_RF_F16) {
        TIDAS_CUDA(cudaFuncSetAttribute(synth_points_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
        synth_points_kernel<__half><<<grid, 256, smem, st>>>(d, pos, amp, n_scat, P.d_sncs,
                                                            (__half*)rf, P.p.c, P.p.t0, P.p.fs,
                                                            P.p.pitch);
    } else {
        TIDAS_CUDA(cudaFuncSetAttribute(synth_points_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
        synth_points_kernel<float><<<grid, 256, smem, st>>>(d, pos, amp, n_scat, P.d_sncs,
                                                           (float*)rf, P.p.c, P.p.t0, P.p.fs,
                                                           P.p.pitch);
    }
    return check_launch("synth_points_kernel");
}

// ------------------------------------------------- synthesis on the grid
// Same row-per-block scheme; the "scatterers" are the pixels, with the split
// delays of DAS, so that this operator and its transpose below use
// identical delays and pulse taps.
__global__ void __launch_bounds__(256) synth_grid_kernel(DasDev d, const float* __restrict__ refl,
                                                         float* __restrict__ rf) {
    extern __shared__ float acc[];
    __shared__ PulseSmem tab;
    const int n = blockIdx.x, a = blockIdx.y, f = blockIdx.z;
    const int S = d.n_samples, NX = d.nx, NZ = d.nz;
    for (int k = threadIdx.x; k < S; k += blockDim.x) acc[k] = 0.f;
    load_pulse_tables(d, tab);
    __syncthreads();
    const float* rp = refl + (size_t)f * NZ * NX;
    for (int ix = 0; ix < NX; ++ix) {
        const float dxs = __ldg(d.dxs + (size_t)n * NX + ix);
        for (int iz = threadIdx.x; iz < NZ; iz += blockDim.x) {
            const float v = __ldg(rp + (size_t)iz * NX + ix);
            if (v == 0.f) continue;
            const float zs = __ldg(d.zs + iz);
            int i;
            float phi;
            pixel_delay(d, a, ix, iz, rx_excess(dxs, zs), i, phi);
            const PulseAt p = pulse_at(d, phi);
            const float ve = v * p.e0;
            float gj = 1.f;
            for (int j = 0; j <= p.jhi; ++j) {
                const int m = i + j;
                if ((unsigned)m < (unsigned)S) {
                    float car = fmaf(tab.c[j + kJ], p.cph, tab.s[j + kJ] * p.sph);
                    atomicAdd(acc + m, ve * (tab.q[j + kJ] * gj) * car);
                }
                gj *= p.g;
            }
            gj = p.ginv;
            for (int j = -1; j >= p.jlo; --j) {
                const int m = i + j;
                if ((unsigned)m < (unsigned)S) {
                    float car = fmaf(tab.c[j + kJ], p.cph, tab.s[j + kJ] * p.sph);
                    atomicAdd(acc + m, ve * (tab.q[j + kJ] * gj) * car);
                }
                gj *= p.ginv;
            }
        }
    }
    __syncthreads();
    float* out = rf + ((size_t)(f * d.n_angles + a) * d.n_elem + n) * S;
    for (int k = threadIdx.x; k < S; k += blockDim.x) out[k] = acc[k];
}

// Gather form of the same sum, used for the grid: each thread owns kGS
// consecutive samples of the channel row and adds, column by column, the
// pixels whose pulse reaches them.  The delay grows with depth down a
// column (d/dz of x sin + z cos + |r - x_n| is cos + z / |r - x_n| > 0), so
// those pixels are a contiguous run found by binary search over the
// column's integer delays.  The pulse is the real part of
// env(t) e^{i pi wcar t} (a1), so
//     rf[k] = Re( e^{i pi wcar k} G[k] ),  G[k] = sum_p c_p env(k - u_p),
// with the complex amplitude c_p = v_p e^{-i pi wcar u_p} formed once per
// pixel and row (e^{-i pi wcar i} from the plan's integer-sample carrier
// table, the fraction's phase by sincospi of a small argument).  At the
// thread's samples k0 + q the envelope factors as
//     env(t0 + q) = exp(-beta t0^2) R^q exp(-beta q^2),  R = exp(-2 beta t0),
// t0 = k0 - u_p, and the last factor, the same for every pixel, is applied
// once per sample after the sum.  Only the nonzero pixels of each column
// enter (compact_columns_kernel lists them in increasing depth), and
// consecutive columns are staged together up to nz pixels per pass, so a
// sparse map (an L1-regularised iterate) costs in proportion to its nonzeros.
// No atomics; each sample is summed in a fixed order (columns, then depth).
constexpr int kGS = 16;
__global__ void __launch_bounds__(256) synth_grid_gather_kernel(DasDev d,
                                                                const int* __restrict__ ccnt,
                                                                const int* __restrict__ cz,
                                                                const float* __restrict__ cv,
                                                                float* __restrict__ rf) {
    extern __shared__ float sm[];
    const int NZ = d.nz, NX = d.nx, S = d.n_samples;
    int* ui = reinterpret_cast<int*>(sm);  // [NZ] integer delay of the staged pixels
    float* uf = sm + NZ;                   // [NZ] fraction
    float* cre = uf + NZ;                  // [NZ] complex amplitude v e^{-i pi wcar u}
    float* cim = cre + NZ;
    int* coff = reinterpret_cast<int*>(cim + NZ);  // [NX + 1] group column offsets
    const int n = blockIdx.x, a = blockIdx.y, f = blockIdx.z;
    const int* cnt = ccnt + (size_t)f * NX;
    const int* czf = cz + (size_t)f * NX * NZ;
    const float* cvf = cv + (size_t)f * NX * NZ;
    const int hi_tap = (int)ceilf(d.thalf) + 1;
    float* out = rf + ((size_t)(f * d.n_angles + a) * d.n_elem + n) * S;
    for (int base = 0; base < S; base += kGS * (int)blockDim.x) {
        const int k0 = base + kGS * (int)threadIdx.x;
        float gr[kGS], gi[kGS];  // G[k0 + q] / exp(-beta q^2)
#pragma unroll
        for (int q = 0; q < kGS; ++q) gr[q] = gi[q] = 0.f;
        for (int ix0 = 0; ix0 < NX;) {
            // columns ix0 .. ix1 - 1 hold at most NZ nonzero pixels together
            // (one column holds at most NZ, so a group has at least one)
            int ix1 = ix0, tot = 0;
            while (ix1 < NX) {
                const int c = __ldg(cnt + ix1);
                if (tot + c > NZ) break;
                tot += c;
                ++ix1;
            }
            if (tot > 0) {
                __syncthreads();  // the previous group has been read
                // coff[k]: staged entries before column ix0 + k of the group
                // (exclusive scan of the counts by the first warp)
                const int G = ix1 - ix0;
                if (threadIdx.x < 32) {
                    const int lane = threadIdx.x;
                    int run = 0;
                    for (int k0c = 0; k0c < G; k0c += 32) {
                        const int k = k0c + lane;
                        const int c = k < G ? __ldg(cnt + ix0 + k) : 0;
                        int incl = c;
#pragma unroll
                        for (int sh = 1; sh < 32; sh <<= 1) {
                            const int y = __shfl_up_sync(0xffffffffu, incl, sh);
                            if (lane >= sh) incl += y;
                        }
                        if (k < G) coff[k] = run + incl - c;
                        run += __shfl_sync(0xffffffffu, incl, 31);
                    }
                    if (lane == 0) coff[G] = run;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < tot; e += blockDim.x) {
                    // the group column of entry e: last k with coff[k] <= e
                    int klo = 0, khi = G - 1;
                    while (klo < khi) {
                        const int mid = (klo + khi + 1) >> 1;
                        if (coff[mid] <= e) klo = mid; else khi = mid - 1;
                    }
                    const int ix = ix0 + klo, j = e - coff[klo];
                    const float dxs = __ldg(d.dxs + (size_t)n * NX + ix);
                    {
                        const int iz = __ldg(czf + (size_t)ix * NZ + j);
                        float v = __ldg(cvf + (size_t)ix * NZ + j);
                        int i;
                        float phi;
                        pixel_delay(d, a, ix, iz, rx_excess(dxs, __ldg(d.zs + iz)), i, phi);
                        // a pixel whose support misses the record adds nothing
                        if (i < -hi_tap || i >= S + hi_tap) v = 0.f;
                        float zr = 0.f, zi = 0.f;
                        if (v != 0.f) {
                            const float2 ci = __ldg(d.carr + i);
                            float sp, cp;
                            sincospif(d.wcar * phi, &sp, &cp);
                            zr = v * (ci.x * cp - ci.y * sp);
                            zi = -v * (ci.x * sp + ci.y * cp);
                        }
                        ui[e] = i;
                        uf[e] = phi;
                        cre[e] = zr;
                        cim[e] = zi;
                    }
                }
                __syncthreads();
                if (k0 < S) {
                    int seg = 0;  // first staged entry of column ix
                    for (int ix = ix0; ix < ix1; ++ix) {
                        const int c = __ldg(cnt + ix);
                        if (c == 0) continue;
                        // first pixel with i >= k0 - hi_tap, last with i <= k0 + kGS - 1 + hi_tap
                        int lo = seg, hi = seg + c;
                        const int want_lo = k0 - hi_tap;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (ui[mid] < want_lo) lo = mid + 1; else hi = mid;
                        }
                        // the run ends at the first pixel with i > k0 + kGS - 1 + hi_tap
                        // (a scan: in sparse columns the run is a pixel or two)
                        const int want_hi = k0 + kGS - 1 + hi_tap;
                        for (int p = lo; p < seg + c; ++p) {
                            const int i = ui[p];
                            if (i > want_hi) break;
                            const float zr = cre[p], zi = cim[p];
                            if (zr == 0.f && zi == 0.f) continue;
                            const float phi = uf[p];
                            // this thread's samples k0 + q inside the support: tap j = k0 + q - i
                            const int j0 = k0 - i;
                            const int qlo = (int)ceilf(phi - d.thalf) - j0,
                                      qhi = (int)floorf(phi + d.thalf) - j0;
                            const float t0 = (float)j0 - phi;
                            const float e0 = expf(-d.beta * t0 * t0);
                            const float R = expf(-2.f * d.beta * t0);
                            const float er = e0 * zr, ei = e0 * zi;
                            float pw = 1.f;  // R^q
#pragma unroll
                            for (int q = 0; q < kGS; ++q) {
                                if (q >= qlo && q <= qhi) {
                                    gr[q] = fmaf(pw, er, gr[q]);
                                    gi[q] = fmaf(pw, ei, gi[q]);
                                }
                                pw *= R;
                            }
                        }
                        seg += c;
                    }
                }
            }
            ix0 = ix1;
        }
        if (k0 < S) {
#pragma unroll
            for (int q = 0; q < kGS; ++q)
                if (k0 + q < S) {
                    const float2 ck = __ldg(d.carr + k0 + q);
                    out[k0 + q] = expf(-d.beta * (float)(q * q)) * (gr[q] * ck.x - gi[q] * ck.y);
                }
        }
    }
}

// One warp per (frame, column) of reflT [nf][nx][nz]: the depths and values of
// the column's nonzero pixels in increasing depth, and their count.
__global__ void __launch_bounds__(256) compact_columns_kernel(const float* __restrict__ reflT,
                                                              int nz, int ncols,
                                                              int* __restrict__ cnt,
                                                              int* __restrict__ cz,
                                                              float* __restrict__ cv) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= ncols) return;  // uniform per warp
    const float* col = reflT + (size_t)w * nz;
    int* oz = cz + (size_t)w * nz;
    float* ov = cv + (size_t)w * nz;
    int c = 0;
    for (int z0 = 0; z0 < nz; z0 += 32) {
        const int z = z0 + lane;
        const float v = z < nz ? col[z] : 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, v != 0.f);
        if (v != 0.f) {
            const int p = c + __popc(m & ((1u << lane) - 1u));
            oz[p] = z;
            ov[p] = v;
        }
        c += __popc(m);
    }
    if (lane == 0) cnt[w] = c;
}

// refl [nf][nz][nx] -> reflT [nf][nx][nz], 32 x 32 tiles through shared memory
__global__ void transpose_grid_kernel(const float* __restrict__ in, float* __restrict__ out, int nz,
                                      int nx) {
    __shared__ float tile[32][33];
    const int f = blockIdx.z;
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32;
    const float* src = in + (size_t)f * nz * nx;
    float* dst = out + (size_t)f * nz * nx;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int z = z0 + j, x = x0 + threadIdx.x;
        tile[j][threadIdx.x] = (z < nz && x < nx) ? src[(size_t)z * nx + x] : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int x = x0 + j, z = z0 + threadIdx.x;
        if (x < nx && z < nz) dst[(size_t)x * nz + z] = tile[threadIdx.x][j];
    }
}

int launch_synthesize_grid(const Plan& P, const float* refl, float* rf, int nf, cudaStream_t st) {
    const DasDev& d = P.dev;
    const size_t smem_g = (size_t)4 * d.nz * sizeof(float) + (size_t)(d.nx + 1) * sizeof(int);
    if (smem_g <= 200 * 1024) {
        // reflT [nf][nx][nz], then per column the count, depths and values of
        // its nonzero pixels
        const size_t cells = (size_t)nf * d.nz * d.nx, ncols = (size_t)nf * d.nx;
        uint8_t* scratch = nullptr;
        const size_t bytes = 3 * sizeof(float) * cells + sizeof(int) * ncols;
        TIDAS_CUDA(cudaMallocAsync((void**)&scratch, bytes, st));
        float* reflT = (float*)scratch;
        float* cv = reflT + cells;
        int* cz = (int*)(cv + cells);
        int* ccnt = cz + cells;
        transpose_grid_kernel<<<dim3((d.nx + 31) / 32, (d.nz + 31) / 32, nf), dim3(32, 8), 0, st>>>(
            refl, reflT, d.nz, d.nx);
        int rc = check_launch("transpose_grid_kernel");
        if (rc == TIDAS_OK) {
            compact_columns_kernel<<<(unsigned)((ncols + 7) / 8), 256, 0, st>>>(reflT, d.nz, (int)ncols,
                                                                             ccnt, cz, cv);
            rc = check_launch("compact_columns_kernel");
        }
        if (rc == TIDAS_OK) {
            rc = check_cuda(cudaFuncSetAttribute(synth_grid_gather_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem_g),
                            "cudaFuncSetAttribute(synth_grid_gather_kernel)");
        }
        if (rc == TIDAS_OK) {
            synth_grid_gather_kernel<<<dim3(d.n_elem, d.n_angles, nf), 256, smem_g, st>>>(
                d, ccnt, cz, cv, rf);
            rc = check_launch("synth_grid_gather_kernel");
        }
        cudaFreeAsync(scratch, st);
        return rc;
    }
    size_t smem = (size_t)d.n_samples * sizeof(float);
    TIDAS_CUDA(cudaFuncSetAttribute(synth_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    synth_grid_kernel<<<dim3(d.n_elem, d.n_angles, nf), 256, smem, st>>>(d, refl, rf);
    return check_launch("synth_grid_kernel");
}

// ------------------------------------------------ synthesis transpose
// The pulse is the real part of env(t) e^{i pi wcar t} (a1): with the channel
// rows rotated to rfc[k] = rf[k] e^{i pi wcar k}, the correlation of row
// (a, n) with the pulse delayed to u = i + phi is
//     sum_m rf[m] p(m - u) = Re( e^{-i pi wcar (i + phi)} sum_j rfc[i + j] env(j - phi) ),
// j over the truncated support.  env(j - phi) follows the recurrence
// env(t + 1) = env(t) r(t), r(t) = exp(-beta (2 t + 1)), r(t + 1) = r(t) exp(-2 beta).
// rfc[k] = rf[k] carr[k], one thread per sample.
__global__ void synth_rotate_kernel(DasDev d, const float* __restrict__ rf, float2* __restrict__ rfc,
                                    long long total) {
    const int S = d.n_samples;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const float v = __ldg(rf + o);
        const float2 c = __ldg(d.carr + (int)(o % S));
        rfc[o] = make_float2(v * c.x, v * c.y);
    }
}

// One thread per pixel: correlate every rotated channel row with the
// envelope at the pixel's delay, then rotate back by the pixel's phase.
// Summation order per pixel: elements, angles, taps upwards.
// One thread per pixel; the transmit delay parts of every angle are staged
// once per thread in shared memory (each thread reads only its own slots), the
// receive correction once per (pixel, element).  The envelope values
// exp(-beta t^2) are evaluated as 2^(-beta log2(e) t^2).
__global__ void __launch_bounds__(256) synth_adjoint_kernel(DasDev d, const float2* __restrict__ rfc,
                                                            float* __restrict__ refl) {
    extern __shared__ int2 s_tx[];  // [A][256]: transmit integer part, fraction bits
    const int lane = threadIdx.x;
    const int tid = threadIdx.y * 32 + lane;
    const int ix = blockIdx.x * 32 + lane;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    if (ix >= d.nx || iz >= d.nz) return;  // no barrier follows
    const int S = d.n_samples, NE = d.n_elem, A = d.n_angles, NX = d.nx;
    for (int a = 0; a < A; ++a)
        s_tx[a * 256 + tid] =
            make_int2(__ldg(d.bxi + a * NX + ix) + __ldg(d.bzi + a * d.nz + iz),
                      __float_as_int(__ldg(d.bxf + a * NX + ix) + __ldg(d.bzf + a * d.nz + iz)));
    const float zs = __ldg(d.zs + iz);
    const float nb = -d.beta * 1.4426950408889634f;  // exp(-beta x) = 2^(nb x)
    const float h = exp2f(2.f * nb);                  // exp(-2 beta)
    const uint64_t h2 = f2(h, h);
    float acc = 0.f;
    for (int n = 0; n < NE; ++n) {
        const float exc = rx_excess(__ldg(d.dxs + (size_t)n * NX + ix), zs);
        const float2* rown = rfc + ((size_t)f * A * NE + n) * S;
        for (int a = 0; a < A; ++a) {
            const int2 b = s_tx[a * 256 + tid];
            const float uf = __int_as_float(b.y) + exc;
            const float fl = floorf(uf);
            const float phi = uf - fl;
            const int i = b.x + (int)fl;
            // taps of the support inside the record
            const int j0 = max((int)ceilf(phi - d.thalf), -i);
            const int j1 = min((int)floorf(phi + d.thalf), S - 1 - i);
            if (j0 > j1) continue;
            const float2* row = rown + (size_t)a * NE * S + i;
            const float t = (float)j0 - phi;
            const float w0 = exp2f(nb * t * t), r0 = exp2f(nb * (2.f * t + 1.f));
            // (w, w), (r, r), (re, im) as packed pairs
            uint64_t w = f2(w0, w0), r = f2(r0, r0), s2 = 0;
            const uint64_t* rp = reinterpret_cast<const uint64_t*>(row);
#pragma unroll 4
            for (int j = j0; j <= j1; ++j) {
                s2 = f2_fma(w, __ldg(rp + j), s2);
                w = f2_mul(w, r);
                r = f2_mul(r, h2);
            }
            const float sr = f2_lo(s2), si = f2_hi(s2);
            // e^{-i pi wcar (i + phi)} = conj(carr[i]) e^{-i pi wcar phi}; i lies in
            // [-kJ, S + kJ) because some tap i + j is inside the record
            const float2 ci = __ldg(d.carr + i);
            float sp, cp;
            sincospif(d.wcar * phi, &sp, &cp);
            const float zr = ci.x * cp - ci.y * sp, zi = -(ci.x * sp + ci.y * cp);
            acc = fmaf(zr, sr, fmaf(-zi, si, acc));
        }
    }
    refl[((size_t)f * d.nz + iz) * NX + ix] = acc;
}

// Moment form of the same correlation (fast Gaussian gridding, Greengard and
// Lee 2004, with the cross term expanded in a Taylor series).  Over the taps
// j of the core [clo, chi], which every fraction phi in [0, 1) keeps in the
// support,
//     sum_j rfc[i + j] env(j - phi) = e^{-beta phi^2} sum_j rfc[i + j] e^{-beta j^2} e^{a s_j},
// s_j = j / JS, a = 2 beta JS phi, and e^{a s} = sum_m a^m s^m / m!, so
//     = e^{-beta phi^2} sum_m (a^m / m!) N_m[i],  N_m[i] = sum_j rfc[i + j] e^{-beta j^2} s_j^m.
// With a <= 0.8 the first omitted term (m = kMom) is below a^10 e^a / 10! < 1e-8 of
// sum |rfc env|.  The moments are computed once per (record, sample); a pixel
// then reads kMom / 2 float4 planes and adds the taps clo - 1 and chi + 1, which
// belong to the support for some fractions only, directly.
constexpr int kMom = 10;
constexpr int kMomMaxCore = 64;

// One thread per (record, sample index ip = i + P): the rotated record window
// of the block is staged in shared memory (zero outside the record).
__global__ void __launch_bounds__(256) synth_moments_kernel(DasDev d, const float* __restrict__ rf,
                                                            float4* __restrict__ planes, int clo,
                                                            int nc, int js, int pad, int li) {
    extern __shared__ float2 smw[];              // [256 + nc - 1]
    __shared__ float tab[kMomMaxCore * kMom];    // [nc][kMom]: e^{-beta j^2} (j / js)^m
    const int R = d.n_angles * d.n_elem, S = d.n_samples;
    const int row = blockIdx.y, f = blockIdx.z;
    const int ip0 = blockIdx.x * 256;
    const int w0 = ip0 - pad + clo;              // sample of smw[0]
    const float* x = rf + ((size_t)f * R + row) * S;
    const float nb = -d.beta * 1.4426950408889634f;  // exp(-beta v) = 2^(nb v)
    for (int t = threadIdx.x; t < 256 + nc - 1; t += blockDim.x) {
        const int m = w0 + t;
        float2 v = make_float2(0.f, 0.f);
        if (m >= 0 && m < S) {
            const float r = __ldg(x + m);
            const float2 c = __ldg(d.carr + m);
            v = make_float2(r * c.x, r * c.y);
        }
        smw[t] = v;
    }
    for (int t = threadIdx.x; t < nc * kMom; t += blockDim.x) {
        const int k = t / kMom, mm = t - k * kMom;
        const int j = clo + k;
        const float sj = (float)j / (float)js;
        float pw = 1.f;
        for (int q = 0; q < mm; ++q) pw *= sj;
        tab[t] = exp2f(nb * (float)(j * j)) * pw;
    }
    __syncthreads();
    const int ip = ip0 + threadIdx.x;
    if (ip >= li) return;  // no barrier follows
    float nr[kMom], ni[kMom];
#pragma unroll
    for (int mm = 0; mm < kMom; ++mm) nr[mm] = ni[mm] = 0.f;
    for (int k = 0; k < nc; ++k) {
        const float2 v = smw[threadIdx.x + k];
#pragma unroll
        for (int mm = 0; mm < kMom; ++mm) {
            const float t = tab[k * kMom + mm];
            nr[mm] = fmaf(v.x, t, nr[mm]);
            ni[mm] = fmaf(v.y, t, ni[mm]);
        }
    }
    float4* out = planes + ((size_t)f * R + row) * (kMom / 2) * li + ip;
#pragma unroll
    for (int k = 0; k < kMom / 2; ++k)
        out[(size_t)k * li] = make_float4(nr[2 * k], ni[2 * k], nr[2 * k + 1], ni[2 * k + 1]);
}

// synth_adjoint_kernel with the core taps from the moment planes.
__global__ void __launch_bounds__(256) synth_adjoint_mom_kernel(DasDev d, const float* __restrict__ rf,
                                                                const float4* __restrict__ planes,
                                                                float* __restrict__ refl, int clo,
                                                                int chi, float ascale, int pad,
                                                                int li) {
    extern __shared__ int2 s_tx[];  // [A][256]: transmit integer part, fraction bits
    const int lane = threadIdx.x;
    const int tid = threadIdx.y * 32 + lane;
    const int ix = blockIdx.x * 32 + lane;
    const int iz = blockIdx.y * blockDim.y + threadIdx.y;
    const int f = blockIdx.z;
    if (ix >= d.nx || iz >= d.nz) return;  // no barrier follows
    const int S = d.n_samples, NE = d.n_elem, A = d.n_angles, NX = d.nx;
    for (int a = 0; a < A; ++a)
        s_tx[a * 256 + tid] =
            make_int2(__ldg(d.bxi + a * NX + ix) + __ldg(d.bzi + a * d.nz + iz),
                      __float_as_int(__ldg(d.bxf + a * NX + ix) + __ldg(d.bzf + a * d.nz + iz)));
    const float zs = __ldg(d.zs + iz);
    const float nb = -d.beta * 1.4426950408889634f;  // exp(-beta x) = 2^(nb x)
    const int jl = clo - 1, jh = chi + 1;
    float acc = 0.f;
    for (int n = 0; n < NE; ++n) {
        const float exc = rx_excess(__ldg(d.dxs + (size_t)n * NX + ix), zs);
        for (int a = 0; a < A; ++a) {
            const int2 b = s_tx[a * 256 + tid];
            const float uf = __int_as_float(b.y) + exc;
            const float fl = floorf(uf);
            const float phi = uf - fl;
            const int i = b.x + (int)fl;
            if (i < -pad || i >= S + pad) continue;  // no tap inside the record
            const int row = (f * A + a) * NE + n;
            const float4* q = planes + (size_t)row * (kMom / 2) * li + (i + pad);
            const float4 v0 = __ldg(q), v1 = __ldg(q + li), v2 = __ldg(q + 2 * (size_t)li),
                         v3 = __ldg(q + 3 * (size_t)li), v4 = __ldg(q + 4 * (size_t)li);
            // sum_m (a^m / m!) N_m by Horner's rule, a = ascale phi
            const float av = ascale * phi;
            float pr = v4.z, pi = v4.w, c;
            c = av * (1.f / 9.f); pr = fmaf(pr, c, v4.x); pi = fmaf(pi, c, v4.y);
            c = av * (1.f / 8.f); pr = fmaf(pr, c, v3.z); pi = fmaf(pi, c, v3.w);
            c = av * (1.f / 7.f); pr = fmaf(pr, c, v3.x); pi = fmaf(pi, c, v3.y);
            c = av * (1.f / 6.f); pr = fmaf(pr, c, v2.z); pi = fmaf(pi, c, v2.w);
            c = av * (1.f / 5.f); pr = fmaf(pr, c, v2.x); pi = fmaf(pi, c, v2.y);
            c = av * (1.f / 4.f); pr = fmaf(pr, c, v1.z); pi = fmaf(pi, c, v1.w);
            c = av * (1.f / 3.f); pr = fmaf(pr, c, v1.x); pi = fmaf(pi, c, v1.y);
            c = av * 0.5f;        pr = fmaf(pr, c, v0.z); pi = fmaf(pi, c, v0.w);
            pr = fmaf(pr, av, v0.x);
            pi = fmaf(pi, av, v0.y);
            const float e0 = exp2f(nb * phi * phi);
            float sr = pr * e0, si = pi * e0;
            // the two taps next to the core, where the support reaches them
            const float* x = rf + (size_t)row * S;
            if (jl >= (int)ceilf(phi - d.thalf)) {
                const int k = i + jl;
                if (k >= 0 && k < S) {
                    const float t = (float)jl - phi;
                    const float w = __ldg(x + k) * exp2f(nb * t * t);
                    const float2 ck = __ldg(d.carr + k);
                    sr = fmaf(w, ck.x, sr);
                    si = fmaf(w, ck.y, si);
                }
            }
            if (jh <= (int)floorf(phi + d.thalf)) {
                const int k = i + jh;
                if (k >= 0 && k < S) {
                    const float t = (float)jh - phi;
                    const float w = __ldg(x + k) * exp2f(nb * t * t);
                    const float2 ck = __ldg(d.carr + k);
                    sr = fmaf(w, ck.x, sr);
                    si = fmaf(w, ck.y, si);
                }
            }
            // e^{-i pi wcar (i + phi)} = conj(carr[i]) e^{-i pi wcar phi}; i lies in
            // [-kJ, S + kJ) because some tap i + j is inside the record
            const float2 ci = __ldg(d.carr + i);
            float sp, cp;
            sincospif(d.wcar * phi, &sp, &cp);
            const float zr = ci.x * cp - ci.y * sp, zi = -(ci.x * sp + ci.y * cp);
            acc = fmaf(zr, sr, fmaf(-zi, si, acc));
        }
    }
    refl[((size_t)f * d.nz + iz) * NX + ix] = acc;
}

int launch_synthesize_adjoint(const Plan& P, const float* rf, float* refl, int nf,
                              cudaStream_t st) {
    const DasDev& d = P.dev;
    // moment form when the core fits the table and the Taylor bound holds
    const int clo = (int)ceilf(1.f - d.thalf), chi = (int)floorf(d.thalf);
    const int nc = chi - clo + 1;
    const int js = max(max(-clo, chi), 1);
    const float ascale = 2.f * d.beta * (float)js;
    const int pad = chi + 2;
    const int li = d.n_samples + 2 * pad;
    const int R = d.n_angles * d.n_elem;
    if (nc >= 1 && nc <= kMomMaxCore && ascale <= 0.8f && clo <= 0 && chi >= 0 &&
        (long long)nf * R <= 65535LL * 65535LL && R <= 65535 && nf <= 65535) {
        float4* planes = nullptr;
        const size_t bytes = (size_t)nf * R * (kMom / 2) * li * sizeof(float4);
        TIDAS_CUDA(cudaMallocAsync((void**)&planes, bytes, st));
        synth_moments_kernel<<<dim3((li + 255) / 256, R, nf), 256,
                               (size_t)(256 + nc - 1) * sizeof(float2), st>>>(d, rf, planes, clo, nc,
                                                                             js, pad, li);
        int rc = check_launch("synth_moments_kernel");
        if (rc == TIDAS_OK) {
            dim3 block(32, 8);
            dim3 grid((d.nx + 31) / 32, (d.nz + 7) / 8, nf);
            synth_adjoint_mom_kernel<<<grid, block, (size_t)d.n_angles * 256 * sizeof(int2), st>>>(
                d, rf, planes, refl, clo, chi, ascale, pad, li);
            rc = check_launch("synth_adjoint_mom_kernel");
        }
        cudaFreeAsync(planes, st);
        return rc;
    }
    const long long total = (long long)nf * d.n_angles * d.n_elem * d.n_samples;
    float2* rfc = nullptr;
    TIDAS_CUDA(cudaMallocAsync((void**)&rfc, sizeof(float2) * (size_t)total, st));
    const long long blocks = (total + 255) / 256;
    synth_rotate_kernel<<<(int)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, st>>>(d, rf, rfc,
                                                                                     total);
    int rc = check_launch("synth_rotate_kernel");
    if (rc == TIDAS_OK) {
        dim3 block(32, 8);
        dim3 grid((d.nx + 31) / 32, (d.nz + 7) / 8, nf);
        synth_adjoint_kernel<<<grid, block, (size_t)d.n_angles * 256 * sizeof(int2), st>>>(d, rfc,
                                                                                       refl);
        rc = check_launch("synth_adjoint_kernel");
    }
    cudaFreeAsync(rfc, st);
    return rc;
}

// ------------------------------------------------------- PSF / kernel fit
// Exact single-scatterer PSF (Eq. (2.6)-(2.7)): the DAS value at pixel
// (ic + t - taps/2, iz) of a unit scatterer on pixel (ic, iz), without
// materialising channel data: the beamformer reads the sampled pulse
// p(m - u_scat) at the interpolation taps m around u_pix.  Delays in FP64.
struct FitArgs {
    int n_elem, n_angles, nx, nz, taps, ic, interp, n_samples;
    int kz;  // output rows per kernel: rows iz + u - kz/2, u = 0..kz-1 (1: the row itself)
    double pitch, c, fs, t0, x0, dx, z0, dz, fnum;
    double thalf, beta, wcar;  // samples
};

__device__ __forceinline__ double delay_fp64(const FitArgs& A, double sn, double cs, int n,
                                             double x, double z) {
    double xn = __dmul_rn(__dsub_rn((double)n, 0.5 * (double)(A.n_elem - 1)), A.pitch);
    double ddx = __dsub_rn(x, xn);
    double tx = __dadd_rn(__dmul_rn(x, sn), __dmul_rn(z, cs));
    double rx = __dsqrt_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(z, z)));
    return __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tx, rx), A.c), A.t0), A.fs);
}

__device__ __forceinline__ double pulse_fp(const FitArgs& A, double t) {
    if (fabs(t) > A.thalf) return 0.0;
    float tf = (float)t;
    return (double)(expf(-(float)A.beta * tf * tf) * cospif((float)A.wcar * tf));
}

__global__ void fit_psf_kernel(FitArgs A, const double* __restrict__ sncs, float* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int u = blockIdx.z;  // output row iz + u - kz/2 (also outside the grid)
    if (t >= A.taps) return;
    const int ix = A.ic + t - A.taps / 2;
    float result = 0.f;
    const double zsc = A.z0 + ((double)iz + 0.5) * A.dz;                  // scatterer
    const double z = A.z0 + ((double)(iz + u - A.kz / 2) + 0.5) * A.dz;   // pixel
    if (ix >= 0 && ix < A.nx && z > 0.0) {
        const double xs = A.x0 + ((double)A.ic + 0.5) * A.dx;  // scatterer
        const double xp = A.x0 + ((double)ix + 0.5) * A.dx;    // pixel
        double acc = 0.0;
        for (int a = 0; a < A.n_angles; ++a) {
            const double sn = sncs[2 * a], cs = sncs[2 * a + 1];
            for (int n = 0; n < A.n_elem; ++n) {
                double w = 1.0;
                if (A.fnum > 0) {
                    double xn = ((double)n - 0.5 * (double)(A.n_elem - 1)) * A.pitch;
                    double r = (xp - xn) * A.fnum / z;
                    if (fabs(r) > 0.5) continue;
                    double cw = cospi(r);
                    w = cw * cw;
                }
                const double up = delay_fp64(A, sn, cs, n, xp, z);
                const double us = delay_fp64(A, sn, cs, n, xs, zsc);
                const double fl = floor(up);
                const double phi = up - fl;
                const int i = (int)fl;
                double v = 0.0;
                if (A.interp == TIDAS_INTERP_CUBIC) {
                    float w0, w1, w2, w3;
                    keys_weights((float)phi, w0, w1, w2, w3);
                    const float wt[4] = {w0, w1, w2, w3};
                    for (int k = 0; k < 4; ++k) {
                        const int m = i - 1 + k;
                        if (m < 0 || m >= A.n_samples) continue;
                        v += (double)wt[k] * pulse_fp(A, (double)m - us);
                    }
                } else {
                    if (i >= 0 && i < A.n_samples) v += (1.0 - phi) * pulse_fp(A, (double)i - us);
                    if (i + 1 >= 0 && i + 1 < A.n_samples)
                        v += phi * pulse_fp(A, (double)(i + 1) - us);
                }
                acc += w * v;
            }
        }
        result = (float)acc;
    }
    out[((size_t)iz * A.kz + u) * A.taps + t] = result;
}

// Rows other than the reference rows become theta * (reference PSF), with
// theta the least-squares weight of Eq. (2.12); reference rows are only read.
__global__ void fit_theta_kernel(int nz, int taps, int ref_stride, float* __restrict__ kern,
                                 float* __restrict__ theta) {
    const int iz = blockIdx.x;
    int s = (iz / ref_stride) * ref_stride + ref_stride / 2;
    if (s > nz - 1) s = nz - 1;
    if (iz == s) {
        if (theta && threadIdx.x == 0) theta[iz] = 1.f;
        return;
    }
    __shared__ double red_ab[256], red_aa[256];
    double ab = 0.0, aa = 0.0;
    for (int t = threadIdx.x; t < taps; t += blockDim.x) {
        double a = kern[(size_t)s * taps + t], b = kern[(size_t)iz * taps + t];
        ab += a * b;
        aa += a * a;
    }
    red_ab[threadIdx.x] = ab;
    red_aa[threadIdx.x] = aa;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            red_ab[threadIdx.x] += red_ab[threadIdx.x + k];
            red_aa[threadIdx.x] += red_aa[threadIdx.x + k];
        }
        __syncthreads();
    }
    const double th = red_aa[0] > 0 ? red_ab[0] / red_aa[0] : 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < taps; t += blockDim.x)
        kern[(size_t)iz * taps + t] = (float)(th * (double)kern[(size_t)s * taps + t]);
    if (theta && threadIdx.x == 0) theta[iz] = (float)th;
}

__global__ void fill_ones_kernel(float* p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 1.f;
}

static FitArgs fit_args(const Plan& P, int taps, int kz) {
    FitArgs A;
    A.kz = kz;
    A.n_elem = P.p.n_elem;
    A.n_angles = P.p.n_angles;
    A.nx = P.p.nx;
    A.nz = P.p.nz;
    A.taps = taps;
    A.ic = P.p.nx / 2;
    A.interp = P.p.interp;
    A.n_samples = P.p.n_samples;
    A.pitch = P.p.pitch;
    A.c = P.p.c;
    A.fs = P.p.fs;
    A.t0 = P.p.t0;
    A.x0 = P.p.x0;
    A.dx = P.p.dx;
    A.z0 = P.p.z0;
    A.dz = P.p.dz;
    A.fnum = P.p.fnum;
    A.thalf = P.thalf_samples;
    A.beta = P.beta_samples;
    A.wcar = P.wcar;
    return A;
}

int launch_fit_kernels(const Plan& P, int taps, int ref_stride, float* kernels, float* theta,
                       cudaStream_t st) {
    const FitArgs A = fit_args(P, taps, 1);
    dim3 grid((taps + 63) / 64, P.p.nz, 1);
    fit_psf_kernel<<<grid, 64, 0, st>>>(A, P.d_sncs, kernels);
    int rc = check_launch("fit_psf_kernel");
    if (rc) return rc;
    if (ref_stride > 1) {
        fit_theta_kernel<<<P.p.nz, 256, 0, st>>>(P.p.nz, taps, ref_stride, kernels, theta);
        rc = check_launch("fit_theta_kernel");
    } else if (theta) {
        fill_ones_kernel<<<(P.p.nz + 255) / 256, 256, 0, st>>>(theta, P.p.nz);
        rc = check_launch("fill_ones_kernel");
    }
    return rc;
}

// 2D band kernels [nz][kz][taps]: the single-scatterer image of every row over
// kz output rows centred on it.
int launch_fit_kernels_2d(const Plan& P, int kz, int taps, float* kernels, cudaStream_t st) {
    const FitArgs A = fit_args(P, taps, kz);
    dim3 grid((taps + 63) / 64, P.p.nz, kz);
    fit_psf_kernel<<<grid, 64, 0, st>>>(A, P.d_sncs, kernels);
    return check_launch("fit_psf_kernel");
}

}  // namespace tidas
