// Delay-and-Sum (Eq. (2.2)) of single frames and batches of up to six frames
// on CUDA cores from per-interval interpolation coefficients, FP32 or FP16
// channel data.
//
// On the sample interval [i, i + 1] of a record x the Keys cubic interpolant
// (Eq. (2.2)'s interpolation of the delayed channel sample) is one cubic
// polynomial in the fraction phi.  Written about the interval's midpoint,
// psi = phi - 1/2 in [-1/2, 1/2],
//   y = d0 + psi (d1 + psi (d2 + psi d3)),
//   d0 = (9 (x[i] + x[i+1]) - (x[i-1] + x[i+2])) / 16,
//   d1 = (11 (x[i+1] - x[i]) - (x[i+2] - x[i-1])) / 8,
//   d2 = (x[i-1] - x[i] - x[i+1] + x[i+2]) / 4,
//   d3 = (x[i+2] - x[i-1]) / 2 + 3 (x[i] - x[i+1]) / 2,
// which is the four-tap Keys sum w0 x[i-1] + .. + w3 x[i+2] with its terms
// regrouped by powers of psi.  Linear interpolation keeps d0 = (x[i] +
// x[i+1]) / 2 and d1 = x[i+1] - x[i].  A first pass writes the coefficients of
// every interval whose taps meet the plan's read window (samples outside the
// window count as zero, as do samples outside the record); the DAS kernel
// then reads one 16-byte (cubic) or 8-byte (linear) vector per (pixel, angle,
// element) and evaluates it by Horner's rule: no per-update weight polynomial
// and one load in place of four.  A 16-byte vector costs about 6 L1
// wavefronts per warp against about 4.3 for four scalar taps, so larger
// batches, whose delays and weights are shared by their frames, gather
// samples instead (das_kernels.cu).
#include <climits>

#include "common.cuh"

namespace tidas {

template <int INTERP>
struct CoefT;
template <>
struct CoefT<TIDAS_INTERP_CUBIC> {
    using T = float4;
};
template <>
struct CoefT<TIDAS_INTERP_LINEAR> {
    using T = float2;
};

// 1.5 * 2^23: adding it to |u| < 2^22 rounds u to the nearest integer, which
// then sits in the low mantissa bits (float_as_int(u + kMagic) - kMagicBits)
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

// batches this path takes (the caller routes larger ones to sample gathers)
constexpr int kCoeffMaxFrames = 6;

template <typename RF>
__device__ __forceinline__ float load_x(const RF* __restrict__ row, int m, int lo, int hi) {
    return (m >= lo && m < hi) ? load_rf(row + m) : 0.f;
}

// One thread per interval entry e of one (angle, element) row: entry e holds
// interval i = I0 + e.
template <typename RF, int INTERP>
__global__ void __launch_bounds__(256) das_coeff_pack_kernel(
    const RF* __restrict__ rf, typename CoefT<INTERP>::T* __restrict__ out, int S, int L, int I0,
    int lo, int hi, int neb) {
    const int eb = blockIdx.x % neb;
    const int row = blockIdx.x / neb;  // angle * n_elem + element
    const int e = eb * 256 + threadIdx.x;
    if (e >= L) return;
    const int i = I0 + e;
    const RF* x = rf + (size_t)row * S;
    const float xm1 = load_x(x, i - 1, lo, hi);
    const float x0 = load_x(x, i, lo, hi);
    const float x1 = load_x(x, i + 1, lo, hi);
    const float x2 = load_x(x, i + 2, lo, hi);
    typename CoefT<INTERP>::T c;
    if constexpr (INTERP == TIDAS_INTERP_CUBIC) {
        c.x = (9.f * (x0 + x1) - (xm1 + x2)) * 0.0625f;
        c.y = (11.f * (x1 - x0) - (x2 - xm1)) * 0.125f;
        c.z = ((xm1 + x2) - (x0 + x1)) * 0.25f;
        c.w = 0.5f * (x2 - xm1) + 1.5f * (x0 - x1);
    } else {
        c.x = 0.5f * (x0 + x1);
        c.y = x1 - x0;
    }
    out[(size_t)row * L + e] = c;
}

template <int INTERP>
__device__ __forceinline__ float coef_eval(const typename CoefT<INTERP>::T& c, float psi) {
    if constexpr (INTERP == TIDAS_INTERP_CUBIC)
        return fmaf(fmaf(fmaf(c.w, psi, c.z), psi, c.y), psi, c.x);
    else
        return fmaf(c.y, psi, c.x);
}

// cos(pi r) for |r| <= 1/2 from its Taylor series in t = r^2 through t^6
// (coefficients (-1)^k pi^(2k) / (2k)!); the first omitted term is at most
// (pi / 2)^14 / 14! < 7e-9, below the FP32 rounding of the sum.
__device__ __forceinline__ float cospi_half(float r) {
    constexpr double p2 = 9.8696044010893586188;  // pi^2
    constexpr float c1 = (float)(-p2 / 2.0);
    constexpr float c2 = (float)(p2 * p2 / 24.0);
    constexpr float c3 = (float)(-p2 * p2 * p2 / 720.0);
    constexpr float c4 = (float)(p2 * p2 * p2 * p2 / 40320.0);
    constexpr float c5 = (float)(-p2 * p2 * p2 * p2 * p2 / 3628800.0);
    constexpr float c6 = (float)(p2 * p2 * p2 * p2 * p2 * p2 / 479001600.0);
    const float t = r * r;
    float p = fmaf(c6, t, c5);
    p = fmaf(p, t, c4);
    p = fmaf(p, t, c3);
    p = fmaf(p, t, c2);
    p = fmaf(p, t, c1);
    return fmaf(p, t, 1.f);
}

// One thread per pixel; a warp covers 32 neighbouring columns of one row, so
// the 32 vectors of one (angle, element) fall in a few lines.  The receive
// correction and the Hann apodization cos^2(pi r), r = (x - x_n) F# / z, of a
// (pixel, element) serve every angle.  The angle count A is a template
// parameter: the angle loop unrolls fully, so a warp has the A loads of one
// element in flight at once (a runtime count of 11 ran 1.2x slower).
// CHECK: some pixel's taps leave the record; the entry index is clamped to
// the row, whose first and last entries (intervals I0 and I0 + L - 1) have no
// tap inside the record and hold zeros.
template <int INTERP, bool CHECK, int A, int FB>
__global__ void __launch_bounds__(256, FB == 1 ? 4 : 2)
    das_coeff_kernel(DasDev d, const typename CoefT<INTERP>::T* __restrict__ cf, int fstride,
                     int L, int I0, float* __restrict__ img, int nf) {
    using T = typename CoefT<INTERP>::T;
    // per thread and angle: (transmit integer part - I0 - kMagicBits, plus the
    // angle's row offset unless CHECK; transmit fraction - 1/2)
    extern __shared__ int2 s_b[];  // [A][256]
    const int lane = threadIdx.x;
    const int tid = threadIdx.y * 32 + lane;
    const int ix = blockIdx.x * 32 + lane;
    // deepest rows first (widest apertures), so the last blocks are the cheap ones
    const int iz = (gridDim.y - 1 - blockIdx.y) * blockDim.y + threadIdx.y;
    if (iz >= d.nz) return;  // uniform per warp; no block-wide barrier follows
    const int NE = d.n_elem, NX = d.nx;
    const bool xin = ix < NX;
    const int ixc = xin ? ix : NX - 1;
    const int rowstride = NE * L;  // entries between angles of one element
#pragma unroll
    for (int a = 0; a < A; ++a) {
        const int bi = __ldg(d.bxi + a * NX + ixc) + __ldg(d.bzi + a * d.nz + iz);
        const float bf = __ldg(d.bxf + a * NX + ixc) + __ldg(d.bzf + a * d.nz + iz);
        const int base = CHECK ? bi - I0 - kMagicBits : bi - I0 - kMagicBits + a * rowstride;
        s_b[a * 256 + tid] = make_int2(base, __float_as_int(bf - 0.5f));
    }
    __syncwarp();
    const float zs = __ldg(d.zs + iz);
    const float fz = d.fnum / zs;  // r = dxs * fz

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

    const int f0 = blockIdx.z * FB;
    const typename CoefT<INTERP>::T* cf0 = cf + (size_t)f0 * fstride;
    float acc[FB];
#pragma unroll
    for (int f = 0; f < FB; ++f) acc[f] = 0.f;
    const int2* sb = s_b + tid;
    for (int n = n_lo; n <= n_hi; ++n) {
        const float dxs = __ldg(d.dxs + (size_t)n * NX + ixc);
        float w = 1.f;
        if (d.fnum > 0.f) {
            const float r = dxs * fz;
            const float cw = cospi_half(r);
            w = fabsf(r) > 0.5f ? 0.f : cw * cw;
        }
        if (!xin) w = 0.f;
        if (__ballot_sync(0xffffffffu, w != 0.f) == 0u) continue;
        const float exc = rx_excess(dxs, zs);
        const int on = n * L;
#pragma unroll
        for (int a = 0; a < A; ++a) {
            const int2 b = sb[a * 256];
            // u = delay - 1/2; round(u) is the interval's first sample, psi its
            // offset from the interval's midpoint
            const float u = __int_as_float(b.y) + exc;
            const float m = u + kMagic;
            const float psi = u - (m - kMagic);
            int o;
            if (CHECK) {
                const int e = min(max(b.x + __float_as_int(m), 0), L - 1);
                o = e + on + a * rowstride;
            } else {
                o = b.x + on + __float_as_int(m);
            }
            T c[FB];
#pragma unroll
            for (int f = 0; f < FB; ++f) c[f] = __ldg(cf0 + o + f * fstride);
#pragma unroll
            for (int f = 0; f < FB; ++f) acc[f] = fmaf(w, coef_eval<INTERP>(c[f], psi), acc[f]);
        }
    }
    if (xin) {
#pragma unroll
        for (int f = 0; f < FB; ++f)
            if (f0 + f < nf) img[((size_t)(f0 + f) * d.nz + iz) * NX + ix] = acc[f];
    }
}

template <int INTERP, bool CHECK, int A>
static void das_coeff_launch(const DasDev& d, const void* cf, int fstride, int L, int I0,
                             float* img, int nf, int fb, cudaStream_t st) {
    using T = typename CoefT<INTERP>::T;
    const T* c = (const T*)cf;
    dim3 block(32, 8);
    dim3 grid((d.nx + 31) / 32, (d.nz + 7) / 8, (nf + fb - 1) / fb);
    const size_t sm = (size_t)A * 256 * sizeof(int2);
    if (fb == 4) das_coeff_kernel<INTERP, CHECK, A, 4><<<grid, block, sm, st>>>(d, c, fstride, L, I0, img, nf);
    else if (fb == 2) das_coeff_kernel<INTERP, CHECK, A, 2><<<grid, block, sm, st>>>(d, c, fstride, L, I0, img, nf);
    else das_coeff_kernel<INTERP, CHECK, A, 1><<<grid, block, sm, st>>>(d, c, fstride, L, I0, img, nf);
}

template <int INTERP, bool CHECK, int A = 1>
static void das_coeff_dispatch(const DasDev& d, const void* cf, int fstride, int L, int I0,
                               float* img, int nf, int fb, cudaStream_t st) {
    if constexpr (A < kMaxAngles) {
        if (d.n_angles != A) {
            das_coeff_dispatch<INTERP, CHECK, A + 1>(d, cf, fstride, L, I0, img, nf, fb, st);
            return;
        }
    }
    das_coeff_launch<INTERP, CHECK, A>(d, cf, fstride, L, I0, img, nf, fb, st);
}

int launch_das_coeff(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st) {
    const DasDev& d = P.dev;
    if (nf < 1 || nf > kCoeffMaxFrames)
        return set_error(TIDAS_ERR_ARG, "das_forward: coefficient path takes 1..%d frames", kCoeffMaxFrames);
    if (P.read_count <= 0) {
        // no tap of any pixel lies in the record: every pixel is zero
        if (cudaMemsetAsync(img, 0, sizeof(float) * (size_t)nf * d.nz * d.nx, st) != cudaSuccess)
            return check_launch("das_forward: memset");
        return TIDAS_OK;
    }
    const bool cubic = d.interp == TIDAS_INTERP_CUBIC;
    const bool f16 = d.rf_dtype == TIDAS_RF_F16;
    const int R = d.n_angles * d.n_elem, S = d.n_samples;
    // intervals I0 .. I0 + L - 1: every interval with a tap in the read window,
    // plus one each side with no tap in it (the CHECK clamp's zero entries)
    const int I0 = P.read_first - 3;
    const int L = P.read_count + 5;
    const size_t esz = cubic ? sizeof(float4) : sizeof(float2);
    const size_t fstride = (size_t)R * L;  // entries per frame
    // frames per thread: a divisor of nf (the per-frame cost falls only
    // slightly with more frames per thread, so padded frames would not pay)
    const int fb = nf % 4 == 0 ? 4 : (nf % 2 == 0 ? 2 : 1);
    if (fstride * nf > (size_t)INT_MAX)
        return set_error(TIDAS_ERR_UNSUPPORTED, "das_forward: record too long");
    // a guard of 1024 entries each side keeps an entry index that left its row
    // inside the allocation
    constexpr size_t kGuard = 1024;
    const size_t need = (fstride * nf + 2 * kGuard) * esz;
    void* ws = nullptr;
    bool fresh = false;  // every entry the kernel reads is written below
    if (int rc = plan_staging(P, need, &ws, 3, &fresh)) return rc;
    uint8_t* base = (uint8_t*)ws + kGuard * esz;
    const int neb = (L + 255) / 256;
    const size_t blocks = (size_t)nf * R * neb;
    const int lo = P.read_first, hi = P.read_first + P.read_count;
    if (f16) {
        if (cubic)
            das_coeff_pack_kernel<__half, TIDAS_INTERP_CUBIC><<<(unsigned)blocks, 256, 0, st>>>(
                (const __half*)rf, (float4*)base, S, L, I0, lo, hi, neb);
        else
            das_coeff_pack_kernel<__half, TIDAS_INTERP_LINEAR><<<(unsigned)blocks, 256, 0, st>>>(
                (const __half*)rf, (float2*)base, S, L, I0, lo, hi, neb);
    } else {
        if (cubic)
            das_coeff_pack_kernel<float, TIDAS_INTERP_CUBIC><<<(unsigned)blocks, 256, 0, st>>>(
                (const float*)rf, (float4*)base, S, L, I0, lo, hi, neb);
        else
            das_coeff_pack_kernel<float, TIDAS_INTERP_LINEAR><<<(unsigned)blocks, 256, 0, st>>>(
                (const float*)rf, (float2*)base, S, L, I0, lo, hi, neb);
    }
    if (int rc = check_launch("das_coeff_pack_kernel")) return rc;
    const bool check = !P.taps_in_range;
    const int fs = (int)fstride;
    if (cubic) {
        if (check) das_coeff_dispatch<TIDAS_INTERP_CUBIC, true>(d, base, fs, L, I0, img, nf, fb, st);
        else das_coeff_dispatch<TIDAS_INTERP_CUBIC, false>(d, base, fs, L, I0, img, nf, fb, st);
    } else {
        if (check) das_coeff_dispatch<TIDAS_INTERP_LINEAR, true>(d, base, fs, L, I0, img, nf, fb, st);
        else das_coeff_dispatch<TIDAS_INTERP_LINEAR, false>(d, base, fs, L, I0, img, nf, fb, st);
    }
    return check_launch("das_coeff_kernel");
}

}  // namespace tidas
