// Single-line experiment of Section 3: focused transmit on the array axis,
// channel data of a unit scatterer on every line point, the DAS line with
// dynamic receive focusing (Eq. (2.2), (2.3), (2.7)), and the sweep of
// Eq. (2.8) / (2.12) over every (fixed delay curve s, scatterer r): the
// windowed channels of r aligned with the delay set of line point s, their
// weight theta (Eq. (2.12), first line: <a, b> / <a, a> with b the
// scatterer's own curve) and the local / global errors of Section 3.3.
//
// Geometry and readings (as in the header): transmit half-aperture from
// Kossoff's criterion, a_tx = sqrt(z_focus lambda / kappa); element m fires at
// (z_focus - |focus - x_m|) / c; receive aperture |x_n| <= z / (2 F#) of the
// focused depth; window: the samples within eps of the scatterer's echo
// arrival on each channel.  Every decision that selects samples or elements
// (apertures, windows, sample indices) is made in FP64 with the operations
// rounded one at a time, so that it matches a plain FP64 evaluation exactly;
// the sums run in FP32.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace tidas {

namespace line {
constexpr int kStage = 32;     // staged samples per channel in the sweep (window + taps)
constexpr int kStride = 33;    // their shared-memory stride: lanes on different channels
                               // fall in different banks
constexpr int kSweepWarps = 8;

struct Dev {
    int N, S, D, interp;
    double pitch, f0, fs, c, z_first, z_last, z_focus, kossoff, fnum;
    double alpha, thalf;  // pulse envelope exp(-alpha t^2), truncated at |t| > thalf
    float du, u0;         // fixed-curve position 2 z_i fs / c ~ u0 + du i (range estimates)
};

__device__ __forceinline__ double elem_x(const Dev& L, int n) {
    return __dmul_rn(__dsub_rn((double)n, __dmul_rn(0.5, (double)(L.N - 1))), L.pitch);
}
__device__ __forceinline__ double depth(const Dev& L, int i) {
    return __dadd_rn(L.z_first,
                     __ddiv_rn(__dmul_rn(__dsub_rn(L.z_last, L.z_first), (double)i),
                               (double)(L.D - 1)));
}
__device__ __forceinline__ double hyp(double x, double z) {
    return __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(z, z)));
}
__device__ __forceinline__ bool rx_active(const Dev& L, double xn, double z) {
    return fabs(xn) <= __ddiv_rn(z, __dmul_rn(2.0, L.fnum));
}
// Eq. (2.3) for the on-axis point at depth z
__device__ __forceinline__ double delay(const Dev& L, double xn, double z) {
    return __ddiv_rn(__dsub_rn(z, hyp(xn, z)), L.c);
}
__device__ __forceinline__ double arrival(const Dev& L, double xn, double z) {
    return __dadd_rn(__ddiv_rn(z, L.c), __ddiv_rn(hyp(xn, z), L.c));
}

// float -> int clamped well inside the int range
__device__ __forceinline__ int clamp_i(float x) { return (int)fminf(fmaxf(x, -1e9f), 1e9f); }

// Sample position -> (index, fraction) and the interpolated value of a row
// accessed through `at` (zero outside what `at` covers).
template <class At>
__device__ __forceinline__ float interp(int interp_mode, int idx, float phi, At at) {
    if (interp_mode == TIDAS_INTERP_CUBIC) {
        float w0, w1, w2, w3;
        keys_weights(phi, w0, w1, w2, w3);
        return w0 * at(idx - 1) + w1 * at(idx) + w2 * at(idx + 1) + w3 * at(idx + 2);
    }
    return (1.f - phi) * at(idx) + phi * at(idx + 1);
}
}  // namespace line

// ------------------------------------------------------------- synthesis
// Block (16 elements, scatterer).  The transmit part of every wavelet's
// arrival (fire_m + |r - x_m| / c) is computed once per block, the receive
// part once per row, both in FP64; the sample loop runs in FP32 on the split
// arrivals (FP64 is a narrow unit on this part), and only the samples at the
// pulse's cut-off repeat the decision in FP64.
constexpr int kSynthRows = 16;
__global__ void __launch_bounds__(256) line_synth_kernel(line::Dev L, int r_first,
                                                         float* __restrict__ rf) {
    using namespace line;
    __shared__ double s_tx[1024];   // transmit part of wavelet m's arrival
    __shared__ double s_tau[1024];  // full arrival on the current row
    __shared__ int s_ki[1024];      // fs tau_m = s_ki[m] + s_kf[m]
    __shared__ float s_kf[1024];
    __shared__ int s_m0, s_m1;      // transmit aperture: elements m0 .. m1 (contiguous)
    __shared__ double s_zr;
    __shared__ long s_klo, s_khi;
    const int rs = blockIdx.y, r = r_first + rs;
    if (threadIdx.x == 0) {
        s_m0 = INT_MAX;
        s_m1 = -1;
        s_zr = depth(L, r);
    }
    __syncthreads();
    const double zr = s_zr;
    const double a_tx = __dsqrt_rn(__ddiv_rn(__dmul_rn(L.z_focus, __ddiv_rn(L.c, L.f0)), L.kossoff));
    for (int m = threadIdx.x; m < L.N; m += blockDim.x) {
        const double xm = elem_x(L, m);
        if (fabs(xm) > a_tx) continue;
        const double fire = __ddiv_rn(__dsub_rn(L.z_focus, hyp(xm, L.z_focus)), L.c);
        s_tx[m] = __dadd_rn(fire, __ddiv_rn(hyp(xm, zr), L.c));
        atomicMin(&s_m0, m);
        atomicMax(&s_m1, m);
    }
    __syncthreads();
    const int m0 = s_m0, m1 = s_m1;
    // the pulse in sample units: exp(-(alpha / fs^2) d^2) cos(2 pi (f0 / fs) d)
    const float a_s = (float)(L.alpha / (L.fs * L.fs));
    const float two_f0 = (float)(2.0 * L.f0 / L.fs);
    const float half_s = (float)(L.thalf * L.fs);
    const int n_end = min(L.N, (int)(blockIdx.x + 1) * kSynthRows);
    for (int n = blockIdx.x * kSynthRows; n < n_end; ++n) {
        if (threadIdx.x < 32) {
            const double rx = __ddiv_rn(hyp(elem_x(L, n), zr), L.c);
            double lo = 1e300, hi = -1e300;
            for (int m = m0 + (int)threadIdx.x; m <= m1; m += 32) {
                const double tau = __dadd_rn(s_tx[m], rx);
                s_tau[m] = tau;
                const double kt = __dmul_rn(tau, L.fs);
                const double fl = floor(kt);
                s_ki[m] = (int)fl;
                s_kf[m] = (float)(kt - fl);
                lo = fmin(lo, tau);
                hi = fmax(hi, tau);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (threadIdx.x == 0) {
                const bool any = m0 <= m1;
                s_klo = any ? (long)floor((lo - L.thalf) * L.fs) - 1 : 1;
                s_khi = any ? (long)ceil((hi + L.thalf) * L.fs) + 1 : 0;
            }
        }
        __syncthreads();
        const long k_lo = s_klo, k_hi = s_khi;
        float* row = rf + ((size_t)rs * L.N + n) * L.S;
        for (int k = threadIdx.x; k < L.S; k += blockDim.x) {
            float acc = 0.f;
            if (k >= k_lo && k <= k_hi) {
                for (int m = m0; m <= m1; ++m) {  // fixed order: same sum in every launch
                    const float d = (float)(k - s_ki[m]) - s_kf[m];
                    const float ad = fabsf(d);
                    if (ad > half_s + 1e-3f) continue;
                    // the cut-off itself is decided in FP64, as t = k / fs - tau
                    if (ad > half_s - 1e-3f &&
                        fabs(__dsub_rn(__ddiv_rn((double)k, L.fs), s_tau[m])) > L.thalf)
                        continue;
                    acc += expf(-a_s * d * d) * cospif(two_f0 * d);
                }
            }
            row[k] = acc;
        }
        __syncthreads();  // s_tau / s_ki of this row are rewritten for the next
    }
}

// ---------------------------------------------------------------- tables
// das_*[i][n] : sample position of the DAS line (dynamic focus) split into
//               integer and FP32 fraction; index INT_MIN = element not active
// u_*[i]      : 2 z_i / c * fs split; v_*[s][n]: D_n(z_s) * fs split, so that
//               the fixed-curve position (2 z_i / c - D_n(z_s)) fs is their
//               difference; act[s][n]: receive aperture of line point s
struct LineTab {
    int* das_idx;
    float* das_frac;
    int* u_idx;
    float* u_frac;
    int* v_idx;
    float* v_frac;
    uint8_t* act;
};

__global__ void line_table_kernel(line::Dev L, LineTab T) {
    using namespace line;
    const int total = L.D * L.N;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int i = q / L.N, n = q % L.N;
        const double zi = depth(L, i), xn = elem_x(L, n);
        const bool on = rx_active(L, xn, zi);
        const double d = delay(L, xn, zi);
        const double u = __dmul_rn(__dsub_rn(__ddiv_rn(__dmul_rn(2.0, zi), L.c), d), L.fs);
        const double fl = floor(u);
        T.das_idx[q] = on ? (int)fl : INT_MIN;
        T.das_frac[q] = (float)(u - fl);
        T.act[q] = on ? 1 : 0;
        const double v = __dmul_rn(d, L.fs);
        const double vf = floor(v);
        T.v_idx[q] = (int)vf;
        T.v_frac[q] = (float)(v - vf);
        if (n == 0) {
            const double uu = __dmul_rn(__ddiv_rn(__dmul_rn(2.0, zi), L.c), L.fs);
            const double uf = floor(uu);
            T.u_idx[i] = (int)uf;
            T.u_frac[i] = (float)(uu - uf);
        }
    }
}

// ----------------------------------------------------------------- DAS line
// Block (32 line points, scatterer); warp per point, lanes over elements.
__global__ void __launch_bounds__(256) line_das_kernel(line::Dev L, LineTab T,
                                                       const float* __restrict__ rf,
                                                       float* __restrict__ lines) {
    using namespace line;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rs = blockIdx.y;
    const float* S = rf + (size_t)rs * L.N * L.S;
    for (int i = blockIdx.x * 32 + warp; i < min(L.D, blockIdx.x * 32 + 32); i += 8) {
        float acc = 0.f;
        for (int n = lane; n < L.N; n += 32) {
            const int idx = T.das_idx[i * L.N + n];
            if (idx == INT_MIN) continue;
            const float* row = S + (size_t)n * L.S;
            acc += interp(L.interp, idx, T.das_frac[i * L.N + n], [&](int k) {
                return (k >= 0 && k < L.S) ? __ldg(row + k) : 0.f;
            });
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) lines[(size_t)rs * L.D + i] = acc;
    }
}

// -------------------------------------------------------------------- sweep
// Block per scatterer r.  The windowed channels of r (kStage samples from
// k_lo - 2 per element) sit in shared memory; each warp takes delay curves
// s = warp, warp + 8, ..., builds the fixed-curve line a_s in its own buffer
// (every element adds its window's contribution to the line points it
// reaches), and reduces theta and the errors.
__device__ void sweep_curve(const line::Dev& L, const LineTab& T, int r, int s, int lane,
                            const float* __restrict__ sw, const int* __restrict__ klo,
                            const int* __restrict__ khi, float* __restrict__ abuf, int& ilo,
                            int& ihi) {
    using namespace line;
    // union of the line points the active elements reach (a conservative
    // range from the linear law of u in i; exact positions below)
    const float du = L.du, u0 = L.u0;
    int lo = INT_MAX, hi = INT_MIN;
    for (int n = lane; n < L.N; n += 32) {
        if (!T.act[s * L.N + n] || klo[n] > khi[n]) continue;
        const float v = (float)T.v_idx[s * L.N + n] + T.v_frac[s * L.N + n];
        lo = min(lo, clamp_i(floorf(((float)(klo[n] - 3) + v - u0) / du)) - 1);
        hi = max(hi, clamp_i(ceilf(((float)(khi[n] + 3) + v - u0) / du)) + 1);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lo > hi) {  // no element reaches the line (also lo = INT_MAX)
        lo = 0;
        hi = -1;
    }
    lo = max(lo, 0);
    hi = min(hi, L.D - 1);
    ilo = lo;
    ihi = hi;
    for (int i = lo + lane; i <= hi; i += 32) abuf[i] = 0.f;
    __syncwarp();
    for (int n = lane; n < L.N; n += 32) {
        if (!T.act[s * L.N + n] || klo[n] > khi[n]) continue;
        const int vi = T.v_idx[s * L.N + n];
        const float vf = T.v_frac[s * L.N + n];
        const float v = (float)vi + vf;
        const int a0 = max(lo, clamp_i(floorf(((float)(klo[n] - 3) + v - u0) / du)) - 1);
        const int a1 = min(hi, clamp_i(ceilf(((float)(khi[n] + 3) + v - u0) / du)) + 1);
        const float* row = sw + n * kStride;
        const int base = klo[n] - 2;
        for (int i = a0; i <= a1; ++i) {
            const float f = T.u_frac[i] - vf;
            const float fl = floorf(f);
            const int idx = T.u_idx[i] - vi + (int)fl;
            if (idx + 2 < klo[n] || idx - 1 > khi[n]) continue;
            const float val = interp(L.interp, idx, f - fl, [&](int k) {
                const int j = k - base;
                return (j >= 0 && j < kStage) ? row[j] : 0.f;
            });
            if (val != 0.f) atomicAdd(&abuf[i], val);
        }
    }
    __syncwarp();
}

// The windows of Eq. (2.8) for scatterer depth zr: per channel the samples k
// with |k / fs - t_n| <= eps (t_n the echo arrival), tested one by one from
// just below t_n - eps, then the windowed samples from k_lo - 2 into shared
// memory (kStage per channel at stride kStride, zero outside the window).
// Called by the whole block; ends with the staged samples visible to it.
__device__ void stage_windows(const line::Dev& L, const float* __restrict__ S, double zr,
                              double eps, float* __restrict__ sw, int* __restrict__ klo,
                              int* __restrict__ khi) {
    using namespace line;
    for (int n = threadIdx.x; n < L.N; n += blockDim.x) {
        const double t = arrival(L, elem_x(L, n), zr);
        const long k0 = (long)floor(__dmul_rn(__dsub_rn(t, eps), L.fs)) - 1;
        const int span = (int)ceil(2.0 * eps * L.fs) + 4;
        long first = 1, last = 0;
        for (int j = 0; j <= span; ++j) {
            const long k = k0 + j;
            if (k < 0 || k >= L.S) continue;
            if (fabs(__dsub_rn(__ddiv_rn((double)k, L.fs), t)) <= eps) {
                if (first > last) first = k;
                last = k;
            }
        }
        klo[n] = (int)first;  // an empty window has klo > khi
        khi[n] = (int)last;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < L.N * kStage; q += blockDim.x) {
        const int n = q / kStage, j = q % kStage;
        const int k = klo[n] - 2 + j;
        sw[n * kStride + j] = (k >= klo[n] && k <= khi[n]) ? __ldg(S + (size_t)n * L.S + k) : 0.f;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(32 * line::kSweepWarps) line_sweep_kernel(
    line::Dev L, LineTab T, const float* __restrict__ rf, const float* __restrict__ lines,
    int r_first, int n_scat, double eps, float* __restrict__ theta, float* __restrict__ e_loc,
    float* __restrict__ e_glob) {
    using namespace line;
    extern __shared__ float sm[];
    const int N = L.N, D = L.D;
    float* sw = sm;                              // [N][kStride] windowed channels
    float* g = sw + N * kStride;                 // [D] DAS line of r
    float* b = g + D;                            // [D] own-curve line of r
    float* abufs = b + D;                        // [kSweepWarps][D]
    int* klo = (int*)(abufs + kSweepWarps * D);  // [N]
    int* khi = klo + N;                          // [N]
    __shared__ double s_gg;
    __shared__ int s_wlo, s_whi;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rs = blockIdx.x, r = r_first + rs;
    const double zr = depth(L, r);
    const float* S = rf + (size_t)rs * N * L.S;

    stage_windows(L, S, zr, eps, sw, klo, khi);
    if (threadIdx.x == 0) {
        s_gg = 0.0;
        // local points: |z_i - z_r| <= c eps / 2
        const double half = __dmul_rn(L.c, eps) / 2.0;
        int wl = r, wh = r;
        while (wl > 0 && fabs(__dsub_rn(depth(L, wl - 1), zr)) <= half) --wl;
        while (wh < D - 1 && fabs(__dsub_rn(depth(L, wh + 1), zr)) <= half) ++wh;
        s_wlo = wl;
        s_whi = wh;
    }
    __syncthreads();
    double gg = 0.0;
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const float v = lines[(size_t)rs * D + i];
        g[i] = v;
        gg += (double)v * v;
    }
    for (int o = 16; o; o >>= 1) gg += __shfl_xor_sync(0xffffffffu, gg, o);
    if (lane == 0) atomicAdd(&s_gg, gg);
    // the scatterer's own curve (s = r) gives b
    if (warp == 0) {
        int lo, hi;
        sweep_curve(L, T, r, r, lane, sw, klo, khi, abufs, lo, hi);
        for (int i = lane; i < D; i += 32) b[i] = (i >= lo && i <= hi) ? abufs[i] : 0.f;
    }
    __syncthreads();
    const float g2f = (float)s_gg;
    const int wlo = s_wlo, whi = s_whi;
    float* abuf = abufs + warp * D;
    for (int s = warp; s < D; s += kSweepWarps) {
        int lo, hi;
        sweep_curve(L, T, r, s, lane, sw, klo, khi, abuf, lo, hi);
        // FP32 sums (at most n_depths terms); FP64 only for the final
        // scalars, on one lane -- the FP64 unit is narrow on this part
        float ab = 0.f, aa = 0.f, ag = 0.f;
        for (int i = lo + lane; i <= hi; i += 32) {
            const float a = abuf[i];
            ab += a * b[i];
            aa += a * a;
            ag += a * g[i];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ab += __shfl_xor_sync(0xffffffffu, ab, o);
            aa += __shfl_xor_sync(0xffffffffu, aa, o);
            ag += __shfl_xor_sync(0xffffffffu, ag, o);
        }
        if (lane == 0) {
            // a warp instruction on the FP64 unit costs about as much with one
            // active lane as with 32, so the per-curve scalars stay in FP32
            const float th = aa > 0.f ? ab / aa : 0.f;
            float num = 0.f, den = 0.f;
            for (int i = wlo; i <= whi; ++i) {
                const float a = (i >= lo && i <= hi) ? abuf[i] : 0.f;
                const float d = th * a - g[i];
                num += d * d;
                den += g[i] * g[i];
            }
            const size_t o = (size_t)s * n_scat + rs;
            theta[o] = th;
            e_loc[o] = den > 0.f ? num / den : 0.f;
            e_glob[o] = g2f > 0.f ? (th * th * aa - 2.f * th * ag + g2f) / g2f : 0.f;
        }
        __syncwarp();
    }
}

// Fixed-curve lines of one delay curve s for every scatterer (Eq. (2.8)),
// each scaled by its theta (Eq. (2.12)): out[rs][i] = theta a_s[i].  Block per
// scatterer; warp 0 builds b (its own curve), warp 1 a_s, then warp 0 scales.
__global__ void __launch_bounds__(64) line_fixed_kernel(line::Dev L, LineTab T,
                                                        const float* __restrict__ rf, int r_first,
                                                        int s, double eps,
                                                        float* __restrict__ out) {
    using namespace line;
    extern __shared__ float sm[];
    const int N = L.N, D = L.D;
    float* sw = sm;                              // [N][kStride]
    float* abufs = sw + N * kStride;             // [2][D]: b, a_s
    int* klo = (int*)(abufs + 2 * D);
    int* khi = klo + N;
    __shared__ int s_rng[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rs = blockIdx.x, r = r_first + rs;
    stage_windows(L, rf + (size_t)rs * N * L.S, depth(L, r), eps, sw, klo, khi);
    {
        int lo, hi;
        sweep_curve(L, T, r, warp == 0 ? r : s, lane, sw, klo, khi, abufs + warp * D, lo, hi);
        if (lane == 0) {
            s_rng[2 * warp] = lo;
            s_rng[2 * warp + 1] = hi;
        }
    }
    __syncthreads();
    if (warp == 0) {
        const int blo = s_rng[0], bhi = s_rng[1], alo = s_rng[2], ahi = s_rng[3];
        const float* b = abufs;
        const float* a = abufs + D;
        float ab = 0.f, aa = 0.f;
        for (int i = alo + lane; i <= ahi; i += 32) {
            const float bi = (i >= blo && i <= bhi) ? b[i] : 0.f;
            ab += a[i] * bi;
            aa += a[i] * a[i];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ab += __shfl_xor_sync(0xffffffffu, ab, o);
            aa += __shfl_xor_sync(0xffffffffu, aa, o);
        }
        const float th = aa > 0.f ? ab / aa : 0.f;
        for (int i = lane; i < D; i += 32)
            out[(size_t)rs * D + i] = (i >= alo && i <= ahi) ? th * a[i] : 0.f;
    }
}

// ------------------------------------------------------- line reconstruction
// Channel data of a line of scatterers from the unit-scatterer data (Eq. (2.1)
// is linear in the reflectivity): out[n][k] = sum_r amps[r] rf[r][n][k], in
// the order of r; zero amplitudes are skipped.
__global__ void __launch_bounds__(256) line_combine_kernel(int n_scat, size_t row_len,
                                                           const float* __restrict__ rf,
                                                           const float* __restrict__ amps,
                                                           float* __restrict__ out) {
    extern __shared__ int s_nz[];  // indices of the non-zero amplitudes, in order
    __shared__ int s_cnt;
    if (threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < n_scat; ++r)
            if (amps[r] != 0.f) s_nz[c++] = r;
        s_cnt = c;
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < row_len;
         q += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int j = 0; j < cnt; ++j) acc += amps[s_nz[j]] * __ldg(rf + (size_t)s_nz[j] * row_len + q);
        out[q] = acc;
    }
}

// Eq. (2.13): L_i = theta_i sum_{n in aperture(z_s)} S~^(i)_n at (2 z_i / c -
// D_n(z_s)) fs, S~^(i) the samples within eps of point i's echo arrival.
// Warp per line point, lanes over elements; positions and window decisions
// in FP64, taps and sums in FP32.
__global__ void __launch_bounds__(256) line_model_kernel(line::Dev L, const float* __restrict__ S,
                                                         int s, const float* __restrict__ theta,
                                                         double eps, float* __restrict__ out) {
    using namespace line;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + warp;
    if (i >= L.D) return;
    const double zi = depth(L, i), zs = depth(L, s);
    float acc = 0.f;
    for (int n = lane; n < L.N; n += 32) {
        const double xn = elem_x(L, n);
        if (!rx_active(L, xn, zs)) continue;
        const double u = __dmul_rn(__dsub_rn(__ddiv_rn(__dmul_rn(2.0, zi), L.c), delay(L, xn, zs)), L.fs);
        const double t_i = arrival(L, xn, zi);
        const double fl = floor(u);
        const int idx = (int)fl;
        const float* row = S + (size_t)n * L.S;
        acc += interp(L.interp, idx, (float)(u - fl), [&](int k) {
            if (k < 0 || k >= L.S) return 0.f;
            return fabs(__dsub_rn(__ddiv_rn((double)k, L.fs), t_i)) <= eps ? __ldg(row + k) : 0.f;
        });
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = theta[i] * acc;
}

// |analytic signal| of each row x[j] (length n): the DFT, negative
// frequencies removed and positive ones doubled, the inverse DFT, its
// modulus.  O(n^2) per row, phases reduced exactly as (j k mod n) / n.
__global__ void __launch_bounds__(256) line_envelope_kernel(int n, const float* __restrict__ x,
                                                            float* __restrict__ env) {
    extern __shared__ float sm[];
    float* xs = sm;           // [n]
    float2* X = (float2*)(sm + ((n + 1) & ~1));  // [n]
    const float* xr = x + (size_t)blockIdx.x * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) xs[j] = xr[j];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int j = 0; j < n; ++j) {
            const int q = (int)(((long long)j * k) % n);
            float sn, cs;
            sincospif(2.f * (float)q / (float)n, &sn, &cs);
            re += xs[j] * cs;
            im -= xs[j] * sn;
        }
        const float h = (k == 0 || 2 * k == n) ? 1.f : (2 * k < n ? 2.f : 0.f);
        X[k] = make_float2(h * re, h * im);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int k = 0; k < n; ++k) {
            const int q = (int)(((long long)j * k) % n);
            float sn, cs;
            sincospif(2.f * (float)q / (float)n, &sn, &cs);
            re += X[k].x * cs - X[k].y * sn;
            im += X[k].x * sn + X[k].y * cs;
        }
        env[(size_t)blockIdx.x * n + j] = sqrtf(re * re + im * im) / (float)n;
    }
}

// ------------------------------------------------------------------ launch
static line::Dev line_dev(const tidas_line_params& p) {
    line::Dev L;
    L.N = p.n_elem;
    L.S = p.n_samples;
    L.D = p.n_depths;
    L.interp = p.interp;
    L.pitch = p.pitch;
    L.f0 = p.f0;
    L.fs = p.fs;
    L.c = p.c;
    L.z_first = p.z_first;
    L.z_last = p.z_last;
    L.z_focus = p.z_focus;
    L.kossoff = p.kossoff;
    L.fnum = p.fnum_rx;
    // the pulse of Eq. (2.1): envelope 6 dB down at f0 (1 +- B / 2), cut at -60 dB
    const double half_bw = 0.5 * p.frac_bw * p.f0;
    const double pi = 3.14159265358979323846;
    L.alpha = pi * pi * half_bw * half_bw / log(pow(10.0, 6.0 / 20.0));
    L.thalf = sqrt(log(pow(10.0, 60.0 / 20.0)) / L.alpha);
    L.du = (float)(2.0 * p.fs * (p.z_last - p.z_first) / ((double)(p.n_depths - 1) * p.c));
    L.u0 = (float)(2.0 * p.z_first / p.c * p.fs);
    return L;
}

double line_window(const tidas_line_params& p) { return sqrt(log(2.0) / line_dev(p).alpha); }

int validate_line(const tidas_line_params* p) {
    TIDAS_REQUIRE(p, "line: null parameters");
    TIDAS_REQUIRE(p->n_elem >= 1 && p->n_elem <= 1024, "line: need 1 <= n_elem <= 1024");
    TIDAS_REQUIRE(p->n_samples >= 8 && p->n_samples <= (1 << 20), "line: bad n_samples");
    TIDAS_REQUIRE(p->n_depths >= 2 && p->n_depths <= 8192, "line: need 2 <= n_depths <= 8192");
    TIDAS_REQUIRE(p->pitch > 0 && p->f0 > 0 && p->fs > 0 && p->c > 0 && p->frac_bw > 0,
                  "line: pitch, f0, fs, c and frac_bw must be positive");
    TIDAS_REQUIRE(p->z_first > 0 && p->z_last > p->z_first && p->z_focus > 0,
                  "line: need 0 < z_first < z_last and z_focus > 0");
    TIDAS_REQUIRE(p->kossoff > 0 && p->fnum_rx > 0, "line: kossoff and fnum_rx must be positive");
    TIDAS_REQUIRE(p->interp == TIDAS_INTERP_LINEAR || p->interp == TIDAS_INTERP_CUBIC,
                  "line: bad interp");
    return TIDAS_OK;
}

int launch_line_synth(const tidas_line_params& p, int r_first, int n_scat, float* rf,
                      cudaStream_t st) {
    const line::Dev L = line_dev(p);
    line_synth_kernel<<<dim3((L.N + kSynthRows - 1) / kSynthRows, n_scat), 256, 0, st>>>(
        L, r_first, rf);
    return check_launch("line_synth_kernel");
}

static size_t table_bytes(const line::Dev& L) {
    const size_t dn = (size_t)L.D * L.N;
    return dn * 4 * 2 + (size_t)L.D * 8 + dn * 4 * 2 + dn + 1024;
}
static LineTab carve(const line::Dev& L, void* ws) {
    const size_t dn = (size_t)L.D * L.N;
    char* p = (char*)ws;
    LineTab T;
    T.das_idx = (int*)p;
    p += dn * 4;
    T.das_frac = (float*)p;
    p += dn * 4;
    T.v_idx = (int*)p;
    p += dn * 4;
    T.v_frac = (float*)p;
    p += dn * 4;
    T.u_idx = (int*)p;
    p += (size_t)L.D * 4;
    T.u_frac = (float*)p;
    p += (size_t)L.D * 4;
    T.act = (uint8_t*)p;
    return T;
}

int launch_line_das(const tidas_line_params& p, const float* rf, int n_scat, float* lines,
                    cudaStream_t st) {
    const line::Dev L = line_dev(p);
    void* ws = nullptr;
    TIDAS_CUDA(cudaMallocAsync(&ws, table_bytes(L), st));
    const LineTab T = carve(L, ws);
    line_table_kernel<<<(L.D * L.N + 255) / 256, 256, 0, st>>>(L, T);
    int rc = check_launch("line_table_kernel");
    if (rc == TIDAS_OK) {
        line_das_kernel<<<dim3((L.D + 31) / 32, n_scat), 256, 0, st>>>(L, T, rf, lines);
        rc = check_launch("line_das_kernel");
    }
    cudaFreeAsync(ws, st);
    return rc;
}

int launch_line_sweep(const tidas_line_params& p, const float* rf, const float* lines,
                      int r_first, int n_scat, double eps, float* theta, float* e_loc,
                      float* e_glob, cudaStream_t st) {
    const line::Dev L = line_dev(p);
    if (2.0 * eps * L.fs + 1.0 > line::kStage - 5)
        return set_error(TIDAS_ERR_UNSUPPORTED,
                         "line sweep: the window (2 eps fs + 1 samples) must stay below %d",
                         line::kStage - 5);
    const size_t smem = sizeof(float) * ((size_t)L.N * line::kStride + (size_t)L.D * (2 + line::kSweepWarps)) +
                        sizeof(int) * 2 * (size_t)L.N;
    if (smem > 220 * 1024)
        return set_error(TIDAS_ERR_UNSUPPORTED, "line sweep: %d depths x %d elements do not fit",
                         L.D, L.N);
    void* ws = nullptr;
    TIDAS_CUDA(cudaMallocAsync(&ws, table_bytes(L), st));
    const LineTab T = carve(L, ws);
    line_table_kernel<<<(L.D * L.N + 255) / 256, 256, 0, st>>>(L, T);
    int rc = check_launch("line_table_kernel");
    if (rc == TIDAS_OK) {
        rc = check_cuda(cudaFuncSetAttribute(line_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem),
                        "cudaFuncSetAttribute(line_sweep_kernel)");
    }
    if (rc == TIDAS_OK) {
        line_sweep_kernel<<<n_scat, 32 * line::kSweepWarps, smem, st>>>(
            L, T, rf, lines, r_first, n_scat, eps, theta, e_loc, e_glob);
        rc = check_launch("line_sweep_kernel");
    }
    cudaFreeAsync(ws, st);
    return rc;
}

}  // namespace tidas

namespace tidas {
int launch_line_combine(const tidas_line_params& p, const float* rf, int n_scat, const float* amps,
                        float* out, cudaStream_t st) {
    const size_t row_len = (size_t)p.n_elem * p.n_samples;
    const int grid = (int)std::min<size_t>((row_len + 255) / 256, (size_t)152 * 8);
    line_combine_kernel<<<grid, 256, sizeof(int) * (size_t)n_scat, st>>>(n_scat, row_len, rf, amps,
                                                                        out);
    return check_launch("line_combine_kernel");
}

int launch_line_model(const tidas_line_params& p, const float* S, int s, const float* theta,
                      double eps, float* out, cudaStream_t st) {
    const line::Dev L = line_dev(p);
    line_model_kernel<<<(L.D + 7) / 8, 256, 0, st>>>(L, S, s, theta, eps, out);
    return check_launch("line_model_kernel");
}

int launch_line_envelope(int n_rows, int n, const float* x, float* env, cudaStream_t st) {
    const size_t smem = sizeof(float) * (((size_t)n + 1) & ~(size_t)1) + sizeof(float2) * (size_t)n;
    if (smem > 220 * 1024)
        return set_error(TIDAS_ERR_UNSUPPORTED, "line envelope: rows of %d points do not fit", n);
    TIDAS_CUDA(cudaFuncSetAttribute(line_envelope_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem));
    line_envelope_kernel<<<n_rows, 256, smem, st>>>(n, x, env);
    return check_launch("line_envelope_kernel");
}
}  // namespace tidas

namespace tidas {
int launch_line_fixed(const tidas_line_params& p, const float* rf, int r_first, int n_scat, int s,
                      double eps, float* out, cudaStream_t st) {
    const line::Dev L = line_dev(p);
    if (2.0 * eps * L.fs + 1.0 > line::kStage - 5)
        return set_error(TIDAS_ERR_UNSUPPORTED,
                         "line fixed: the window (2 eps fs + 1 samples) must stay below %d",
                         line::kStage - 5);
    const size_t smem = sizeof(float) * ((size_t)L.N * line::kStride + 2 * (size_t)L.D) +
                        sizeof(int) * 2 * (size_t)L.N;
    if (smem > 220 * 1024)
        return set_error(TIDAS_ERR_UNSUPPORTED, "line fixed: %d depths x %d elements do not fit",
                         L.D, L.N);
    void* ws = nullptr;
    TIDAS_CUDA(cudaMallocAsync(&ws, table_bytes(L), st));
    const LineTab T = carve(L, ws);
    line_table_kernel<<<(L.D * L.N + 255) / 256, 256, 0, st>>>(L, T);
    int rc = check_launch("line_table_kernel");
    if (rc == TIDAS_OK) {
        rc = check_cuda(cudaFuncSetAttribute(line_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem),
                        "cudaFuncSetAttribute(line_fixed_kernel)");
    }
    if (rc == TIDAS_OK) {
        line_fixed_kernel<<<n_scat, 64, smem, st>>>(L, T, rf, r_first, s, eps, out);
        rc = check_launch("line_fixed_kernel");
    }
    cudaFreeAsync(ws, st);
    return rc;
}
}  // namespace tidas
