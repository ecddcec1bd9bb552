// Shared host/device helpers of the sm_103a DAS / tiDAS library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "tidas.h"

// ---------------------------------------------------------------- errors
namespace tidas {

int set_error(int code, const char* fmt, ...);
int check_launch(const char* what);
int check_cuda(cudaError_t e, const char* what);

#define TIDAS_REQUIRE(cond, ...)                                   \
    do {                                                           \
        if (!(cond)) return ::tidas::set_error(TIDAS_ERR_ARG, __VA_ARGS__); \
    } while (0)

#define TIDAS_CUDA(call)                                           \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::tidas::check_cuda(e_, #call); \
    } while (0)

// ------------------------------------------------------- plan (device view)
constexpr int kMaxAngles = 16;
constexpr int kJ = 40;  // pulse tap tables cover j = -kJ..kJ (needs half support < kJ - 1)

// Everything a DAS-family kernel needs, passed by value.
struct DasDev {
    int n_elem, n_angles, n_samples, nx, nz, interp, rf_dtype;
    float fnum;          // <= 0: whole array, unit weights
    float thalf;         // pulse half support, samples
    float beta;          // pulse envelope exp(-beta t^2), t in samples
    float wcar;          // carrier 2 f0 / fs: cos(pi * wcar * t), t in samples
    // transmit split: u_tx(ix, iz, a) = (bxi + bzi) + (bxf + bzf)   [samples]
    const int* bxi;      // [A][nx]
    const float* bxf;    // [A][nx]
    const int* bzi;      // [A][nz]
    const float* bzf;    // [A][nz]
    const float* dxs;    // [n_elem][nx]  (x_ix - x_n) * fs / c
    const float* zs;     // [nz]          z_iz * fs / c
    const float* xs;     // [nx]          x_ix * fs / c (grid-free element range search)
    float elem0_s;       // x_0 * fs / c
    float pitch_s;       // pitch * fs / c
    const float* ptab;   // [3][2 kJ + 1]: exp(-beta j^2), cos(pi wcar j), sin(pi wcar j)
    const float2* carr;  // carr[k] = e^{i pi wcar k}, valid for k = -kJ .. n_samples + kJ - 1
};

// Host-side plan object.
struct Plan {
    das_params p;
    double angles[kMaxAngles];
    double sn[kMaxAngles], cs[kMaxAngles];
    DasDev dev;
    void* blob;             // single device allocation holding every table
    const double* d_sncs;   // device [A][2]: sin, cos of each angle (host libm values)
    bool taps_in_range;     // every interpolation tap of every pixel lies in [0, n_samples)
    int read_first = 0;     // samples [read_first, read_first + read_count) hold every
    int read_count = 0;     // tap that any pixel weights (das_plan_read_window)
    double thalf_samples, beta_samples, wcar;
    // tensor-core DAS of FP16 plans: per-(tile, angle, element) sample windows
    int* tc_tab = nullptr;
    int2* tc_range = nullptr;
    uint8_t* tc_rounds = nullptr;  // per tile: its rounds of one or two pairs
    int tc_tiles_x = 0, tc_tiles = 0;
    bool tc_ok = false;     // every window fits the 64-sample operand tile
    int tc_mode = 1;        // 0: CUDA cores only, 1: tensor cores for >= 16 FP16 frames
    // staging buffer of the repacked channel data (tensor-core DAS), grown on demand
    mutable void* tc_ws = nullptr;
    mutable size_t tc_ws_bytes = 0;
    // layout the staging buffer was last filled in (0: unknown contents)
    mutable long long tc_ws_layout = 0;
    mutable std::mutex tc_ws_mutex;
};

// ---------------------------------------------------------- device helpers
// Receive correction in samples: sqrt(dx^2 + z^2) - z written without
// cancellation, dx^2 / (sqrt(dx^2 + z^2) + z).
__device__ __forceinline__ float rx_excess(float dxs, float zs) {
    float d2 = dxs * dxs;
    float s = sqrtf(fmaf(zs, zs, d2));
    return __fdiv_rn(d2, s + zs);
}

// Hann receive apodization cos^2(pi r), r = (x - x_n) F# / z, |r| <= 1/2.
__device__ __forceinline__ float apod_weight(float dxs, float zs, float fnum) {
    if (fnum <= 0.f) return 1.f;
    float r = dxs * fnum / zs;
    if (fabsf(r) > 0.5f) return 0.f;
    float cw = cospif(r);
    return cw * cw;
}

// Two single-precision FMAs / products in one packed instruction (sm_100
// f32x2): each half is rounded exactly as the scalar fmaf / multiply.
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Keys (a = -0.5) weights of samples i-1, i, i+1, i+2 at fraction phi.
__device__ __forceinline__ void keys_weights(float phi, float& w0, float& w1, float& w2,
                                             float& w3) {
    float p2 = phi * phi;
    float p3 = p2 * phi;
    w0 = fmaf(-0.5f, p3, fmaf(1.0f, p2, -0.5f * phi));
    w1 = fmaf(1.5f, p3, fmaf(-2.5f, p2, 1.0f));
    w2 = fmaf(-1.5f, p3, fmaf(2.0f, p2, 0.5f * phi));
    w3 = fmaf(0.5f, p3, -0.5f * p2);
}

// Split delay of pixel (ix, iz) for angle a and element n:
// integer sample i and fraction phi in [0, 1).
__device__ __forceinline__ void pixel_delay(const DasDev& d, int a, int ix, int iz, float excess,
                                            int& i, float& phi) {
    int bi = __ldg(d.bxi + a * d.nx + ix) + __ldg(d.bzi + a * d.nz + iz);
    float bf = __ldg(d.bxf + a * d.nx + ix) + __ldg(d.bzf + a * d.nz + iz);
    float uf = bf + excess;
    float fl = floorf(uf);
    phi = uf - fl;
    i = bi + (int)fl;
}

__device__ __forceinline__ float load_rf(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_rf(const __half* p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ void store_rf(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_rf(__half* p, float v) { *p = __float2half_rn(v); }

}  // namespace tidas

// launchers implemented in the .cu files
namespace tidas {
int launch_delay_table(const Plan& P, int angle, int32_t* idx, float* frac, cudaStream_t st);
int launch_das_forward(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st);
int launch_das_tc(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st);
int launch_das_coeff(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st);
// The plan's staging buffer, at least `need` bytes.  *fresh tells whether
// its previous contents were written in another `layout` (or none).
int plan_staging(const Plan& P, size_t need, void** out, long long layout, bool* fresh);
int das_tc_prepare(Plan& P);
int launch_das_adjoint(const Plan& P, const float* img, float* rf, int nf, cudaStream_t st);
int launch_synthesize(const Plan& P, const double* pos, const float* amp, int n_scat, int nf,
                      void* rf, cudaStream_t st);
int launch_synthesize_grid(const Plan& P, const float* refl, float* rf, int nf, cudaStream_t st);
int launch_synthesize_adjoint(const Plan& P, const float* rf, float* refl, int nf,
                              cudaStream_t st);
int launch_fit_kernels(const Plan& P, int taps, int ref_stride, float* kernels, float* theta,
                       cudaStream_t st);
int launch_tidas(const float* kernels, int taps, int center, bool flip, int nz, int nx,
                 const void* in, float* out, int nf, int variant, cudaStream_t st);
}  // namespace tidas
