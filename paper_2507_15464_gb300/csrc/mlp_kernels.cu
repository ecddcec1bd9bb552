// Learned tiDAS kernel generator: exact PSF training targets, a tcgen05 BF16
// GEMM with fused bias / ReLU epilogue, and the small kernels of MLP
// training (Adam on FP32 master weights, ReLU backward, bias gradients,
// transposes, mean-squared error) and inference (feature encoding, kernel
// fallback and scaling).
#include <atomic>

#include "common.cuh"
#include "sm103_primitives.cuh"

namespace tidas {
using namespace sm103;

// wait flag of the GEMM below (read by tidas_mlp_status)
__device__ int g_mlp_wait_error = 0;

// ------------------------------------------------------------ BF16 GEMM
// C[M x N] = act(A[M x K] * B[N x K]^T + bias[N]); A, B BF16 row-major with K
// contiguous (K % 64 == 0), FP32 accumulation in tensor memory.  One CTA per
// 128-row x BN-column tile (BN <= 256, multiple of 16); K streamed by TMA in
// 64-column chunks through a 4-stage ring; warp 0 lane 0 loads, warp 1 lane 0
// issues MMAs, all four warps run the epilogue (bias, ReLU, FP32 and/or BF16
// stores).
namespace mg {
constexpr int kM = 128;
constexpr int kKC = 64;
constexpr int kStages = 4;
constexpr int kABytes = kM * kKC * 2;  // 16 KB
constexpr int kMaxBN = 256;
constexpr int kBBytes = kMaxBN * kKC * 2;  // 32 KB (max)
constexpr size_t kSmem = 1024 + (size_t)kStages * (kABytes + kBBytes) + 256;
}  // namespace mg

// skip_loads (failure-path tests only): the producer issues no copies, so the
// MMA thread's first wait runs out after wait_ns with nothing in flight,
// records code 202 and the CTA returns without writing its tile.
__global__ void __launch_bounds__(128, 1)
    mlp_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                    int M, int N, int K, int BN, const float* __restrict__ bias, int relu,
                    float* __restrict__ c32, __nv_bfloat16* __restrict__ c16, int ldc,
                    int skip_loads, unsigned long long wait_ns) {
    using namespace mg;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_align1024(smem_raw);
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kABytes;
    uint64_t* full = (uint64_t*)(sB + kStages * kBBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kM, n0 = blockIdx.y * BN;
    const int nk = K / kKC;
    const uint32_t tcols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    const uint32_t idesc = idesc_bf16_f32(kM, BN);
    const uint32_t tx = (uint32_t)(kABytes + BN * kKC * 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        fence_barrier_init();
        prefetch_tensormap(&ta);
        prefetch_tensormap(&tb);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0 && !skip_loads) {
        uint32_t st = 0, ph = 0;
        for (int kc = 0; kc < nk; ++kc) {
            if (!mbar_wait(&empty[st], ph ^ 1, &g_mlp_wait_error, 201, wait_ns)) {
                *s_abort = 1;
                break;
            }
            mbar_arrive_expect_tx(&full[st], tx);
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(sA + st * kABytes)),
                "l"(reinterpret_cast<uint64_t>(&ta)), "r"(kc * kKC), "r"(m0),
                "r"(smem_u32(&full[st]))
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(sB + st * kBBytes)),
                "l"(reinterpret_cast<uint64_t>(&tb)), "r"(kc * kKC), "r"(n0),
                "r"(smem_u32(&full[st]))
                : "memory");
            if (++st == kStages) { st = 0; ph ^= 1; }
        }
    } else if (warp == 1 && lane == 0) {
        uint32_t st = 0, ph = 0;
        for (int kc = 0; kc < nk; ++kc) {
            if (*s_abort || !mbar_wait(&full[st], ph, &g_mlp_wait_error, 202, wait_ns)) {
                *s_abort = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(sA + st * kABytes), b = smem_u32(sB + st * kBBytes);
#pragma unroll
            for (int kk = 0; kk < kKC / 16; ++kk)
                mma_f16(tmem, desc_sw128_kmajor(a) + 2 * kk, desc_sw128_kmajor(b) + 2 * kk, idesc,
                        (kc > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&empty[st]);
            if (++st == kStages) { st = 0; ph ^= 1; }
        }
        mma_commit(done);
    }
    __syncwarp();
    if (!mbar_wait(done, 0, &g_mlp_wait_error, 203, wait_ns)) *s_abort = 1;
    tc_fence_after();
    if (!*s_abort) {
        const int row = m0 + warp * 32 + lane;
        for (int j = 0; j < BN; j += 32) {
            uint32_t r[32];
            tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j, r);
            tmem_ld_wait();
            if (row < M) {
#pragma unroll
                for (int v = 0; v < 32; v += 8) {
                    const int col = n0 + j + v;
                    if (col >= N || j + v >= BN) break;
                    float o[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        float x = __uint_as_float(r[v + e]);
                        if (bias) x += __ldg(bias + col + e);
                        if (relu) x = fmaxf(x, 0.f);
                        o[e] = x;
                    }
                    if (c32) {
                        float4* d = reinterpret_cast<float4*>(c32 + (size_t)row * ldc + col);
                        d[0] = make_float4(o[0], o[1], o[2], o[3]);
                        d[1] = make_float4(o[4], o[5], o[6], o[7]);
                    }
                    if (c16) {
                        __nv_bfloat162 p[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) p[e] = __floats2bfloat162_rn(o[2 * e], o[2 * e + 1]);
                        *reinterpret_cast<uint4*>(c16 + (size_t)row * ldc + col) =
                            *reinterpret_cast<uint4*>(p);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// read and clear the bounded-wait flag of the GEMM above (see tidas_device_status)
int read_clear_mlp_wait_flag(int* v) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_mlp_wait_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_mlp_wait_error, &zero, sizeof(int));
    return check_cuda(e, "mlp wait flag");
}

int make_map_2d_bf16(CUtensorMap* map, const void* ptr, int rows, int cols, int box_rows);

// Failure-path test hooks of the GEMM (tidas_set_debug_option), read by the
// host when it launches the kernel.
static std::atomic<int> g_dbg_skip_loads{0};
static std::atomic<unsigned long long> g_dbg_wait_ns{1000000000ull};

int launch_mlp_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K,
                    const float* bias, int relu, float* c32, __nv_bfloat16* c16, int ldc,
                    cudaStream_t st) {
    using namespace mg;
    const int BN = N <= kMaxBN ? N : kMaxBN;
    CUtensorMap ta, tb;
    int rc = make_map_2d_bf16(&ta, A, M, K, kM);
    if (rc) return rc;
    rc = make_map_2d_bf16(&tb, B, N, K, BN);
    if (rc) return rc;
    TIDAS_CUDA(cudaFuncSetAttribute(mlp_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    dim3 grid((M + kM - 1) / kM, (N + BN - 1) / BN);
    mlp_gemm_kernel<<<grid, 128, kSmem, st>>>(ta, tb, M, N, K, BN, bias, relu, c32, c16, ldc,
                                              g_dbg_skip_loads.load(), g_dbg_wait_ns.load());
    return check_launch("mlp_gemm_kernel");
}

// ------------------------------------------------------- small kernels
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int rows, int cols,
                                      __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k;
        t[k][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * cols + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    const int oc = r0 + threadIdx.x, orow0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int orow = orow0 + k;
        if (orow < cols && oc < rows) out[(size_t)orow * rows + oc] = t[threadIdx.x][k];
    }
}

// dpre = dpost * (pre > 0) (pre = 0 marks ReLU inputs that were clipped: the
// stored activation is post-ReLU, so act > 0 <=> pre > 0); writes BF16 copy
// and its transpose is done separately.
__global__ void relu_backward_kernel(const float* __restrict__ dpost, const float* __restrict__ act,
                                     long long n, float* __restrict__ dpre32,
                                     __nv_bfloat16* __restrict__ dpre16) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float g = (act == nullptr || act[i] > 0.f) ? dpost[i] : 0.f;
        if (dpre32) dpre32[i] = g;
        dpre16[i] = __float2bfloat16_rn(g);
    }
}

// dst[i] = src[idx[i]] for rows of `words` 32-bit words (mini-batch gather)
__global__ void gather_rows_kernel(const uint32_t* __restrict__ src, const int32_t* __restrict__ idx,
                                   long long n, int words, uint32_t* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (i >= n) return;
    const uint32_t* s = src + (long long)idx[i] * words;
    uint32_t* d = dst + i * words;
    for (int w = threadIdx.x; w < words; w += blockDim.x) d[w] = s[w];
}

// db[j] = sum_i d[i][j]
__global__ void colsum_kernel(const float* __restrict__ d, int rows, int cols, int ld,
                              float* __restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; ++i) s += d[(size_t)i * ld + j];
    db[j] = s;
}

// AdamW on FP32 master weights; refreshes the BF16 copy (and, when given, its
// transpose; the tensor is rows x cols).
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int rows, int cols, float lr, float b1,
                            float b2, float eps, float wd, float bc1, float bc2,
                            __nv_bfloat16* __restrict__ w16, __nv_bfloat16* __restrict__ w16t) {
    const long long n = (long long)rows * cols;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float wi = w[i] * (1.f - lr * wd);
        wi -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        const __nv_bfloat16 h = __float2bfloat16_rn(wi);
        if (w16) w16[i] = h;
        if (w16t) w16t[(i % cols) * rows + i / cols] = h;
    }
}

// mean squared error over the first `cols_used` columns; grad = 2 (p - t) / (rows * cols_used)
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ target,
                           int rows, int cols_used, int ldp, int ldt, float* __restrict__ dpred,
                           double* __restrict__ partial) {
    double s = 0.0;
    const long long n = (long long)rows * ldp;
    const float scale = 2.f / ((float)rows * (float)cols_used);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / ldp), c = (int)(i % ldp);
        float d = 0.f;
        if (c < cols_used) {
            d = pred[i] - target[(size_t)r * ldt + c];
            s += (double)d * d;
        }
        dpred[i] = scale * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        partial[blockIdx.x] = t;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ p, int np, double scale,
                                    double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += p[i];
        *out = s * scale;
    }
}

// features (x, z, fnum, angle) -> [-1, 1] inputs, BF16, padded to 64 columns
// Eight threads per row, one 16-byte chunk of 8 BF16 each (coalesced rows).
__global__ void encode_kernel(const double* __restrict__ samples, int n, const float* __restrict__ lo,
                              const float* __restrict__ hi, __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long i = t >> 3;
    const int c = (int)(t & 7);
    if (i >= n) return;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (c == 0) {
        float f[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            f[k] = 2.f * ((float)samples[i * 4 + k] - lo[k]) / (hi[k] - lo[k]) - 1.f;
        const __nv_bfloat162 a = __floats2bfloat162_rn(f[0], f[1]);
        const __nv_bfloat162 b = __floats2bfloat162_rn(f[2], f[3]);
        v.x = *reinterpret_cast<const uint32_t*>(&a);
        v.y = *reinterpret_cast<const uint32_t*>(&b);
    }
    reinterpret_cast<uint4*>(out + i * 64)[c] = v;
}

}  // namespace tidas

// ------------------------------------------------------------ PSF batch
// Exact single-scatterer DAS PSF rows (Section 2.2, Eq. (2.6)-(2.7)) for a
// batch of acquisitions: sample i = (x, z, F#, theta) places a unit scatterer
// at (x, z), transmits one plane wave at theta, beamforms with receive
// f-number F# and returns the row through the scatterer at lateral offsets
// (t - taps/2) dx.  Same evaluation as tidas_fit_kernels (FP64 delays, the
// plan's interpolation and pulse).  With `norm` given, the row is divided by
// the scatterer pixel's sum of apodization weights, which is written there.
namespace tidas {
struct PsfArgs {
    int n_elem, interp, n_samples, taps;
    double pitch, c, fs, t0, dx, dz;
    double thalf, beta, wcar;  // samples
};

__device__ __forceinline__ double psf_delay(const PsfArgs& A, double sn, double cs, int n, double x,
                                            double z) {
    double xn = __dmul_rn(__dsub_rn((double)n, 0.5 * (double)(A.n_elem - 1)), A.pitch);
    double ddx = __dsub_rn(x, xn);
    double tx = __dadd_rn(__dmul_rn(x, sn), __dmul_rn(z, cs));
    double rx = __dsqrt_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(z, z)));
    return __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tx, rx), A.c), A.t0), A.fs);
}

__device__ __forceinline__ double psf_pulse(const PsfArgs& A, double t) {
    if (fabs(t) > A.thalf) return 0.0;
    float tf = (float)t;
    return (double)(expf(-(float)A.beta * tf * tf) * cospif((float)A.wcar * tf));
}

__device__ __forceinline__ double psf_apod(const PsfArgs& A, int n, double x, double z, double fnum) {
    if (fnum <= 0) return 1.0;
    double xn = ((double)n - 0.5 * (double)(A.n_elem - 1)) * A.pitch;
    double r = (x - xn) * fnum / z;
    if (fabs(r) > 0.5) return 0.0;
    double cw = cospi(r);
    return cw * cw;
}

__global__ void psf_batch_kernel(PsfArgs A, const double* __restrict__ samples, int n,
                                 float* __restrict__ out, int ldo, float* __restrict__ norm) {
    const int i = blockIdx.x;
    const int t = threadIdx.x;
    if (i >= n) return;
    const double xs = samples[4 * i], z = samples[4 * i + 1], fnum = samples[4 * i + 2];
    const double th = samples[4 * i + 3];
    double sn, cs;
    sincos(th, &sn, &cs);
    double s = 0.0;
    for (int e = 0; e < A.n_elem; ++e) s += psf_apod(A, e, xs, z, fnum);
    if (t < A.taps) {
        const double xp = xs + (double)(t - A.taps / 2) * A.dx;
        double acc = 0.0;
        for (int e = 0; e < A.n_elem; ++e) {
            const double w = psf_apod(A, e, xp, z, fnum);
            if (w == 0.0) continue;
            const double up = psf_delay(A, sn, cs, e, xp, z);
            const double us = psf_delay(A, sn, cs, e, xs, z);
            const double fl = floor(up);
            const double phi = up - fl;
            const int ii = (int)fl;
            double v = 0.0;
            if (A.interp == TIDAS_INTERP_CUBIC) {
                float w0, w1, w2, w3;
                keys_weights((float)phi, w0, w1, w2, w3);
                const float wt[4] = {w0, w1, w2, w3};
                for (int k = 0; k < 4; ++k) {
                    const int m = ii - 1 + k;
                    if (m < 0 || m >= A.n_samples) continue;
                    v += (double)wt[k] * psf_pulse(A, (double)m - us);
                }
            } else {
                if (ii >= 0 && ii < A.n_samples) v += (1.0 - phi) * psf_pulse(A, (double)ii - us);
                if (ii + 1 >= 0 && ii + 1 < A.n_samples)
                    v += phi * psf_pulse(A, (double)(ii + 1) - us);
            }
            acc += w * v;
        }
        out[(size_t)i * ldo + t] = (float)(norm ? acc / s : acc);
    } else if (t < ldo) {
        out[(size_t)i * ldo + t] = 0.f;
    }
    if (norm && t == 0) norm[i] = (float)s;
}

// Band patches of the same PSFs: the image of the unit scatterer of sample i
// at rows z + (u - kz/2) dz and columns x + (t - taps/2) dx, written to
// out[i][u * ldk + t] (zeros in the padding t >= taps); row u = kz/2 is the
// row of psf_batch_kernel, evaluated by the same operations.  One block per
// sample, threads over the (u, t) pairs.
__global__ void psf_batch2d_kernel(PsfArgs A, const double* __restrict__ samples, int n, int kz,
                                   int ldk, float* __restrict__ out, int ldo,
                                   float* __restrict__ norm) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const double xs = samples[4 * i], z = samples[4 * i + 1], fnum = samples[4 * i + 2];
    const double th = samples[4 * i + 3];
    double sn, cs;
    sincos(th, &sn, &cs);
    double s = 0.0;
    for (int e = 0; e < A.n_elem; ++e) s += psf_apod(A, e, xs, z, fnum);
    for (int q = threadIdx.x; q < ldo; q += blockDim.x) {
        const int u = q / ldk, t = q - u * ldk;
        if (u >= kz || t >= A.taps) {
            out[(size_t)i * ldo + q] = 0.f;
            continue;
        }
        const double xp = xs + (double)(t - A.taps / 2) * A.dx;
        const double zp = z + (double)(u - kz / 2) * A.dz;
        double acc = 0.0;
        for (int e = 0; e < A.n_elem; ++e) {
            const double w = psf_apod(A, e, xp, zp, fnum);
            if (w == 0.0) continue;
            const double up = psf_delay(A, sn, cs, e, xp, zp);
            const double us = psf_delay(A, sn, cs, e, xs, z);
            const double fl = floor(up);
            const double phi = up - fl;
            const int ii = (int)fl;
            double v = 0.0;
            if (A.interp == TIDAS_INTERP_CUBIC) {
                float w0, w1, w2, w3;
                keys_weights((float)phi, w0, w1, w2, w3);
                const float wt[4] = {w0, w1, w2, w3};
                for (int k = 0; k < 4; ++k) {
                    const int m = ii - 1 + k;
                    if (m < 0 || m >= A.n_samples) continue;
                    v += (double)wt[k] * psf_pulse(A, (double)m - us);
                }
            } else {
                if (ii >= 0 && ii < A.n_samples) v += (1.0 - phi) * psf_pulse(A, (double)ii - us);
                if (ii + 1 >= 0 && ii + 1 < A.n_samples)
                    v += phi * psf_pulse(A, (double)(ii + 1) - us);
            }
            acc += w * v;
        }
        out[(size_t)i * ldo + q] = (float)(norm ? acc / s : acc);
    }
    if (norm && threadIdx.x == 0) norm[i] = (float)s;
}

// per-pixel NRMSE of learned vs exact kernels; where it exceeds `thresh` the
// exact kernel replaces the learned one in `out`
__global__ void kernel_fallback_kernel(const float* __restrict__ learned, int ldl,
                                       const float* __restrict__ exact, int lde, long long npix,
                                       int taps, float thresh, float* __restrict__ out, int ldo,
                                       float* __restrict__ nrmse) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double num = 0.0, den = 0.0;
    for (int t = 0; t < taps; ++t) {
        const double l = learned[p * ldl + t], e = exact[p * lde + t];
        num += (l - e) * (l - e);
        den += e * e;
    }
    const float r = den > 0 ? (float)sqrt(num / den) : 0.f;
    if (nrmse) nrmse[p] = r;
    const bool fb = r > thresh;
    for (int t = 0; t < taps; ++t) out[p * ldo + t] = fb ? exact[p * lde + t] : learned[p * ldl + t];
}

// rows of a per-sample table multiplied by a per-sample scale (kernel
// de-normalisation): out[i][t] = in[i][t] * s[i], t < cols
__global__ void row_scale_kernel(const float* __restrict__ in, int ldi, const float* __restrict__ s,
                                 long long rows, int cols, float* __restrict__ out, int ldo) {
    const long long i = (long long)blockIdx.x * blockDim.y + threadIdx.y;
    if (i >= rows) return;
    for (int t = threadIdx.x; t < cols; t += blockDim.x) out[i * ldo + t] = in[i * ldi + t] * s[i];
}

// sum of apodization weights at (x, z) for receive f-number F# (the kernel scale)
// FP32: the sum only rescales the network's kernels (relative error ~1e-6
// against FP64, far below the kernels' own error).
__global__ void apod_sum_kernel(PsfArgs A, const double* __restrict__ samples, long long n,
                                float* __restrict__ s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = (float)samples[4 * i], z = (float)samples[4 * i + 1];
    const float fnum = (float)samples[4 * i + 2];
    if (fnum <= 0.f) {
        s[i] = (float)A.n_elem;
        return;
    }
    const float pitch = (float)A.pitch, mid = 0.5f * (float)(A.n_elem - 1);
    const float k = fnum / z;
    // only the elements within the aperture half-width z / (2 F#), one
    // element of margin on each side; each one still passes the exact test
    const float half = 0.5f / fabsf(k);
    const float lo_f = floorf((x - half) / pitch + mid) - 1.f;
    const float hi_f = ceilf((x + half) / pitch + mid) + 1.f;
    const int e_lo = lo_f > 0.f ? (lo_f < (float)A.n_elem ? (int)lo_f : A.n_elem) : 0;
    const int e_hi = hi_f < (float)(A.n_elem - 1) ? (hi_f >= 0.f ? (int)hi_f : -1) : A.n_elem - 1;
    float acc = 0.f;
    for (int e = e_lo; e <= e_hi; ++e) {
        const float r = (x - ((float)e - mid) * pitch) * k;
        if (fabsf(r) <= 0.5f) {
            // fast cosine: absolute error about 5e-7 per weight
            const float cw = __cosf(3.14159265358979f * r);
            acc = fmaf(cw, cw, acc);
        }
    }
    s[i] = acc;
}

static PsfArgs psf_args(const Plan& P, int taps) {
    PsfArgs A;
    A.n_elem = P.p.n_elem;
    A.interp = P.p.interp;
    A.n_samples = P.p.n_samples;
    A.taps = taps;
    A.pitch = P.p.pitch;
    A.c = P.p.c;
    A.fs = P.p.fs;
    A.t0 = P.p.t0;
    A.dx = P.p.dx;
    A.dz = P.p.dz;
    A.thalf = P.thalf_samples;
    A.beta = P.beta_samples;
    A.wcar = P.wcar;
    return A;
}
}  // namespace tidas

using namespace tidas;

static inline cudaStream_t ST(void* s) { return (cudaStream_t)s; }
static int vblocks(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

extern "C" int tidas_psf_batch(das_plan plan, const double* samples, int32_t n, int32_t taps,
                               float* out, int32_t ldo, float* norm, void* stream) {
    TIDAS_REQUIRE(plan && samples && out, "tidas_psf_batch: null pointer");
    TIDAS_REQUIRE(n >= 1 && taps >= 1 && taps <= 255 && ldo >= taps && ldo <= 1024,
                  "tidas_psf_batch: bad sizes");
    const Plan& P = *(const Plan*)plan;
    psf_batch_kernel<<<n, ((ldo + 31) / 32) * 32, 0, ST(stream)>>>(psf_args(P, taps), samples, n,
                                                                    out, ldo, norm);
    return check_launch("psf_batch_kernel");
}

extern "C" int tidas_psf_batch_2d(das_plan plan, const double* samples, int32_t n, int32_t kz,
                                  int32_t taps, int32_t ldk, float* out, int32_t ldo, float* norm,
                                  void* stream) {
    TIDAS_REQUIRE(plan && samples && out, "tidas_psf_batch_2d: null pointer");
    TIDAS_REQUIRE(n >= 1 && kz >= 1 && kz <= 64 && taps >= 1 && taps <= 255 && ldk >= taps &&
                      ldo >= kz * ldk && ldo <= 65536,
                  "tidas_psf_batch_2d: bad sizes");
    const Plan& P = *(const Plan*)plan;
    psf_batch2d_kernel<<<n, 256, 0, ST(stream)>>>(psf_args(P, taps), samples, n, kz, ldk, out, ldo,
                                                  norm);
    return check_launch("psf_batch2d_kernel");
}

extern "C" int tidas_apod_sum(das_plan plan, const double* samples, int64_t n, float* out,
                              void* stream) {
    TIDAS_REQUIRE(plan && samples && out && n >= 1, "tidas_apod_sum: bad arguments");
    const Plan& P = *(const Plan*)plan;
    apod_sum_kernel<<<(int)((n + 255) / 256), 256, 0, ST(stream)>>>(psf_args(P, 1), samples, n, out);
    return check_launch("apod_sum_kernel");
}

extern "C" int tidas_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                               const float* bias, int32_t relu, float* c32, void* c16, int32_t ldc,
                               void* stream) {
    TIDAS_REQUIRE(A && B && (c32 || c16), "tidas_gemm_bf16: null pointer");
    TIDAS_REQUIRE(M >= 1 && N >= 16 && N % 16 == 0 && K >= 64 && K % 64 == 0,
                  "tidas_gemm_bf16: need N %% 16 == 0 and K %% 64 == 0 (M=%d N=%d K=%d)", M, N, K);
    TIDAS_REQUIRE(ldc >= N && ldc % 8 == 0, "tidas_gemm_bf16: ldc must be >= N and a multiple of 8");
    TIDAS_REQUIRE(((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0 &&
                      ((uintptr_t)c32 % 16) == 0 && ((uintptr_t)c16 % 16) == 0,
                  "tidas_gemm_bf16: 16-byte aligned arrays required");
    return launch_mlp_gemm((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, M, N, K, bias, relu,
                           c32, (__nv_bfloat16*)c16, ldc, ST(stream));
}

extern "C" int tidas_transpose_bf16(const void* in, int32_t rows, int32_t cols, void* out,
                                    void* stream) {
    TIDAS_REQUIRE(in && out && rows >= 1 && cols >= 1, "tidas_transpose_bf16: bad arguments");
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    transpose_bf16_kernel<<<grid, dim3(32, 8), 0, ST(stream)>>>((const __nv_bfloat16*)in, rows, cols,
                                                                (__nv_bfloat16*)out);
    return check_launch("transpose_bf16_kernel");
}

extern "C" int tidas_gather_rows(const void* src, const int32_t* idx, int64_t n, int32_t row_bytes,
                                 void* dst, void* stream) {
    TIDAS_REQUIRE(src && idx && dst && n >= 1 && row_bytes >= 4 && row_bytes % 4 == 0,
                  "tidas_gather_rows: bad arguments");
    gather_rows_kernel<<<(int)((n + 7) / 8), dim3(32, 8), 0, ST(stream)>>>(
        (const uint32_t*)src, idx, n, row_bytes / 4, (uint32_t*)dst);
    return check_launch("gather_rows_kernel");
}

extern "C" int tidas_relu_backward(const float* dpost, const float* act, int64_t n, float* dpre32,
                                   void* dpre16, void* stream) {
    TIDAS_REQUIRE(dpost && dpre16 && n >= 1, "tidas_relu_backward: bad arguments");
    relu_backward_kernel<<<vblocks(n), 256, 0, ST(stream)>>>(dpost, act, n, dpre32,
                                                             (__nv_bfloat16*)dpre16);
    return check_launch("relu_backward_kernel");
}

extern "C" int tidas_colsum(const float* d, int32_t rows, int32_t cols, int32_t ld, float* db,
                            void* stream) {
    TIDAS_REQUIRE(d && db && rows >= 1 && cols >= 1 && ld >= cols, "tidas_colsum: bad arguments");
    colsum_kernel<<<(cols + 127) / 128, 128, 0, ST(stream)>>>(d, rows, cols, ld, db);
    return check_launch("colsum_kernel");
}

extern "C" int tidas_adam(float* w, float* m, float* v, const float* g, int32_t rows, int32_t cols,
                          float lr, float b1, float b2, float eps, float wd, int32_t step, void* w16,
                          void* w16t, void* stream) {
    TIDAS_REQUIRE(w && m && v && g && rows >= 1 && cols >= 1 && step >= 1,
                  "tidas_adam: bad arguments");
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<vblocks((long long)rows * cols), 256, 0, ST(stream)>>>(
        w, m, v, g, rows, cols, lr, b1, b2, eps, wd, bc1, bc2, (__nv_bfloat16*)w16,
        (__nv_bfloat16*)w16t);
    return check_launch("adam_kernel");
}

extern "C" int tidas_mse(const float* pred, const float* target, int32_t rows, int32_t cols_used,
                         int32_t ldp, int32_t ldt, float* dpred, double* loss, void* stream) {
    TIDAS_REQUIRE(pred && target && dpred && loss && rows >= 1 && cols_used >= 1 &&
                      ldp >= cols_used && ldt >= cols_used,
                  "tidas_mse: bad arguments");
    const int nb = 64;
    double* partial = nullptr;
    TIDAS_CUDA(cudaMallocAsync((void**)&partial, sizeof(double) * nb, ST(stream)));
    mse_kernel<<<nb, 256, 0, ST(stream)>>>(pred, target, rows, cols_used, ldp, ldt, dpred, partial);
    int rc = check_launch("mse_kernel");
    if (!rc) {
        sum_partials_kernel<<<1, 32, 0, ST(stream)>>>(partial, nb,
                                                      1.0 / ((double)rows * cols_used), loss);
        rc = check_launch("sum_partials_kernel");
    }
    cudaError_t e = cudaFreeAsync(partial, ST(stream));
    if (rc) return rc;
    return check_cuda(e, "cudaFreeAsync(mse partials)");
}

extern "C" int tidas_encode(const double* samples, int32_t n, const float* lo4, const float* hi4,
                            void* out16, void* stream) {
    TIDAS_REQUIRE(samples && lo4 && hi4 && out16 && n >= 1, "tidas_encode: bad arguments");
    TIDAS_REQUIRE(((uintptr_t)out16 % 16) == 0, "tidas_encode: out16 must be 16-byte aligned");
    encode_kernel<<<(unsigned)(((long long)n * 8 + 255) / 256), 256, 0, ST(stream)>>>(
        samples, n, lo4, hi4, (__nv_bfloat16*)out16);
    return check_launch("encode_kernel");
}

extern "C" int tidas_kernel_fallback(const float* learned, int32_t ldl, const float* exact,
                                     int32_t lde, int64_t npix, int32_t taps, float thresh,
                                     float* out, int32_t ldo, float* nrmse, void* stream) {
    TIDAS_REQUIRE(learned && exact && out && npix >= 1 && taps >= 1 && ldl >= taps &&
                      lde >= taps && ldo >= taps,
                  "tidas_kernel_fallback: bad arguments");
    kernel_fallback_kernel<<<(int)((npix + 255) / 256), 256, 0, ST(stream)>>>(
        learned, ldl, exact, lde, npix, taps, thresh, out, ldo, nrmse);
    return check_launch("kernel_fallback_kernel");
}

extern "C" int tidas_row_scale(const float* in, int32_t ldi, const float* s, int64_t rows,
                               int32_t cols, float* out, int32_t ldo, void* stream) {
    TIDAS_REQUIRE(in && s && out && rows >= 1 && cols >= 1 && ldi >= cols && ldo >= cols,
                  "tidas_row_scale: bad arguments");
    row_scale_kernel<<<(int)((rows + 7) / 8), dim3(32, 8), 0, ST(stream)>>>(in, ldi, s, rows, cols,
                                                                           out, ldo);
    return check_launch("row_scale_kernel");
}

extern "C" int tidas_set_debug_option(int32_t option, int64_t value) {
    switch (option) {
        case TIDAS_DEBUG_WAIT_LIMIT_NS:
            TIDAS_REQUIRE(value >= 1000 && value <= 10000000000ll,
                          "tidas_set_debug_option: wait limit %lld ns outside [1e3, 1e10]",
                          (long long)value);
            g_dbg_wait_ns.store((unsigned long long)value);
            return TIDAS_OK;
        case TIDAS_DEBUG_SKIP_COPIES:
            TIDAS_REQUIRE(value == 0 || value == 1, "tidas_set_debug_option: skip must be 0 or 1");
            g_dbg_skip_loads.store((int)value);
            return TIDAS_OK;
        default:
            return set_error(TIDAS_ERR_ARG, "tidas_set_debug_option: unknown option %d", option);
    }
}
