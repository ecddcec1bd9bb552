// Vector kernels of the deconvolution driver: FP64 reductions (dot products,
// absolute sums) and the fused FISTA update (soft threshold + momentum).
#include "common.cuh"

namespace tidas {

constexpr int kRedThreads = 256;

// Per-block partial sums in FP64; op 0: sum a*b, op 1: sum |a|.
__global__ void __launch_bounds__(kRedThreads) reduce_partial_kernel(const float* __restrict__ a,
                                                                     const float* __restrict__ b,
                                                                     long long n, int op,
                                                                     double* __restrict__ partial) {
    double s = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (op == 0) {
        for (; i < n; i += stride) s += (double)a[i] * (double)b[i];
    } else {
        for (; i < n; i += stride) s += fabs((double)a[i]);
    }
    __shared__ double red[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

// Sum of the partials in a fixed order (deterministic result).
__global__ void reduce_final_kernel(const double* __restrict__ partial, int np,
                                    double* __restrict__ out) {
    __shared__ double red[kRedThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

int reduce_blocks(long long n) {
    long long b = (n + kRedThreads - 1) / kRedThreads;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

int launch_reduce(const float* a, const float* b, long long n, int op, double* partial, int nb,
                  double* out, cudaStream_t st) {
    reduce_partial_kernel<<<nb, kRedThreads, 0, st>>>(a, b, n, op, partial);
    int rc = check_launch("reduce_partial_kernel");
    if (rc) return rc;
    reduce_final_kernel<<<1, kRedThreads, 0, st>>>(partial, nb, out);
    return check_launch("reduce_final_kernel");
}

// z = y - step * grad; x_new = sign(z) max(|z| - thresh, 0);
// y = x_new + beta (x_new - x); x = x_new.
__global__ void fista_update_kernel(float* __restrict__ x, float* __restrict__ y,
                                    const float* __restrict__ grad, long long n, float step,
                                    float thresh, float beta) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float z = fmaf(-step, grad[i], y[i]);
        const float m = fabsf(z) - thresh;
        const float xn = m > 0.f ? copysignf(m, z) : 0.f;
        y[i] = fmaf(beta, xn - x[i], xn);
        x[i] = xn;
    }
}

// out = alpha a + beta b
__global__ void axpby_kernel(const float* __restrict__ a, const float* __restrict__ b,
                             float* __restrict__ out, long long n, float alpha, float beta) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = fmaf(alpha, a[i], beta * b[i]);
}

static int vec_blocks(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace tidas

using namespace tidas;

static int reduce_entry(const char* who, const float* a, const float* b, long long n, int op,
                        double* out, void* stream) {
    TIDAS_REQUIRE(out && (n == 0 || (a && (op == 1 || b))), "%s: null pointer", who);
    TIDAS_REQUIRE(n >= 0, "%s: negative length", who);
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = reduce_blocks(n);
    double* partial = nullptr;
    TIDAS_CUDA(cudaMallocAsync((void**)&partial, sizeof(double) * nb, st));
    int rc = launch_reduce(a, b, n, op, partial, nb, out, st);
    cudaError_t e = cudaFreeAsync(partial, st);
    if (rc) return rc;
    return check_cuda(e, "cudaFreeAsync(reduction partials)");
}

extern "C" int tidas_dot(const float* a, const float* b, int64_t n, double* out, void* stream) {
    return reduce_entry("tidas_dot", a, b, n, 0, out, stream);
}

extern "C" int tidas_asum(const float* a, int64_t n, double* out, void* stream) {
    return reduce_entry("tidas_asum", a, nullptr, n, 1, out, stream);
}

extern "C" int tidas_fista_update(float* x, float* y, const float* grad, int64_t n, float step,
                                  float thresh, float beta, void* stream) {
    TIDAS_REQUIRE(x && y && grad && n >= 0, "tidas_fista_update: bad arguments");
    TIDAS_REQUIRE(step > 0.f && thresh >= 0.f, "tidas_fista_update: step must be > 0, thresh >= 0");
    if (n == 0) return TIDAS_OK;
    fista_update_kernel<<<vec_blocks(n), 256, 0, (cudaStream_t)stream>>>(x, y, grad, n, step,
                                                                          thresh, beta);
    return check_launch("fista_update_kernel");
}

extern "C" int tidas_axpby(const float* a, const float* b, float* out, int64_t n, float alpha,
                           float beta, void* stream) {
    TIDAS_REQUIRE(a && b && out && n >= 0, "tidas_axpby: bad arguments");
    if (n == 0) return TIDAS_OK;
    axpby_kernel<<<vec_blocks(n), 256, 0, (cudaStream_t)stream>>>(a, b, out, n, alpha, beta);
    return check_launch("axpby_kernel");
}

// ---------------------------------------------------------------------------
// Allocation-free FP64 dot product.
//
// Some callers cannot let the library allocate device memory: a scanner or
// streaming pipeline that reserves its whole device budget when it starts and
// treats any later allocation as a failure, or a host thread that must not
// wait on an allocator.  For them the per-block partial sums of tidas_dot live
// in the fixed array below instead of a stream-ordered allocation.
//
// The array is a file-scope device variable: every GPU that loads the library
// holds it until the process exits.  Host code cannot use the name of the
// array as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and keeps
// it; make that first call before any stream capture.  The kept address is
// the array's place in the module loaded into the device's context; a
// cudaDeviceReset unloads that module, so it is not valid across a reset.
// All calls share the
// array and it keeps the previous call's contents; every partial this call
// reads is written by the same call first, so nothing needs clearing.  Calls
// that overlap on the GPU (for example on two streams) race on the array.
namespace tidas {
constexpr int kNoAllocPartials = 4096;                       // 32 KB of FP64 partials
constexpr long long kNoAllocPerBlock = 4096;                 // elements per partial sum
constexpr long long kNoAllocMaxN = kNoAllocPartials * kNoAllocPerBlock;  // 16,777,216
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];
}  // namespace tidas

#include <mutex>

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[256] = {nullptr};

extern "C" int tidas_dot_noalloc(const float* a, const float* b, int64_t n, double* out,
                                 void* stream) {
    TIDAS_REQUIRE(out && (n == 0 || (a && b)), "tidas_dot_noalloc: null pointer");
    TIDAS_REQUIRE(n >= 0, "tidas_dot_noalloc: negative length");
    TIDAS_REQUIRE(n <= kNoAllocMaxN,
                  "tidas_dot_noalloc: n = %lld exceeds the fixed scratch limit of %lld elements",
                  (long long)n, kNoAllocMaxN);
    int dev = 0;
    TIDAS_CUDA(cudaGetDevice(&dev));
    TIDAS_REQUIRE(dev >= 0 && dev < 256, "tidas_dot_noalloc: device index %d out of range", dev);
    double* partial;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            TIDAS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
            g_noalloc_ptr[dev] = (double*)p;
        }
        partial = g_noalloc_ptr[dev];
    }
    long long nb = (n + kNoAllocPerBlock - 1) / kNoAllocPerBlock;
    if (nb < 1) nb = 1;
    return launch_reduce(a, b, n, 0, partial, (int)nb, out, (cudaStream_t)stream);
}
