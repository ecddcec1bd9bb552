// Plan construction, error reporting and the FP64 delay-table builder.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace tidas {

static thread_local char t_last_error[512] = "";

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TIDAS_OK;
    return set_error(TIDAS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_launch(const char* what) { return check_cuda(cudaGetLastError(), what); }

// ------------------------------------------------------------------------
// Delay-index table, FP64, every operation individually rounded in the
// order ((x sin + z cos) + sqrt(ddx^2 + z^2)) / c - t0) * fs.
struct TableArgs {
    int n_elem, nx, nz;
    double pitch, c, fs, t0, x0, dx, z0, dz, sn, cs;
};

__global__ void delay_table_kernel(TableArgs t, int32_t* idx, float* frac) {
    long long total = (long long)t.nz * t.nx * t.n_elem;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        int n = (int)(o % t.n_elem);
        long long p = o / t.n_elem;
        int ix = (int)(p % t.nx);
        int iz = (int)(p / t.nx);
        double x = __dadd_rn(t.x0, __dmul_rn((double)ix + 0.5, t.dx));
        double z = __dadd_rn(t.z0, __dmul_rn((double)iz + 0.5, t.dz));
        double xn = __dmul_rn(__dsub_rn((double)n, 0.5 * (double)(t.n_elem - 1)), t.pitch);
        double ddx = __dsub_rn(x, xn);
        double tx = __dadd_rn(__dmul_rn(x, t.sn), __dmul_rn(z, t.cs));
        double rx = __dsqrt_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(z, z)));
        double u = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tx, rx), t.c), t.t0), t.fs);
        double fl = floor(u);
        idx[o] = (int32_t)fl;
        frac[o] = __double2float_rn(__dsub_rn(u, fl));
    }
}

int launch_delay_table(const Plan& P, int angle, int32_t* idx, float* frac, cudaStream_t st) {
    TableArgs t;
    t.n_elem = P.p.n_elem;
    t.nx = P.p.nx;
    t.nz = P.p.nz;
    t.pitch = P.p.pitch;
    t.c = P.p.c;
    t.fs = P.p.fs;
    t.t0 = P.p.t0;
    t.x0 = P.p.x0;
    t.dx = P.p.dx;
    t.z0 = P.p.z0;
    t.dz = P.p.dz;
    t.sn = P.sn[angle];
    t.cs = P.cs[angle];
    long long total = (long long)t.nz * t.nx * t.n_elem;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    delay_table_kernel<<<blocks, 256, 0, st>>>(t, idx, frac);
    return check_launch("delay_table_kernel");
}

}  // namespace tidas

using namespace tidas;

static void split_fp64(double v, int* i, float* f) {
    double fl = floor(v);
    *i = (int)fl;
    *f = (float)(v - fl);
}

extern "C" int das_plan_create(const das_params* params, das_plan* out_plan) {
    TIDAS_REQUIRE(params && out_plan, "das_plan_create: null argument");
    *out_plan = nullptr;
    const das_params& p = *params;
    TIDAS_REQUIRE(p.n_elem >= 1 && p.n_elem <= 1024, "n_elem out of range: %d", p.n_elem);
    TIDAS_REQUIRE(p.n_angles >= 1 && p.n_angles <= kMaxAngles, "n_angles out of range: %d",
                  p.n_angles);
    TIDAS_REQUIRE(p.angles_rad != nullptr, "angles_rad is null");
    TIDAS_REQUIRE(p.n_samples >= 4 && p.n_samples <= (1 << 22), "n_samples out of range: %d",
                  p.n_samples);
    TIDAS_REQUIRE(p.nx >= 1 && p.nx <= 8192 && p.nz >= 1 && p.nz <= 8192, "grid size out of range");
    TIDAS_REQUIRE(p.pitch > 0 && p.c > 0 && p.fs > 0 && p.f0 > 0 && p.dx > 0 && p.dz > 0,
                  "non-positive physical parameter");
    TIDAS_REQUIRE(p.frac_bw > 0 && p.frac_bw <= 2.0, "frac_bw out of range");
    TIDAS_REQUIRE(p.z0 + 0.5 * p.dz > 0, "grid must lie below the array (z > 0)");
    TIDAS_REQUIRE(p.interp == TIDAS_INTERP_LINEAR || p.interp == TIDAS_INTERP_CUBIC,
                  "interp must be 0 (linear) or 1 (cubic)");
    TIDAS_REQUIRE(p.rf_dtype == TIDAS_RF_F32 || p.rf_dtype == TIDAS_RF_F16, "bad rf_dtype");

    Plan* P = new Plan();
    P->p = p;
    P->p.angles_rad = nullptr;
    for (int a = 0; a < p.n_angles; ++a) {
        P->angles[a] = p.angles_rad[a];
        P->sn[a] = sin(p.angles_rad[a]);
        P->cs[a] = cos(p.angles_rad[a]);
    }
    const int A = p.n_angles, NX = p.nx, NZ = p.nz, NE = p.n_elem;
    const double k = p.fs / p.c;  // samples per metre of path

    // host tables
    std::vector<int> bxi(A * NX), bzi(A * NZ);
    std::vector<float> bxf(A * NX), bzf(A * NZ), dxs((size_t)NE * NX), zs(NZ), xs(NX);
    for (int a = 0; a < A; ++a) {
        for (int ix = 0; ix < NX; ++ix) {
            double x = p.x0 + ((double)ix + 0.5) * p.dx;
            split_fp64(x * P->sn[a] * k, &bxi[a * NX + ix], &bxf[a * NX + ix]);
        }
        for (int iz = 0; iz < NZ; ++iz) {
            double z = p.z0 + ((double)iz + 0.5) * p.dz;
            split_fp64((z * P->cs[a] + z) * k - p.t0 * p.fs, &bzi[a * NZ + iz], &bzf[a * NZ + iz]);
        }
    }
    for (int n = 0; n < NE; ++n) {
        double xn = ((double)n - 0.5 * (double)(NE - 1)) * p.pitch;
        for (int ix = 0; ix < NX; ++ix) {
            double x = p.x0 + ((double)ix + 0.5) * p.dx;
            dxs[(size_t)n * NX + ix] = (float)((x - xn) * k);
        }
    }
    for (int iz = 0; iz < NZ; ++iz) zs[iz] = (float)((p.z0 + ((double)iz + 0.5) * p.dz) * k);
    for (int ix = 0; ix < NX; ++ix) xs[ix] = (float)((p.x0 + ((double)ix + 0.5) * p.dx) * k);

    // pulse: Gaussian envelope exp(-alpha t^2) whose spectrum is 6 dB down at
    // f0 (1 +- frac_bw / 2); support where the envelope is above -60 dB
    const double alpha = M_PI * M_PI * (0.5 * p.frac_bw * p.f0) * (0.5 * p.frac_bw * p.f0) /
                         log(pow(10.0, 6.0 / 20.0));
    P->thalf_samples = sqrt(log(pow(10.0, 60.0 / 20.0)) / alpha) * p.fs;
    P->beta_samples = alpha / (p.fs * p.fs);
    P->wcar = 2.0 * p.f0 / p.fs;
    std::vector<float> ptab(3 * (2 * kJ + 1));
    for (int j = -kJ; j <= kJ; ++j) {
        ptab[j + kJ] = (float)exp(-P->beta_samples * j * j);
        ptab[(2 * kJ + 1) + j + kJ] = (float)cos(M_PI * P->wcar * j);
        ptab[2 * (2 * kJ + 1) + j + kJ] = (float)sin(M_PI * P->wcar * j);
    }
    // carrier at integer samples, e^{i pi wcar k} for k = -kJ .. S + kJ - 1, from
    // the FP64 phase reduced modulo 2 (so that large k lose no accuracy)
    std::vector<float2> carr((size_t)p.n_samples + 2 * kJ);
    for (int k = -kJ; k < p.n_samples + kJ; ++k) {
        const double ph = fmod(P->wcar * (double)k, 2.0);
        carr[(size_t)(k + kJ)] = make_float2((float)cos(M_PI * ph), (float)sin(M_PI * ph));
    }
    std::vector<double> sncs(2 * A);
    for (int a = 0; a < A; ++a) {
        sncs[2 * a] = P->sn[a];
        sncs[2 * a + 1] = P->cs[a];
    }

    // Are all interpolation taps inside the record?  u increases with z for
    // every steering angle below 90 degrees, so the extremes lie on the first
    // and last rows; one sample of margin covers the split-delay rounding.
    {
        double umin = 1e300, umax = -1e300;
        const double zf = p.z0 + 0.5 * p.dz, zl = p.z0 + ((double)NZ - 0.5) * p.dz;
        for (int a = 0; a < A; ++a)
            for (int n = 0; n < NE; ++n) {
                double xn = ((double)n - 0.5 * (double)(NE - 1)) * p.pitch;
                for (int ix = 0; ix < NX; ++ix) {
                    double x = p.x0 + ((double)ix + 0.5) * p.dx;
                    double u1 = ((x * P->sn[a] + zf * P->cs[a] + sqrt((x - xn) * (x - xn) + zf * zf)) /
                                     p.c - p.t0) * p.fs;
                    double u2 = ((x * P->sn[a] + zl * P->cs[a] + sqrt((x - xn) * (x - xn) + zl * zl)) /
                                     p.c - p.t0) * p.fs;
                    umin = fmin(umin, fmin(u1, u2));
                    umax = fmax(umax, fmax(u1, u2));
                }
            }
        P->taps_in_range = (floor(umin) - 2.0 >= 0.0) && (floor(umax) + 3.0 <= p.n_samples - 1.0);
        // samples any pixel can weight: taps floor(u) - 1 .. floor(u) + 2 of the
        // extreme delays, one more sample each side for the split-delay rounding
        const double first = fmax(0.0, floor(umin) - 3.0);
        const double last = fmin((double)p.n_samples - 1.0, floor(umax) + 4.0);
        P->read_first = (int)first;
        P->read_count = last >= first ? (int)(last - first) + 1 : 0;
    }

    // one blob, 256-byte aligned pieces
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t o_bxi = 0, o_bxf = o_bxi + al(4 * A * NX), o_bzi = o_bxf + al(4 * A * NX),
           o_bzf = o_bzi + al(4 * A * NZ), o_dxs = o_bzf + al(4 * A * NZ),
           o_zs = o_dxs + al(4 * (size_t)NE * NX), o_xs = o_zs + al(4 * NZ),
           o_ptab = o_xs + al(4 * NX), o_sncs = o_ptab + al(4 * ptab.size()),
           o_carr = o_sncs + al(8 * sncs.size()), total = o_carr + al(8 * carr.size());
    void* blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, total);
    if (e != cudaSuccess) {
        delete P;
        return check_cuda(e, "cudaMalloc(plan tables)");
    }
    char* b = (char*)blob;
    struct {
        size_t off;
        const void* src;
        size_t n;
    } up[] = {{o_bxi, bxi.data(), 4 * bxi.size()}, {o_bxf, bxf.data(), 4 * bxf.size()},
              {o_bzi, bzi.data(), 4 * bzi.size()}, {o_bzf, bzf.data(), 4 * bzf.size()},
              {o_dxs, dxs.data(), 4 * dxs.size()}, {o_zs, zs.data(), 4 * zs.size()},
              {o_xs, xs.data(), 4 * xs.size()},  {o_ptab, ptab.data(), 4 * ptab.size()},
              {o_sncs, sncs.data(), 8 * sncs.size()}, {o_carr, carr.data(), 8 * carr.size()}};
    for (auto& u : up) {
        e = cudaMemcpy(b + u.off, u.src, u.n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(blob);
            delete P;
            return check_cuda(e, "cudaMemcpy(plan tables)");
        }
    }
    P->blob = blob;
    DasDev& d = P->dev;
    d.n_elem = NE;
    d.n_angles = A;
    d.n_samples = p.n_samples;
    d.nx = NX;
    d.nz = NZ;
    d.interp = p.interp;
    d.rf_dtype = p.rf_dtype;
    d.fnum = (float)p.fnum;
    d.thalf = (float)P->thalf_samples;
    d.beta = (float)P->beta_samples;
    d.wcar = (float)P->wcar;
    d.ptab = (const float*)(b + o_ptab);
    d.carr = (const float2*)(b + o_carr) + kJ;
    P->d_sncs = (const double*)(b + o_sncs);
    d.bxi = (const int*)(b + o_bxi);
    d.bxf = (const float*)(b + o_bxf);
    d.bzi = (const int*)(b + o_bzi);
    d.bzf = (const float*)(b + o_bzf);
    d.dxs = (const float*)(b + o_dxs);
    d.zs = (const float*)(b + o_zs);
    d.xs = (const float*)(b + o_xs);
    d.elem0_s = (float)(-0.5 * (double)(NE - 1) * p.pitch * k);
    d.pitch_s = (float)(p.pitch * k);
    if (p.rf_dtype == TIDAS_RF_F16 && p.n_samples % 8 == 0) {
        // sample windows of the tensor-core DAS; without them the CUDA-core
        // kernel serves every batch
        int rc = das_tc_prepare(*P);
        if (rc) {
            cudaFree(P->tc_tab);
            cudaFree(P->blob);
            delete P;
            return rc;
        }
    }
    *out_plan = (das_plan)P;
    return TIDAS_OK;
}

extern "C" int das_plan_set_option(das_plan plan, int32_t option, int32_t value) {
    TIDAS_REQUIRE(plan, "das_plan_set_option: null plan");
    Plan* P = (Plan*)plan;
    if (option == DAS_OPT_TENSOR_CORES) {
        TIDAS_REQUIRE(value == 0 || value == 1, "das_plan_set_option: value must be 0 or 1");
        P->tc_mode = value;
        return TIDAS_OK;
    }
    return set_error(TIDAS_ERR_ARG, "das_plan_set_option: unknown option %d", option);
}

extern "C" int das_plan_read_window(das_plan plan, int32_t* first_sample, int32_t* n_samples) {
    TIDAS_REQUIRE(plan && first_sample && n_samples, "das_plan_read_window: null argument");
    const Plan* P = (const Plan*)plan;
    *first_sample = P->read_first;
    *n_samples = P->read_count;
    return TIDAS_OK;
}

extern "C" int das_upload_window(das_plan plan, const void* host_rf, void* rf, int32_t n_frames,
                                 void* stream) {
    TIDAS_REQUIRE(plan && host_rf && rf, "das_upload_window: null argument");
    TIDAS_REQUIRE(n_frames >= 1, "das_upload_window: n_frames must be >= 1");
    const Plan* P = (const Plan*)plan;
    if (P->read_count == 0) return TIDAS_OK;
    const size_t es = P->p.rf_dtype == TIDAS_RF_F16 ? 2 : 4;
    const size_t pitch = (size_t)P->p.n_samples * es;
    const size_t rows = (size_t)n_frames * P->p.n_angles * P->p.n_elem;
    const size_t off = (size_t)P->read_first * es;
    TIDAS_CUDA(cudaMemcpy2DAsync((char*)rf + off, pitch, (const char*)host_rf + off, pitch,
                                 (size_t)P->read_count * es, rows, cudaMemcpyHostToDevice,
                                 (cudaStream_t)stream));
    return TIDAS_OK;
}

extern "C" int das_plan_destroy(das_plan plan) {
    if (!plan) return TIDAS_OK;
    Plan* P = (Plan*)plan;
    cudaError_t e = cudaDeviceSynchronize();
    cudaError_t e2 = cudaFree(P->blob);
    if (P->tc_tab) {
        cudaError_t e3 = cudaFree(P->tc_tab);
        if (e2 == cudaSuccess) e2 = e3;
    }
    if (P->tc_ws) {
        cudaError_t e4 = cudaFree(P->tc_ws);
        if (e2 == cudaSuccess) e2 = e4;
    }
    delete P;
    if (e != cudaSuccess) return check_cuda(e, "cudaDeviceSynchronize(plan destroy)");
    return check_cuda(e2, "cudaFree(plan tables)");
}

extern "C" const char* tidas_last_error(void) { return tidas::t_last_error; }

