// extern "C" entry points: argument validation, then one launcher call each.
#include "common.cuh"

namespace tidas {
int launch_tidas_direct(const float* kern, int taps, int center, bool adjoint, int nz, int nx,
                        const float* in, float* out, int nf, cudaStream_t st);
int launch_tidas_gemm(const float* kern, int taps, int center, bool adjoint, int nz, int nx,
                      const void* in, float* out, int nf, bool resid, cudaStream_t st);
int launch_tidas_direct2d(const float* kern, int kz, int taps, bool adjoint, int nz, int nx,
                          const float* in, float* out, int nf, cudaStream_t st);
int launch_tidas_gemm2d(const float* kern, int kz, int taps, bool adjoint, int nz, int nx,
                        const void* in, float* out, int nf, void* workspace, size_t ws_bytes,
                        cudaStream_t st);
size_t band_pack_bytes(int nz, int nx, int nf);
int validate_line(const tidas_line_params* p);
double line_window(const tidas_line_params& p);
int launch_line_combine(const tidas_line_params& p, const float* rf, int n_scat, const float* amps,
                        float* out, cudaStream_t st);
int launch_line_model(const tidas_line_params& p, const float* S, int s, const float* theta,
                      double eps, float* out, cudaStream_t st);
int launch_line_envelope(int n_rows, int n, const float* x, float* env, cudaStream_t st);
int launch_line_fixed(const tidas_line_params& p, const float* rf, int r_first, int n_scat, int s,
                      double eps, float* out, cudaStream_t st);
int launch_line_synth(const tidas_line_params& p, int r_first, int n_scat, float* rf,
                      cudaStream_t st);
int launch_line_das(const tidas_line_params& p, const float* rf, int n_scat, float* lines,
                    cudaStream_t st);
int launch_line_sweep(const tidas_line_params& p, const float* rf, const float* lines,
                      int r_first, int n_scat, double eps, float* theta, float* e_loc,
                      float* e_glob, cudaStream_t st);
int launch_fit_kernels_2d(const Plan& P, int kz, int taps, float* kernels, cudaStream_t st);
}  // namespace tidas

using namespace tidas;

static inline cudaStream_t S_(void* s) { return (cudaStream_t)s; }

#define PLAN_OR_FAIL(plan)                                      \
    TIDAS_REQUIRE(plan != nullptr, "%s: null plan", __func__); \
    const Plan& P = *(const Plan*)(plan)

extern "C" int das_synthesize(das_plan plan, const double* pos_xz, const float* amp,
                              int32_t n_scat, int32_t n_frames, void* rf, void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(n_frames >= 1 && n_scat >= 0, "das_synthesize: bad sizes");
    TIDAS_REQUIRE(rf && (n_scat == 0 || (pos_xz && amp)), "das_synthesize: null pointer");
    TIDAS_REQUIRE(P.p.n_samples <= 49152, "das_synthesize: n_samples > 49152 unsupported");
    return launch_synthesize(P, pos_xz, amp, n_scat, n_frames, rf, S_(stream));
}

extern "C" int das_synthesize_grid(das_plan plan, const float* refl, void* rf, int32_t n_frames,
                                   void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(n_frames >= 1 && refl && rf, "das_synthesize_grid: bad arguments");
    TIDAS_REQUIRE(P.p.rf_dtype == TIDAS_RF_F32, "das_synthesize_grid: needs an FP32 plan");
    TIDAS_REQUIRE(P.p.n_samples <= 49152, "das_synthesize_grid: n_samples > 49152 unsupported");
    if (P.thalf_samples > kJ - 2)
        return set_error(TIDAS_ERR_UNSUPPORTED, "pulse longer than %d samples", kJ - 2);
    return launch_synthesize_grid(P, refl, (float*)rf, n_frames, S_(stream));
}

extern "C" int das_synthesize_adjoint(das_plan plan, const void* rf, float* refl,
                                      int32_t n_frames, void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(n_frames >= 1 && refl && rf, "das_synthesize_adjoint: bad arguments");
    TIDAS_REQUIRE(P.p.rf_dtype == TIDAS_RF_F32, "das_synthesize_adjoint: needs an FP32 plan");
    if (P.thalf_samples > kJ - 2)
        return set_error(TIDAS_ERR_UNSUPPORTED, "pulse longer than %d samples", kJ - 2);
    return launch_synthesize_adjoint(P, (const float*)rf, refl, n_frames, S_(stream));
}

extern "C" int das_forward(das_plan plan, const void* rf, float* img, int32_t n_frames,
                           void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(n_frames >= 1 && rf && img, "das_forward: bad arguments");
    TIDAS_REQUIRE(n_frames <= 65535 * 8, "das_forward: too many frames");
    return launch_das_forward(P, rf, img, n_frames, S_(stream));
}

extern "C" int das_adjoint(das_plan plan, const float* img, float* rf, int32_t n_frames,
                           void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(n_frames >= 1 && rf && img, "das_adjoint: bad arguments");
    TIDAS_REQUIRE(P.p.rf_dtype == TIDAS_RF_F32, "das_adjoint: needs an FP32 plan");
    TIDAS_REQUIRE(n_frames <= 65535, "das_adjoint: too many frames");
    if (P.p.n_samples > 49152)
        return set_error(TIDAS_ERR_UNSUPPORTED, "das_adjoint: n_samples > 49152");
    return launch_das_adjoint(P, img, rf, n_frames, S_(stream));
}

extern "C" int das_delay_table(das_plan plan, int32_t angle, int32_t* idx, float* frac,
                               void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(idx && frac, "das_delay_table: null pointer");
    TIDAS_REQUIRE(angle >= 0 && angle < P.p.n_angles, "das_delay_table: bad angle %d", angle);
    return launch_delay_table(P, angle, idx, frac, S_(stream));
}

extern "C" int tidas_fit_kernels(das_plan plan, int32_t taps, int32_t ref_stride, float* kernels,
                                 float* theta, void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(kernels, "tidas_fit_kernels: null kernels");
    TIDAS_REQUIRE(taps >= 1 && taps <= 255, "tidas_fit_kernels: taps out of range");
    return launch_fit_kernels(P, taps, ref_stride, kernels, theta, S_(stream));
}

static int tidas_common(const char* who, const float* kernels, int32_t taps, int32_t nz, int32_t nx,
                        const void* in, float* out, int32_t n_frames, int32_t variant,
                        bool adjoint, void* stream) {
    TIDAS_REQUIRE(kernels && in && out, "%s: null pointer", who);
    TIDAS_REQUIRE(taps >= 1 && taps <= 255, "%s: taps out of range", who);
    TIDAS_REQUIRE(nz >= 1 && nz <= 65535 && nx >= 1 && nx <= 16384, "%s: bad grid", who);
    TIDAS_REQUIRE(n_frames >= 1 && n_frames <= 65535 * 4, "%s: bad frame count", who);
    const int center = taps / 2;
    if (variant == TIDAS_VARIANT_DIRECT)
        return launch_tidas_direct(kernels, taps, center, adjoint, nz, nx, (const float*)in, out,
                                   n_frames, S_(stream));
    if (variant == TIDAS_VARIANT_GEMM_BF16 || variant == TIDAS_VARIANT_GEMM_RESID) {
        TIDAS_REQUIRE(taps <= 63, "%s: GEMM variants need taps <= 63", who);
        TIDAS_REQUIRE(nx % 8 == 0, "%s: GEMM variants need nx %% 8 == 0", who);
        TIDAS_REQUIRE(((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0,
                      "%s: GEMM variants need 16-byte aligned arrays", who);
        return launch_tidas_gemm(kernels, taps, center, adjoint, nz, nx, in, out, n_frames,
                                 variant == TIDAS_VARIANT_GEMM_RESID, S_(stream));
    }
    return set_error(TIDAS_ERR_ARG, "%s: unknown variant %d", who, variant);
}

extern "C" int tidas_forward(const float* kernels, int32_t taps, int32_t nz, int32_t nx,
                             const void* refl, float* img, int32_t n_frames, int32_t variant,
                             void* stream) {
    return tidas_common("tidas_forward", kernels, taps, nz, nx, refl, img, n_frames, variant,
                        false, stream);
}

extern "C" int tidas_adjoint(const float* kernels, int32_t taps, int32_t nz, int32_t nx,
                             const void* img, float* refl, int32_t n_frames, int32_t variant,
                             void* stream) {
    return tidas_common("tidas_adjoint", kernels, taps, nz, nx, img, refl, n_frames, variant, true,
                        stream);
}

// ------------------------------------------------ 2D band kernels
extern "C" int tidas_fit_kernels_2d(das_plan plan, int32_t kz, int32_t taps, float* kernels,
                                    void* stream) {
    PLAN_OR_FAIL(plan);
    TIDAS_REQUIRE(kernels, "tidas_fit_kernels_2d: null kernels");
    TIDAS_REQUIRE(taps >= 1 && taps <= 255 && kz >= 1 && kz <= 64,
                  "tidas_fit_kernels_2d: need 1 <= taps <= 255 and 1 <= kz <= 64");
    return launch_fit_kernels_2d(P, kz, taps, kernels, S_(stream));
}

extern "C" size_t tidas_band_workspace_bytes(int32_t nz, int32_t nx, int32_t n_frames,
                                            int32_t variant) {
    if (variant != TIDAS_VARIANT_GEMM_BF16 || nz < 1 || nx < 1 || n_frames < 1) return 0;
    return band_pack_bytes(nz, nx, n_frames);
}

static int tidas2d_common(const char* who, const float* kernels, int32_t kz, int32_t taps,
                          int32_t nz, int32_t nx, const void* in, float* out, int32_t n_frames,
                          int32_t variant, void* workspace, size_t ws_bytes, bool adjoint,
                          void* stream) {
    TIDAS_REQUIRE(kernels && in && out, "%s: null pointer", who);
    TIDAS_REQUIRE(taps >= 1 && taps <= 255 && kz >= 1 && kz <= 64, "%s: bad kernel shape", who);
    TIDAS_REQUIRE(nz >= 1 && nz <= 65535 && nx >= 1 && nx <= 2048, "%s: bad grid", who);
    TIDAS_REQUIRE(n_frames >= 1 && n_frames <= 65535, "%s: bad frame count", who);
    if (variant == TIDAS_VARIANT_DIRECT)
        return launch_tidas_direct2d(kernels, kz, taps, adjoint, nz, nx, (const float*)in, out,
                                     n_frames, S_(stream));
    if (variant == TIDAS_VARIANT_GEMM_BF16) {
        TIDAS_REQUIRE(taps <= 63, "%s: the GEMM variant needs taps <= 63", who);
        TIDAS_REQUIRE(nx % 8 == 0, "%s: the GEMM variant needs nx %% 8 == 0", who);
        TIDAS_REQUIRE(((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0,
                      "%s: the GEMM variant needs 16-byte aligned arrays", who);
        return launch_tidas_gemm2d(kernels, kz, taps, adjoint, nz, nx, in, out, n_frames,
                                   workspace, ws_bytes, S_(stream));
    }
    return set_error(TIDAS_ERR_ARG, "%s: variant %d is not available for 2D kernels", who,
                     variant);
}

extern "C" int tidas_forward_2d(const float* kernels, int32_t kz, int32_t taps, int32_t nz,
                                int32_t nx, const void* refl, float* img, int32_t n_frames,
                                int32_t variant, void* workspace, size_t workspace_bytes,
                                void* stream) {
    return tidas2d_common("tidas_forward_2d", kernels, kz, taps, nz, nx, refl, img, n_frames,
                          variant, workspace, workspace_bytes, false, stream);
}

extern "C" int tidas_adjoint_2d(const float* kernels, int32_t kz, int32_t taps, int32_t nz,
                                int32_t nx, const void* img, float* refl, int32_t n_frames,
                                int32_t variant, void* workspace, size_t workspace_bytes,
                                void* stream) {
    return tidas2d_common("tidas_adjoint_2d", kernels, kz, taps, nz, nx, img, refl, n_frames,
                          variant, workspace, workspace_bytes, true, stream);
}

// ------------------------------------------------ single-line experiment
extern "C" int tidas_line_synthesize(const tidas_line_params* p, int32_t r_first, int32_t n_scat,
                                     float* rf, void* stream) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(rf, "tidas_line_synthesize: null rf");
    TIDAS_REQUIRE(n_scat >= 1 && n_scat <= 65535 && r_first >= 0 && r_first + n_scat <= p->n_depths,
                  "tidas_line_synthesize: scatterers outside the line");
    return launch_line_synth(*p, r_first, n_scat, rf, S_(stream));
}

extern "C" int tidas_line_das(const tidas_line_params* p, const float* rf, int32_t n_scat,
                              float* lines, void* stream) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(rf && lines, "tidas_line_das: null pointer");
    TIDAS_REQUIRE(n_scat >= 1 && n_scat <= 65535, "tidas_line_das: bad n_scat");
    return launch_line_das(*p, rf, n_scat, lines, S_(stream));
}

extern "C" int tidas_line_sweep(const tidas_line_params* p, const float* rf, const float* lines,
                                int32_t r_first, int32_t n_scat, double eps, float* theta,
                                float* err_local, float* err_global, void* stream) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(rf && lines && theta && err_local && err_global, "tidas_line_sweep: null pointer");
    TIDAS_REQUIRE(n_scat >= 1 && r_first >= 0 && r_first + n_scat <= p->n_depths,
                  "tidas_line_sweep: scatterers outside the line");
    TIDAS_REQUIRE(eps > 0.0, "tidas_line_sweep: eps must be positive");
    return launch_line_sweep(*p, rf, lines, r_first, n_scat, eps, theta, err_local, err_global,
                             S_(stream));
}

extern "C" int tidas_line_window(const tidas_line_params* p, double* eps) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(eps, "tidas_line_window: null eps");
    *eps = line_window(*p);
    return TIDAS_OK;
}

extern "C" int tidas_line_combine(const tidas_line_params* p, const float* rf, int32_t n_scat,
                                  const float* amps, float* rf_line, void* stream) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(rf && amps && rf_line, "tidas_line_combine: null pointer");
    TIDAS_REQUIRE(n_scat >= 1 && n_scat <= 8192, "tidas_line_combine: need 1 <= n_scat <= 8192");
    return launch_line_combine(*p, rf, n_scat, amps, rf_line, S_(stream));
}

extern "C" int tidas_line_model(const tidas_line_params* p, const float* rf_line, int32_t s,
                                const float* theta, double eps, float* out, void* stream) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(rf_line && theta && out, "tidas_line_model: null pointer");
    TIDAS_REQUIRE(s >= 0 && s < p->n_depths, "tidas_line_model: curve outside the line");
    TIDAS_REQUIRE(eps > 0.0, "tidas_line_model: eps must be positive");
    return launch_line_model(*p, rf_line, s, theta, eps, out, S_(stream));
}

extern "C" int tidas_line_envelope(int32_t n_rows, int32_t n, const float* x, float* env,
                                   void* stream) {
    TIDAS_REQUIRE(x && env, "tidas_line_envelope: null pointer");
    TIDAS_REQUIRE(n_rows >= 1 && n_rows <= 65535 && n >= 1 && n <= 18000,
                  "tidas_line_envelope: need 1 <= n_rows <= 65535 and 1 <= n <= 18000");
    return launch_line_envelope(n_rows, n, x, env, S_(stream));
}

extern "C" int tidas_line_fixed(const tidas_line_params* p, const float* rf, int32_t r_first,
                                int32_t n_scat, int32_t s, double eps, float* out, void* stream) {
    int rc = validate_line(p);
    if (rc) return rc;
    TIDAS_REQUIRE(rf && out, "tidas_line_fixed: null pointer");
    TIDAS_REQUIRE(n_scat >= 1 && r_first >= 0 && r_first + n_scat <= p->n_depths,
                  "tidas_line_fixed: scatterers outside the line");
    TIDAS_REQUIRE(s >= 0 && s < p->n_depths, "tidas_line_fixed: curve outside the line");
    TIDAS_REQUIRE(eps > 0.0, "tidas_line_fixed: eps must be positive");
    return launch_line_fixed(*p, rf, r_first, n_scat, s, eps, out, S_(stream));
}
