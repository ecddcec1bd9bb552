/*
 * tidas.h -- C ABI of the GB300 (sm_103a) Delay-and-Sum / tiDAS library.
 *
 * Method: C. Razzetta et al., "tiDAS: a time invariant approximation of the
 * Delay and Sum algorithm for biomedical ultrasound PSF reconstructions",
 * arXiv 2507.15464.  Each entry point cites the section / equation that
 * defines the operation it computes.
 *
 * Conventions shared by every call
 *  - Array arguments are DEVICE pointers owned by the caller, C-contiguous,
 *    with the layout given beside each argument.  The library never frees
 *    them and never keeps them after the call returns.  A plan owns only its
 *    own tables, freed by das_plan_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return without synchronising;
 *    outputs are overwritten, never accumulated into.
 *  - Every call returns TIDAS_OK (0) or a negative status; the text of the
 *    last error of the calling thread is returned by tidas_last_error().
 *    Argument errors are detected before anything is enqueued.  Kernels
 *    that wait on asynchronous copies or tensor-core completions use bounded
 *    waits: if one gives up, the kernel records it in a device flag and
 *    returns; tidas_device_status() reads and clears that flag.
 *  - Geometry: linear array on z = 0, element centres
 *    x_n = (n - (n_elem-1)/2) * pitch (Section 2.1); pixel (ix, iz) at
 *    x = x0 + (ix + 1/2) dx, z = z0 + (iz + 1/2) dz; time of sample k is
 *    t0 + k / fs.  Transmit events are plane waves at angles_rad[a].
 *  - Channel data rf: [n_frames][n_angles][n_elem][n_samples], float32 or
 *    IEEE half (params.rf_dtype).  Images and reflectivity maps:
 *    [n_frames][nz][nx] float32 (x contiguous).
 *  - Counts (n_frames, grid and kernel sizes) must be >= 1; a zero count is
 *    TIDAS_ERR_ARG.  The one empty input that is valid is a scene without
 *    scatterers (das_synthesize with n_scat = 0, pos and amp may be NULL),
 *    whose channel data are all zero.
 */
#ifndef TIDAS_H
#define TIDAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TIDAS_OK 0
#define TIDAS_ERR_ARG (-1)         /* bad argument: null pointer, size, alignment, dtype */
#define TIDAS_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define TIDAS_ERR_TIMEOUT (-3)     /* a bounded device wait gave up (see tidas_device_status) */
#define TIDAS_ERR_UNSUPPORTED (-4) /* valid request the library does not implement */

#define TIDAS_RF_F32 0
#define TIDAS_RF_F16 1

#define TIDAS_INTERP_LINEAR 0
#define TIDAS_INTERP_CUBIC 1 /* Keys kernel, a = -0.5, samples floor(u)-1 .. floor(u)+2 */

#define TIDAS_VARIANT_DIRECT 0    /* FP32 direct convolution on CUDA cores */
#define TIDAS_VARIANT_GEMM_BF16 1 /* Toeplitz GEMM on tcgen05 tensor cores, BF16 in, FP32 acc */
#define TIDAS_VARIANT_GEMM_RESID 2 /* BF16 GEMM + low-part residual products, FP32 in/out */

/* Acquisition and reconstruction parameters (SI units). */
typedef struct {
    int32_t n_elem;            /* array elements */
    double pitch;              /* element spacing, m */
    double f0;                 /* pulse centre frequency, Hz */
    double fs;                 /* sampling rate, Hz */
    double c;                  /* speed of sound, m/s (Eq. (2.3)) */
    double frac_bw;            /* -6 dB fractional bandwidth of the Gaussian pulse */
    int32_t n_angles;          /* plane-wave transmit events */
    const double* angles_rad;  /* HOST array [n_angles]; copied by das_plan_create */
    int32_t n_samples;         /* samples per channel */
    double t0;                 /* time of sample 0, s */
    int32_t nx, nz;            /* image grid: lateral, axial pixel counts */
    double x0, dx, z0, dz;     /* grid origin and spacing, m */
    int32_t interp;            /* TIDAS_INTERP_* */
    double fnum;               /* receive f-number; <= 0: whole array, unit weights */
    int32_t rf_dtype;          /* TIDAS_RF_F32 or TIDAS_RF_F16 (channel-data storage) */
} das_params;

typedef struct das_plan_s* das_plan;

/* Validate `params`, copy them, and build the plan's device tables: per
 * (angle, column) and (angle, row) splits of the plane-wave transmit delay
 * into an integer sample and an FP32 fraction (built in FP64), per
 * (element, column) lateral offsets in samples, per-row depths.  Sizes:
 * 1 <= n_elem <= 1024, 1 <= n_angles <= 16, 4 <= n_samples <= 2^22,
 * 1 <= nx, nz <= 8192, dx, dz, pitch, c, fs, f0 > 0, 0 < frac_bw <= 2.
 * Synchronous (allocates and uploads).  *out_plan receives the handle. */
int das_plan_create(const das_params* params, das_plan* out_plan);

/* Free the plan's device tables.  Waits for the device first.  NULL is a no-op. */
int das_plan_destroy(das_plan plan);

/* Plan options.  DAS_OPT_TENSOR_CORES: 1 (default) runs das_forward of FP16
 * plans on the tcgen05 tensor cores when n_frames >= 16, every
 * (32 x 4-pixel tile, angle, element) window of samples fits 64 samples and
 * every window in use starts within 16376 samples of the record's start
 * (checked when the plan is built); 0 keeps every batch on CUDA cores.  The
 * tensor-core path rounds the apodized interpolation weights to FP16
 * (relative 2^-11).  It first repacks the batch into a staging buffer that
 * the plan owns (about the size of the channel data; allocated on first use
 * and grown when a larger batch arrives), so das_forward calls on one FP16
 * plan must not overlap in time (issue them on one stream, or synchronise). */
#define DAS_OPT_TENSOR_CORES 1
int das_plan_set_option(das_plan plan, int32_t option, int32_t value);

/* The samples of every channel record that das_forward weights: every
 * interpolation tap of every pixel (Eq. (2.2) with the plan's delays, Eq.
 * (2.3)) lies in [*first_sample, *first_sample + *n_samples) (the extreme
 * delays over the grid, with one sample of margin each side).  Samples
 * outside the window never change the image as long as they are finite:
 * they are not read, or (the tensor-core path's aligned windows) multiplied
 * by exact zeros. */
int das_plan_read_window(das_plan plan, int32_t* first_sample, int32_t* n_samples);

/* Host -> device copy of the read window of every record of a batch:
 * rf[f][a][n][k] = host_rf[f][a][n][k] for k in the window, other samples of
 * rf untouched (keep them finite, e.g. zeroed once).  host_rf is a HOST
 * pointer [n_frames][n_angles][n_elem][n_samples] of the plan's rf_dtype
 * (page-locked for the copy to be asynchronous), rf a DEVICE pointer of the
 * same layout.  One cudaMemcpy2DAsync on `stream`. */
int das_upload_window(das_plan plan, const void* host_rf, void* rf, int32_t n_frames,
                      void* stream);

/* Channel data of point scatterers under the Born approximation, Eq. (2.1):
 * rf[f][a][n][k] = sum_j Re(A_fj * p(t_k - tau_a,n(x_fj, z_fj))), with the
 * Gaussian-modulated pulse p (6 dB band f0(1 +- frac_bw/2), truncated at the
 * -60 dB envelope) and round-trip time of flight
 * tau = (x sin(theta_a) + z cos(theta_a) + sqrt((x - x_n)^2 + z^2)) / c.
 *   pos_xz [n_frames][n_scat][2] float64 (x, z), metres
 *   amp    [n_frames][n_scat][2] float32 (Re A, Im A)
 *   rf     [n_frames][n_angles][n_elem][n_samples], plan's rf_dtype (output)
 * Delays are evaluated in FP64 per (scatterer, angle, element); samples are
 * accumulated in FP32 (summation order is not fixed). */
int das_synthesize(das_plan plan, const double* pos_xz, const float* amp, int32_t n_scat,
                   int32_t n_frames, void* rf, void* stream);

/* Eq. (2.1) for real reflectivities sitting on the pixel centres (the
 * forward operator A of deconvolution):
 *   refl [n_frames][nz][nx] float32 -> rf [n_frames][n_angles][n_elem][n_samples]
 * (rf_dtype must be TIDAS_RF_F32).  Transpose of das_synthesize_adjoint to FP32
 * rounding. */
int das_synthesize_grid(das_plan plan, const float* refl, void* rf, int32_t n_frames,
                        void* stream);

/* Transpose of das_synthesize_grid (A^T): every pixel correlates the channel
 * data with the pulse delayed to its own round-trip time:
 *   rf [n_frames][n_angles][n_elem][n_samples] float32 -> refl [n_frames][nz][nx] float32
 * The correlation over the pulse's core taps is evaluated from per-sample moments and
 * a ten-term series of the envelope's cross term whose remainder is below 1e-8 of the
 * sum of |tap| (under FP32 rounding); it allocates about 10 complex values per
 * channel sample of stream-ordered scratch for the call. */
int das_synthesize_adjoint(das_plan plan, const void* rf, float* refl, int32_t n_frames,
                           void* stream);

/* Delay and Sum, Eq. (2.2), compounded coherently over the angles:
 * img[f][iz][ix] = sum_a sum_n w_n(x, z) * S_{f,a,n}(u), with
 * u = (tau_tx + tau_rx - t0) fs samples, S sampled with the plan's
 * interpolation (zero outside [0, n_samples)), and the Hann receive
 * aperture w = cos^2(pi (x - x_n) F# / z) for |x - x_n| <= z / (2 F#)
 * (Section 3.1 fixes the f-number).  Accumulation is FP32.
 *   rf  [n_frames][n_angles][n_elem][n_samples], plan's rf_dtype
 *   img [n_frames][nz][nx] float32 (output)
 * Every plan restages the channel data in a staging buffer the plan owns,
 * allocated on first use and grown for larger batches: the Keys / linear
 * polynomial coefficients of every sample interval in the read window (FP32,
 * for up to 6 FP32 or 4 FP16 frames), frames innermost (FP16, 5 to 15
 * frames) or the tensor-core repack (FP16, >= 16 frames, see
 * DAS_OPT_TENSOR_CORES); FP32 batches of 7 or more frames are read in place.
 * das_forward calls on one plan must therefore not overlap in time (issue
 * them on one stream, or synchronise). */
int das_forward(das_plan plan, const void* rf, float* img, int32_t n_frames, void* stream);

/* Transpose of das_forward (B^T), for FP32 channel data plans:
 *   img [n_frames][nz][nx] float32 -> rf [n_frames][n_angles][n_elem][n_samples] float32
 * Each channel sample receives w * (interpolation weight) * img from the
 * pixels that read it.  The contributions are summed with shared-memory
 * atomics, so their order is not fixed: repeated calls agree to FP32
 * rounding, not necessarily bit for bit. */
int das_adjoint(das_plan plan, const float* img, float* rf, int32_t n_frames, void* stream);

/* Delay-index table of one angle, the integer/fraction split of
 * u = ((x sin(theta) + z cos(theta) + sqrt((x - x_n)^2 + z^2)) / c - t0) * fs
 * evaluated in FP64 with every operation rounded separately (no fused
 * multiply-add), in that order; Eq. (2.3) generalised to steered plane waves:
 *   idx  [nz][nx][n_elem] int32  = floor(u)
 *   frac [nz][nx][n_elem] float32 = u - floor(u), rounded to nearest. */
int das_delay_table(das_plan plan, int32_t angle, int32_t* idx, float* frac, void* stream);

/* tiDAS kernels from exact single-scatterer PSFs (Sections 2.2-2.3,
 * Eq. (2.6)-(2.8)).  For every row iz a unit scatterer on pixel (ic, iz),
 * ic = nx / 2, is synthesised and beamformed by the plan's DAS; the kernel
 * of row iz is that PSF row at columns ic + t - taps/2, t = 0..taps-1.
 * ref_stride > 1: rows share the PSF of a reference row s (the middle row
 * of each block of ref_stride rows) scaled by the least-squares weight of
 * Eq. (2.12), theta = <h_s, h_iz> / <h_s, h_s>.
 *   kernels [nz][taps] float32 (output), theta [nz] float32 or NULL (output;
 *   all ones when ref_stride <= 1).  1 <= taps <= 255. */
int tidas_fit_kernels(das_plan plan, int32_t taps, int32_t ref_stride, float* kernels,
                      float* theta, void* stream);

/* tiDAS forward, the convolutional line model of Eq. (2.13) applied row by
 * row along the lateral axis with depth-dependent kernels:
 *   img[f][iz][ix] = sum_t h_iz[t] * refl[f][iz][ix - t + taps/2]   (zero outside)
 *   kernels [nz][taps] float32
 *   refl    [n_frames][nz][nx]: float32 (variants DIRECT, GEMM_RESID) or
 *           bfloat16 (variant GEMM_BF16)
 *   img     [n_frames][nz][nx] float32 (output)
 * GEMM variants: each row is Y[frames x nx] = R[frames x nx] * T(h_iz) with
 * T the banded Toeplitz matrix of the kernel, on tcgen05 tensor cores with
 * FP32 accumulation in tensor memory; they need taps <= 63, nx % 8 == 0 and
 * 16-byte aligned refl / img.  GEMM_RESID splits refl and kernels into BF16
 * high and low parts and adds the two first-order low-part products. */
int tidas_forward(const float* kernels, int32_t taps, int32_t nz, int32_t nx, const void* refl,
                  float* img, int32_t n_frames, int32_t variant, void* stream);

/* Transpose of tidas_forward (correlation with the same kernels):
 *   refl[f][iz][j] = sum_t h_iz[t] * img[f][iz][j + t - taps/2]
 * Argument types as tidas_forward with the roles of refl and img exchanged
 * (img is the input: bfloat16 for GEMM_BF16, else float32; refl is float32). */
int tidas_adjoint(const float* kernels, int32_t taps, int32_t nz, int32_t nx, const void* img,
                  float* refl, int32_t n_frames, int32_t variant, void* stream);

/* 2D band kernels (axial x lateral):
 * keep the PSF's axial extent that the row-wise kernels drop.  kernels
 * [nz][kz][taps] float32; slice u of row j is the image of a unit scatterer on
 * pixel (nx/2, j) at output row j + u - kz/2 and columns nx/2 + t - taps/2
 * (Sections 2.2-2.3, Eq. (2.6)-(2.7), with the axial dimension kept).
 * tidas_fit_kernels_2d computes them with the plan's exact DAS (FP64 delays;
 * columns outside the grid are zero, rows outside it are evaluated).
 * 1 <= kz <= 64, 1 <= taps <= 255. */
int tidas_fit_kernels_2d(das_plan plan, int32_t kz, int32_t taps, float* kernels, void* stream);

/* Eq. (2.13) with the 2D band kernels, every pixel of r adding its row's
 * single-scatterer image:
 *   img[f][i][x] = sum_{u, t} kernels[j][u][t] refl[f][j][x - t + taps/2],
 *                  j = i - u + kz/2 (rows and columns outside the grid skipped);
 * tidas_adjoint_2d is the transpose.  variant: TIDAS_VARIANT_DIRECT (FP32
 * CUDA cores, refl float32) or TIDAS_VARIANT_GEMM_BF16 (tcgen05 Toeplitz
 * GEMMs over the kz input rows; refl BF16, taps <= 63, nx % 8 == 0, 16-byte
 * aligned arrays).  nx <= 2048.
 * workspace: device scratch of at least tidas_band_workspace_bytes(nz, nx,
 * n_frames, variant) bytes, 16-byte aligned, owned by the caller and not
 * read or written by any other work on the stream until the call's kernels
 * end; NULL makes the call take it from the stream-ordered allocator and
 * release it after its kernels (0 bytes are needed by the direct variant). */
int tidas_forward_2d(const float* kernels, int32_t kz, int32_t taps, int32_t nz, int32_t nx,
                     const void* refl, float* img, int32_t n_frames, int32_t variant,
                     void* workspace, size_t workspace_bytes, void* stream);
int tidas_adjoint_2d(const float* kernels, int32_t kz, int32_t taps, int32_t nz, int32_t nx,
                     const void* img, float* refl, int32_t n_frames, int32_t variant,
                     void* workspace, size_t workspace_bytes, void* stream);
/* ------------------------------------------------------------------------
 * Single-line experiment of Section 3 (Eq. (2.8), (2.12), (2.13) in the
 * channel domain).  One image line on the array axis, x = 0, with n_depths
 * points z_i = z_first + (z_last - z_first) i / (n_depths - 1); scatterers
 * sit on these points.  Transmit: focused on the axis at z_focus by the
 * elements with |x_m| <= a_tx, a_tx = sqrt(z_focus (c / f0) / kossoff)
 * (Kossoff's criterion, normalised focal distance z_focus / (a_tx^2 /
 * lambda) = kossoff); element m fires at (z_focus - |focus - x_m|) / c.
 * Receive: the elements with |x_n| <= z / (2 fnum_rx) of the depth z being
 * focused, unit weights.  Pulse: as in das_params (f0, frac_bw), real part.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t n_elem;            /* linear array, x_n = (n - (n_elem - 1) / 2) pitch */
    double pitch, f0, fs, c, frac_bw;
    int32_t n_samples;         /* channel record length, sample k at t = k / fs */
    int32_t n_depths;          /* line points (>= 2) */
    double z_first, z_last;    /* metres */
    double z_focus;            /* transmit focus depth */
    double kossoff;            /* Kossoff parameter of the transmit aperture (0.6) */
    double fnum_rx;            /* receive F-number (1) */
    int32_t interp;            /* TIDAS_INTERP_* */
} tidas_line_params;

/* Channel data rf[n_scat][n_elem][n_samples] (FP32, overwritten) of a unit
 * scatterer on each line point r_first .. r_first + n_scat - 1 (Eq. (2.1),
 * (2.6)): S_n(t_k) = sum_{m in transmit aperture} p(t_k - fire_m -
 * |r - x_m| / c - |r - x_n| / c), summed over m in index order. */
int tidas_line_synthesize(const tidas_line_params* p, int32_t r_first, int32_t n_scat,
                          float* rf, void* stream);
/* DAS lines lines[n_scat][n_depths] of the channel data rf[n_scat][n_elem]
 * [n_samples] (Eq. (2.2) with dynamic receive focusing): point z_i sums,
 * over the receive aperture of z_i, S_n at sample (2 z_i / c - D_n(z_i)) fs,
 * D_n of Eq. (2.3), interpolated.  Uses a stream-ordered table of a few MB. */
int tidas_line_das(const tidas_line_params* p, const float* rf, int32_t n_scat, float* lines,
                   void* stream);
/* Sweep of Eq. (2.8) / (2.12) over every delay curve s = 0 .. n_depths - 1
 * for the scatterers on points r_first .. r_first + n_scat - 1, given their
 * channel data rf[n_scat][n_elem][n_samples] and DAS lines
 * lines[n_scat][n_depths]:
 *   a_s[i] = sum_{n in aperture(z_s)} S~_n((2 z_i / c - D_n(z_s)) fs),
 * S~_n = the samples within eps seconds of the scatterer's echo arrival on
 * channel n (z_r / c + |r - x_n| / c), zero elsewhere; b = a_r (its own
 * curve).  Outputs, [n_depths][n_scat] (row = delay curve s, column =
 * scatterer), FP32:
 *   theta     = <a_s, b> / <a_s, a_s>                   (Eq. (2.12); 0 if a_s = 0)
 *   err_local = sum_W (theta a_s - g)^2 / sum_W g^2,  W = {i : |z_i - z_r| <= c eps / 2}
 *   err_global= sum_i (theta a_s - g)^2 / sum_i g^2,  g the DAS line.
 * 2 eps fs + 1 must stay below 27 samples (TIDAS_ERR_UNSUPPORTED otherwise);
 * n_elem x 136 + n_depths x 40 bytes of shared memory must fit in 220 KB. */
int tidas_line_sweep(const tidas_line_params* p, const float* rf, const float* lines,
                     int32_t r_first, int32_t n_scat, double eps, float* theta,
                     float* err_local, float* err_global, void* stream);
/* The tiDAS reconstruction of every scatterer under one delay curve s
 * (Eq. (2.8) with its theta, Eq. (2.12)): out[n_scat][n_depths] (FP32) row
 * rs = theta a_s for the scatterer on point r_first + rs, with rf, eps and
 * the window as in tidas_line_sweep (theta = 0 where a_s vanishes). */
int tidas_line_fixed(const tidas_line_params* p, const float* rf, int32_t r_first, int32_t n_scat,
                     int32_t s, double eps, float* out, void* stream);
/* The window half-width of Section 3.2: half the FWHM of the DAS PSF at the
 * focal point.  There the transmit and receive delays align every
 * contribution, so the PSF's time profile is the pulse and
 * *eps = sqrt(ln 2 / alpha), alpha the envelope rate of the pulse. */
int tidas_line_window(const tidas_line_params* p, double* eps);
/* Channel data of a line of scatterers from unit-scatterer data (Eq. (2.1)
 * is linear in the reflectivity): rf_line[n][k] = sum_r amps[r]
 * rf[r][n][k] over rf[n_scat][n_elem][n_samples], amps[n_scat] (device);
 * summed in the order of r, zero amplitudes skipped.  n_scat <= 8192. */
int tidas_line_combine(const tidas_line_params* p, const float* rf, int32_t n_scat,
                       const float* amps, float* rf_line, void* stream);
/* Line model of Eq. (2.13) on line channel data rf_line[n_elem][n_samples]:
 *   out[i] = theta[i] * sum_{n in aperture(z_s)} S~^(i)_n((2 z_i / c - D_n(z_s)) fs),
 * S~^(i)_n the samples within eps of the echo arrival of point i on channel
 * n (the window of Eq. (2.8) for a scatterer on point i); theta[n_depths]
 * (device), typically row s of tidas_line_sweep's theta. */
int tidas_line_model(const tidas_line_params* p, const float* rf_line, int32_t s,
                     const float* theta, double eps, float* out, void* stream);
/* Envelope (modulus of the analytic signal) of n_rows real rows of length n
 * (x, env: [n_rows][n], device): the DFT with negative frequencies removed
 * and positive ones doubled, inverted.  n <= 18000. */
int tidas_line_envelope(int32_t n_rows, int32_t n, const float* x, float* env, void* stream);

/* Scratch bytes of the 2D band calls: the input repacked into the GEMM's
 * operand tiles (128 frames x 64 columns, 16 KB each, per row); 0 for
 * variants that need none or for invalid sizes. */
size_t tidas_band_workspace_bytes(int32_t nz, int32_t nx, int32_t n_frames, int32_t variant);

/* ------------------------------------------------------------------------
 * Deconvolution on the convolutional model (the use the paper names for it in
 * its abstract, introduction and conclusion): min_x 1/2 ||H x - b||^2 +
 * lambda ||x||_1 by FISTA, with H the exact DAS operator (das_forward after
 * das_synthesize_grid) or tiDAS (tidas_forward).  Vector kernels of the
 * iteration; n counts float32 elements. */

/* *out (DEVICE double) = sum_i a[i] * b[i], accumulated in FP64.  Per-block
 * partial sums live in a stream-ordered scratch allocation (cudaMallocAsync /
 * cudaFreeAsync on `stream`); the final sum runs in a fixed order. */
int tidas_dot(const float* a, const float* b, int64_t n, double* out, void* stream);

/* Same result as tidas_dot, without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot let a library allocate,
 * such as a streaming scanner pipeline that reserves its whole device budget
 * at start-up and treats later allocations as failures, or a host thread
 * that must not wait on an allocator.  The per-block partial sums live in a
 * fixed 32 KB device array inside the library (held on every GPU that loads
 * it until exit), so n is limited to 16,777,216 elements; larger n returns
 * TIDAS_ERR_ARG before anything is enqueued.  The first call on each device
 * looks up the array's device address (with that device current) and keeps
 * it; make that call before any stream capture.  A cudaDeviceReset destroys
 * the module that holds the array, so the kept address is then stale: do not
 * call this entry point after resetting a device it was used on.  All calls
 * share the array: calls that overlap on the GPU, for example on two
 * streams, race and give wrong sums. */
int tidas_dot_noalloc(const float* a, const float* b, int64_t n, double* out, void* stream);

/* *out (DEVICE double) = sum_i |a[i]|, FP64; scratch as tidas_dot. */
int tidas_asum(const float* a, int64_t n, double* out, void* stream);

/* One FISTA update, in place: z = y - step * grad; x' = sign(z) max(|z| - thresh, 0);
 * y = x' + beta (x' - x); x = x'.  step > 0, thresh >= 0. */
int tidas_fista_update(float* x, float* y, const float* grad, int64_t n, float step, float thresh,
                       float beta, void* stream);

/* out = alpha a + beta b (element-wise; out may alias a or b). */
int tidas_axpby(const float* a, const float* b, float* out, int64_t n, float alpha, float beta,
                void* stream);

/* ------------------------------------------------------------------------
 * Learned kernel generator.  The paper's conclusion names learned scaling
 * parameters Theta as the way forward; here a small MLP maps (x, z, F#,
 * transmit angle) to the row kernel, trained on exact PSFs.  These are its
 * training targets, its GEMM, and the small kernels of training and
 * inference.  BF16 arrays are passed as void*. */

/* Exact single-scatterer PSF rows (Section 2.2, Eq. (2.6)-(2.7)) for a batch
 * of acquisitions: samples [n][4] float64 = (x, z, F#, theta_rad), a unit
 * scatterer at (x, z), one plane wave at theta, receive f-number F#, the
 * plan's array, pulse, interpolation and lateral spacing dx.  out[i][t]
 * (row stride ldo >= taps, columns >= taps zeroed) = DAS value at
 * (x + (t - taps/2) dx, z).  If norm != NULL, rows are divided by the sum of
 * the apodization weights at (x, z), written to norm[i]. */
int tidas_psf_batch(das_plan plan, const double* samples, int32_t n, int32_t taps, float* out,
                    int32_t ldo, float* norm, void* stream);

/* Band patches of the same exact PSFs (Eq. (2.6)-(2.7) with the axial extent
 * kept): for sample i the image of its unit scatterer at rows
 * z + (u - kz/2) dz and columns x + (t - taps/2) dx, u < kz, t < taps, of the
 * plan's grid spacing, written to out[i][u * ldk + t] (zero for
 * taps <= t < ldk and columns >= kz * ldk); the row u = kz/2 equals
 * tidas_psf_batch's row.  norm as for tidas_psf_batch.  1 <= kz <= 64,
 * ldk >= taps, kz * ldk <= ldo <= 65536. */
int tidas_psf_batch_2d(das_plan plan, const double* samples, int32_t n, int32_t kz, int32_t taps,
                       int32_t ldk, float* out, int32_t ldo, float* norm, void* stream);


/* out[i] = sum of the receive apodization weights at (x, z) for F#
 * (samples as tidas_psf_batch; the kernel scale).  Evaluated in FP32. */
int tidas_apod_sum(das_plan plan, const double* samples, int64_t n, float* out, void* stream);

/* C[M x N] = act(A[M x K] * B[N x K]^T + bias[N]) on tcgen05 tensor cores.
 * A, B: row-major BF16 with K contiguous; FP32 accumulation.  K % 64 == 0,
 * N % 16 == 0, 16-byte aligned arrays.  bias: float[N] or NULL; relu != 0
 * applies max(., 0).  Outputs (either may be NULL): c32 float, c16 BF16,
 * row stride ldc (ldc % 8 == 0). */
int tidas_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                    const float* bias, int32_t relu, float* c32, void* c16, int32_t ldc,
                    void* stream);

/* out[cols][rows] = in[rows][cols]^T, BF16. */
int tidas_transpose_bf16(const void* in, int32_t rows, int32_t cols, void* out, void* stream);

/* dst[i] = src[idx[i]], i < n, for rows of row_bytes (multiple of 4) bytes. */
int tidas_gather_rows(const void* src, const int32_t* idx, int64_t n, int32_t row_bytes, void* dst,
                      void* stream);

/* ReLU backward: dpre = act > 0 ? dpost : 0 (act = post-ReLU activation, or
 * NULL for a plain copy); dpre32 (float, may be NULL) and dpre16 (BF16) outputs. */
int tidas_relu_backward(const float* dpost, const float* act, int64_t n, float* dpre32,
                        void* dpre16, void* stream);

/* db[j] = sum_i d[i * ld + j], i < rows, j < cols. */
int tidas_colsum(const float* d, int32_t rows, int32_t cols, int32_t ld, float* db, void* stream);

/* AdamW step `step` (>= 1) on FP32 master weights w[rows][cols] with moments
 * m, v and gradient g; refreshes the BF16 copy w16 and its transpose w16t
 * (either may be NULL). */
int tidas_adam(float* w, float* m, float* v, const float* g, int32_t rows, int32_t cols, float lr,
               float b1, float b2, float eps, float wd, int32_t step, void* w16, void* w16t,
               void* stream);

/* Mean squared error over the first cols_used columns: *loss (DEVICE double),
 * dpred = 2 (pred - target) / (rows cols_used), zero in unused columns.
 * Partial sums use stream-ordered scratch (cudaMallocAsync / cudaFreeAsync). */
int tidas_mse(const float* pred, const float* target, int32_t rows, int32_t cols_used, int32_t ldp,
              int32_t ldt, float* dpred, double* loss, void* stream);

/* Network inputs: out16[i][0..63] = BF16(2 (s_ic - lo[c]) / (hi[c] - lo[c]) - 1)
 * for the 4 features of samples [n][4], zeros in columns 4..63.  lo4 / hi4
 * are DEVICE float[4]; out16 is 16-byte aligned. */
int tidas_encode(const double* samples, int32_t n, const float* lo4, const float* hi4, void* out16,
                 void* stream);

/* Fused inference of the kernel generator (the 4-layer MLP above), no
 * hidden activations in global memory:
 *   out[i][0..n_out-1] = scale[i] * (W4 relu(W3 relu(W2 relu(W1 x_i + b1) + b2) + b3) + b4)
 * with x_i the encoding of samples[i] (as tidas_encode; lo4 / hi4 are HOST
 * float[4] here), BF16 operands and activations, FP32 accumulation.
 * n_out = 64 for a row kernel, kz * 64 for a band patch of kz rows: one of
 * 64, 128, 192, 256, 512 (the last layer runs in output chunks of 256).
 *   w16  HOST array of 4 DEVICE pointers to the BF16 weights, row-major
 *        [out][in]: W1 [256][64], W2 [256][256], W3 [256][256], W4 [n_out][256]
 *   bias HOST array of 4 DEVICE pointers: b1, b2, b3 [256], b4 [n_out] float32
 *   scale DEVICE float[n] or NULL (all ones); out [n][ldo] float32,
 *   ldo >= n_out and a multiple of 4, 16-byte aligned. */
int tidas_mlp_infer(const double* samples, int64_t n, const float* lo4, const float* hi4,
                    const void* const* w16, const float* const* bias, const float* scale,
                    float* out, int32_t ldo, int32_t n_out, void* stream);

/* Spatially varying tiDAS: Eq. (2.13) with a kernel per pixel, the kernel of
 * pixel (j, s) being the single-scatterer image of that pixel (Eq. (2.6)-
 * (2.7)) over kz rows x taps columns centred on it.  Eq. (2.1) and (2.2) are
 * linear in the reflectivity, so every pixel of refl adds its own image,
 * scaled by its reflectivity (the kernel is the INPUT pixel's):
 *   img[f][i][x] = sum_{u, t} K[j][s][u][t] * refl[f][j][s],
 *                  j = i - u + kz/2,  s = x - t + taps/2,
 * rows and columns outside the grid contributing nothing.
 *   kernels  [nz][nx][kz][ld] float32, element (j, s, u, t) at
 *            ((j nx + s) kz + u) ld + t; 1 <= taps <= 64, ld >= taps,
 *            1 <= kz <= 64
 *   refl     [n_frames][nz][nx]: float32 for TIDAS_VARIANT_DIRECT (FP32 CUDA
 *            cores), bfloat16 for TIDAS_VARIANT_GEMM_BF16 (forward only:
 *            tcgen05 GEMMs, per output row and 128-column tile, over the kz
 *            slices and three 64-column input chunks, the B operand built
 *            from the chunk's per-pixel kernels rounded to BF16; FP32 sums;
 *            nx % 8 == 0, 16-byte aligned kernels, refl and img; kernels
 *            whose pitch ld is not a multiple of 4 are first copied to a
 *            padded stream-ordered scratch (ld % 4 == 0 avoids it); its stream-ordered
 *            scratch, the input repacked as for tidas_forward_2d, comes from
 *            cudaMallocAsync on `stream` and is freed after the call's kernels)
 *   img      [n_frames][nz][nx] float32 (overwritten)
 * tidas_forward_varying is the row form (kz = 1, kernels [nz * nx][ld],
 * FP32 direct).  tidas_adjoint_varying_2d (FP32 direct) is the transpose:
 * each pixel correlates img with its own kernel,
 * refl[f][j][s] = sum_{u,t} K[j][s][u][t] img[f][j+u-kz/2][s+t-taps/2].
 * Other variants return TIDAS_ERR_UNSUPPORTED.  Sums run in a fixed order. */
int tidas_forward_varying(const float* kernels, int32_t ld, int32_t taps, int32_t nz, int32_t nx,
                          const float* refl, float* img, int32_t n_frames, void* stream);
int tidas_forward_varying_2d(const float* kernels, int32_t ld, int32_t kz, int32_t taps,
                             int32_t nz, int32_t nx, const void* refl, float* img,
                             int32_t n_frames, int32_t variant, void* stream);
int tidas_adjoint_varying_2d(const float* kernels, int32_t ld, int32_t kz, int32_t taps,
                             int32_t nz, int32_t nx, const void* img, float* refl,
                             int32_t n_frames, int32_t variant, void* stream);
/* The tcgen05 form of tidas_forward_varying_2d with the per-pixel kernels
 * stored in BF16 (kernels16 [nz][nx][kz][ld] bfloat16, the same layout):
 * half the bytes of the dominant stream.  The builders otherwise round the
 * FP32 kernels to BF16 (round to nearest even), so kernels rounded the same
 * way give bit-identical images.  refl bfloat16; the GEMM variant's
 * conditions (nx % 8 == 0, 16-byte aligned arrays); kernels whose pitch ld
 * is not a multiple of 8 are first copied to a padded stream-ordered
 * scratch. */
int tidas_forward_varying_2d_bf16k(const void* kernels16, int32_t ld, int32_t kz, int32_t taps,
                                   int32_t nz, int32_t nx, const void* refl, float* img,
                                   int32_t n_frames, void* stream);

/* Per-pixel NRMSE of learned vs exact kernels (nrmse[p], may be NULL); out
 * takes the exact kernel where the NRMSE exceeds thresh, else the learned one. */
int tidas_kernel_fallback(const float* learned, int32_t ldl, const float* exact, int32_t lde,
                          int64_t npix, int32_t taps, float thresh, float* out, int32_t ldo,
                          float* nrmse, void* stream);

/* out[i][t] = in[i][t] * s[i] for t < cols (kernel de-normalisation). */
int tidas_row_scale(const float* in, int32_t ldi, const float* s, int64_t rows, int32_t cols,
                    float* out, int32_t ldo, void* stream);

/* Text of the calling thread's last error ("" if none). */
const char* tidas_last_error(void);

/* Synchronise the device, then read and clear the bounded-wait flag of the
 * tensor-core kernels: *status = 0 if no wait gave up since the last call,
 * otherwise a code naming the wait.  Returns TIDAS_ERR_TIMEOUT when set. */
int tidas_device_status(int32_t* status);

/* Failure-path test hooks (the paper has no counterpart).  They exist so that
 * a test can make a bounded device wait run out without faulting or hanging
 * the GPU, and check that the flag reaches tidas_device_status.  Both apply
 * to tidas_gemm_bf16 launches made after the call, process-wide:
 *   TIDAS_DEBUG_WAIT_LIMIT_NS  limit of that kernel's bounded waits, in ns
 *                              (default 1e9; 1e3 <= value <= 1e10)
 *   TIDAS_DEBUG_SKIP_COPIES    1: its producer issues no copies, so its MMA
 *                              thread's first wait runs out (code 202) with
 *                              nothing in flight and the output is left
 *                              unwritten; 0 (default): normal operation
 * Unknown options and out-of-range values return TIDAS_ERR_ARG. */
#define TIDAS_DEBUG_WAIT_LIMIT_NS 1
#define TIDAS_DEBUG_SKIP_COPIES 2
int tidas_set_debug_option(int32_t option, int64_t value);

#ifdef __cplusplus
}
#endif
#endif /* TIDAS_H */
