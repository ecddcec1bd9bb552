/*
 * FP64 CPU oracle for Delay-and-Sum (DAS) and its time-invariant
 * approximation (tiDAS) -- TEST INFRASTRUCTURE ONLY.
 *
 * Paper: C. Razzetta et al., "tiDAS: a time invariant approximation of the
 * Delay and Sum algorithm for biomedical ultrasound PSF reconstructions",
 * arXiv 2507.15464.  Citations below name the paper's sections and
 * equations.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header or table with the GPU
 * path.  Every routine is a plain loop over the definition it cites: no
 * blocking, no fusion, no reordering of the arithmetic.  OpenMP only splits
 * independent outputs across threads.  The file is compiled with
 * -ffp-contract=off so that no a*b+c is ever fused, and sqrt / division are
 * the IEEE correctly rounded operations.
 *
 * Geometry (Section 2.1): a linear array of n_elem elements on z = 0 with
 * centres x_n = (n - (n_elem-1)/2) * pitch; the imaging plane is y = 0 and a
 * point is r = (x, z).  Pixel (ix, iz) sits at x = x0 + (ix + 1/2) dx,
 * z = z0 + (iz + 1/2) dz.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t n_elem;
    double pitch, f0, fs, c, frac_bw;
    int32_t n_angles;
    const double* angles; /* transmit plane-wave angles, radians */
    int32_t n_samples;
    double t0; /* time of sample 0, seconds */
    int32_t nx, nz;
    double x0, dx, z0, dz;
    int32_t interp; /* 0 linear, 1 cubic (Keys, a = -0.5) */
    double fnum;    /* receive f-number; <= 0 means the full array, unit weights */
} orc_geom;

/* ---------------------------------------------------------------- geometry */

double orc_elem_x(const orc_geom* g, int n) {
    return ((double)n - 0.5 * (double)(g->n_elem - 1)) * g->pitch;
}
double orc_pix_x(const orc_geom* g, int ix) { return g->x0 + ((double)ix + 0.5) * g->dx; }
double orc_pix_z(const orc_geom* g, int iz) { return g->z0 + ((double)iz + 0.5) * g->dz; }

/* ------------------------------------------------------------------- pulse
 * Transmitted pulse S^F of Eq. (2.1): a Gaussian-modulated sinusoid
 * env(t) * exp(i 2 pi f0 t), env(t) = exp(-alpha t^2).  The magnitude
 * spectrum of the modulated Gaussian is proportional to
 * exp(-pi^2 (f - f0)^2 / alpha); alpha is chosen so that it is 6 dB down
 * at f0 (1 +- frac_bw / 2).  The pulse is truncated where the envelope falls
 * below -60 dB.  The real part is the radio-frequency pulse. */
double orc_pulse_alpha(const orc_geom* g) {
    double half_bw = 0.5 * g->frac_bw * g->f0;
    return M_PI * M_PI * half_bw * half_bw / log(pow(10.0, 6.0 / 20.0));
}
double orc_pulse_halfwidth(const orc_geom* g) {
    return sqrt(log(pow(10.0, 60.0 / 20.0)) / orc_pulse_alpha(g));
}
/* complex pulse value at time t (seconds) */
static void pulse_c(const orc_geom* g, double alpha, double thalf, double t, double* re,
                    double* im) {
    if (fabs(t) > thalf) {
        *re = 0.0;
        *im = 0.0;
        return;
    }
    double env = exp(-alpha * t * t);
    double ph = 2.0 * M_PI * g->f0 * t;
    *re = env * cos(ph);
    *im = env * sin(ph);
}
void orc_pulse(const orc_geom* g, const double* t, int n, double* re, double* im) {
    double alpha = orc_pulse_alpha(g), thalf = orc_pulse_halfwidth(g);
    for (int i = 0; i < n; ++i) pulse_c(g, alpha, thalf, t[i], &re[i], &im[i]);
}

/* ----------------------------------------------------------------- delays
 * Round-trip time of flight for transmit angle a, element n and point
 * (x, z), expressed in samples of the channel data:
 *   tau_tx = (x sin(theta_a) + z cos(theta_a)) / c    plane-wave transmit
 *   tau_rx = sqrt((x - x_n)^2 + z^2) / c              receive, Eq. (2.3)
 *   u      = (tau_tx + tau_rx - t0) * fs.
 * Eq. (2.3) is the relative receive delay z/c - tau_rx of an on-axis point;
 * the absolute form is what aligns recorded samples.  The operations are
 * performed in exactly the order written. */
double orc_delay_samples(const orc_geom* g, int a, int n, double x, double z) {
    double th = g->angles[a];
    double sn = sin(th);
    double cs = cos(th);
    double ddx = x - orc_elem_x(g, n);
    double tx = x * sn + z * cs;
    double rx = sqrt(ddx * ddx + z * z);
    return ((tx + rx) / g->c - g->t0) * g->fs;
}

/* Receive delay of Eq. (2.3), seconds (negative or zero). */
double orc_receive_delay_eq23(const orc_geom* g, int n, double z) {
    double xn = orc_elem_x(g, n);
    return (z - sqrt(xn * xn + z * z)) / g->c;
}

/* Full delay table for one angle: idx[iz][ix][n] = floor(u), frac = u - floor(u). */
void orc_delay_table(const orc_geom* g, int a, int32_t* idx, double* frac) {
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < g->nz; ++iz) {
        double z = orc_pix_z(g, iz);
        for (int ix = 0; ix < g->nx; ++ix) {
            double x = orc_pix_x(g, ix);
            for (int n = 0; n < g->n_elem; ++n) {
                double u = orc_delay_samples(g, a, n, x, z);
                double fl = floor(u);
                size_t o = ((size_t)iz * g->nx + ix) * g->n_elem + n;
                idx[o] = (int32_t)fl;
                frac[o] = u - fl;
            }
        }
    }
}

/* ------------------------------------------------------------ apodization
 * Receive aperture by f-number (Section 3.1 keeps the f-number fixed):
 * element n is active for point (x, z) when |x - x_n| <= z / (2 F#); the
 * active elements are weighted by a Hann window cos^2(pi (x - x_n) F# / z).
 * fnum <= 0 selects the whole array with unit weights. */
double orc_apod(const orc_geom* g, int n, double x, double z) {
    if (g->fnum <= 0.0) return 1.0;
    double r = (x - orc_elem_x(g, n)) * g->fnum / z;
    if (fabs(r) > 0.5) return 0.0;
    double cw = cos(M_PI * r);
    return cw * cw;
}

/* ------------------------------------------------------------ interpolation
 * Fractional-delay sampling of one channel signal, S_n * delta_D in Eq. (2.2).
 * Samples outside [0, n_samples) are zero.
 *  linear: weights (1 - phi, phi) on samples floor(u), floor(u) + 1;
 *  cubic:  the Keys convolution kernel with a = -0.5 on floor(u)-1 .. floor(u)+2. */
double orc_keys(double s) {
    const double a = -0.5;
    double t = fabs(s);
    if (t <= 1.0) return (a + 2.0) * t * t * t - (a + 3.0) * t * t + 1.0;
    if (t < 2.0) return a * t * t * t - 5.0 * a * t * t + 8.0 * a * t - 4.0 * a;
    return 0.0;
}
static double sample_at(const orc_geom* g, const double* row, long m) {
    if (m < 0 || m >= g->n_samples) return 0.0;
    return row[m];
}
/* interpolation weight that sample m receives at fractional position u */
static double interp_weight(const orc_geom* g, double u, long m) {
    double fl = floor(u);
    if (g->interp == 0) {
        double phi = u - fl;
        if (m == (long)fl) return 1.0 - phi;
        if (m == (long)fl + 1) return phi;
        return 0.0;
    }
    if (m < (long)fl - 1 || m > (long)fl + 2) return 0.0;
    return orc_keys(u - (double)m);
}
double orc_interp(const orc_geom* g, const double* row, double u) {
    long fl = (long)floor(u);
    double acc = 0.0;
    for (long m = fl - 1; m <= fl + 2; ++m) acc += interp_weight(g, u, m) * sample_at(g, row, m);
    return acc;
}

/* -------------------------------------------------------------- synthesis
 * Channel data under the Born approximation, Eq. (2.1): every scatterer j at
 * (x_j, z_j) with complex amplitude A_j returns the transmitted pulse,
 * delayed by its round-trip time of flight, to every element:
 *   rf[a][n][k] = sum_j Re( A_j * p(t_k - tau_j,a,n) ),  t_k = t0 + k / fs.
 * The element impulse response is folded into the pulse (no attenuation,
 * directivity or spreading).  One frame; pos_xz[j] = (x, z),
 * amp_reim[j] = (Re A, Im A).  rf is overwritten. */
void orc_synthesize(const orc_geom* g, const double* pos_xz, const double* amp_reim, int n_scat,
                    double* rf) {
    double alpha = orc_pulse_alpha(g), thalf = orc_pulse_halfwidth(g);
    int nrow = g->n_angles * g->n_elem;
#pragma omp parallel for schedule(dynamic)
    for (int row = 0; row < nrow; ++row) {
        int a = row / g->n_elem, n = row % g->n_elem;
        double* out = rf + (size_t)row * g->n_samples;
        for (int k = 0; k < g->n_samples; ++k) out[k] = 0.0;
        for (int j = 0; j < n_scat; ++j) {
            double u = orc_delay_samples(g, a, n, pos_xz[2 * j], pos_xz[2 * j + 1]);
            double tau = u / g->fs; /* time of flight relative to t0 */
            long k_lo = (long)ceil((tau - thalf) * g->fs) - 1;
            long k_hi = (long)floor((tau + thalf) * g->fs) + 1;
            if (k_lo < 0) k_lo = 0;
            if (k_hi > g->n_samples - 1) k_hi = g->n_samples - 1;
            for (long k = k_lo; k <= k_hi; ++k) {
                double re, im;
                pulse_c(g, alpha, thalf, (double)k / g->fs - tau, &re, &im);
                out[k] += amp_reim[2 * j] * re - amp_reim[2 * j + 1] * im;
            }
        }
    }
}

/* Transpose of orc_synthesize for scatterers on the pixel grid with real
 * amplitudes: refl[iz][ix] = sum_{a,n,k} rf[a][n][k] * Re p(t_k - tau). */
void orc_synth_adjoint(const orc_geom* g, const double* rf, double* refl) {
    double alpha = orc_pulse_alpha(g), thalf = orc_pulse_halfwidth(g);
#pragma omp parallel for schedule(dynamic)
    for (int iz = 0; iz < g->nz; ++iz) {
        double z = orc_pix_z(g, iz);
        for (int ix = 0; ix < g->nx; ++ix) {
            double x = orc_pix_x(g, ix), acc = 0.0;
            for (int a = 0; a < g->n_angles; ++a)
                for (int n = 0; n < g->n_elem; ++n) {
                    const double* row = rf + ((size_t)a * g->n_elem + n) * g->n_samples;
                    double tau = orc_delay_samples(g, a, n, x, z) / g->fs;
                    long k_lo = (long)ceil((tau - thalf) * g->fs) - 1;
                    long k_hi = (long)floor((tau + thalf) * g->fs) + 1;
                    if (k_lo < 0) k_lo = 0;
                    if (k_hi > g->n_samples - 1) k_hi = g->n_samples - 1;
                    for (long k = k_lo; k <= k_hi; ++k) {
                        double re, im;
                        pulse_c(g, alpha, thalf, (double)k / g->fs - tau, &re, &im);
                        acc += row[k] * re;
                    }
                }
            refl[(size_t)iz * g->nx + ix] = acc;
        }
    }
}

/* ------------------------------------------------------------------- DAS
 * Delay and Sum, Eq. (2.2), compounded coherently over the transmit angles:
 *   img(x, z) = sum_a sum_n w_n(x, z) * S_{a,n}( u_{a,n}(x, z) ).
 * One frame; rf is [n_angles][n_elem][n_samples], img is [nz][nx]. */
static double das_pixel(const orc_geom* g, const double* rf, int ix, int iz) {
    double x = orc_pix_x(g, ix), z = orc_pix_z(g, iz), acc = 0.0;
    for (int a = 0; a < g->n_angles; ++a)
        for (int n = 0; n < g->n_elem; ++n) {
            double w = orc_apod(g, n, x, z);
            if (w == 0.0) continue;
            double u = orc_delay_samples(g, a, n, x, z);
            const double* row = rf + ((size_t)a * g->n_elem + n) * g->n_samples;
            acc += w * orc_interp(g, row, u);
        }
    return acc;
}
void orc_das(const orc_geom* g, const double* rf, double* img) {
#pragma omp parallel for schedule(dynamic)
    for (int iz = 0; iz < g->nz; ++iz)
        for (int ix = 0; ix < g->nx; ++ix) img[(size_t)iz * g->nx + ix] = das_pixel(g, rf, ix, iz);
}
/* DAS at a list of flat pixel indices iz * nx + ix (sampled checks at full size). */
void orc_das_pixels(const orc_geom* g, const double* rf, const int64_t* pix, int64_t npix,
                    double* out) {
#pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < npix; ++i)
        out[i] = das_pixel(g, rf, (int)(pix[i] % g->nx), (int)(pix[i] / g->nx));
}

/* Transpose of orc_das: every pixel sends w * (interpolation weight) * img
 * back to the samples it read.  Threads own disjoint rf rows. */
void orc_das_adjoint(const orc_geom* g, const double* img, double* rf) {
    int nrow = g->n_angles * g->n_elem;
#pragma omp parallel for schedule(dynamic)
    for (int row = 0; row < nrow; ++row) {
        int a = row / g->n_elem, n = row % g->n_elem;
        double* out = rf + (size_t)row * g->n_samples;
        for (int k = 0; k < g->n_samples; ++k) out[k] = 0.0;
        for (int iz = 0; iz < g->nz; ++iz) {
            double z = orc_pix_z(g, iz);
            for (int ix = 0; ix < g->nx; ++ix) {
                double x = orc_pix_x(g, ix);
                double w = orc_apod(g, n, x, z);
                if (w == 0.0) continue;
                double u = orc_delay_samples(g, a, n, x, z);
                long fl = (long)floor(u);
                double v = img[(size_t)iz * g->nx + ix];
                for (long m = fl - 1; m <= fl + 2; ++m) {
                    if (m < 0 || m >= g->n_samples) continue;
                    out[m] += w * interp_weight(g, u, m) * v;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ tiDAS
 * Convolutional line model, Eq. (2.13), applied row by row along the lateral
 * axis with a depth-dependent kernel h_z of `taps` coefficients whose index
 * `center` sits on the output pixel:
 *   y[z][x] = sum_t h_z[t] * r[z][x - t + center]     (r = 0 outside the row).
 * One frame; kernels [nz][taps], r and y [nz][nx]. */
void orc_tidas_conv(int nz, int nx, int taps, int center, const double* kernels, const double* r,
                    double* y) {
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix) {
            double acc = 0.0;
            for (int t = 0; t < taps; ++t) {
                int j = ix - t + center;
                if (j < 0 || j >= nx) continue;
                acc += kernels[(size_t)iz * taps + t] * r[(size_t)iz * nx + j];
            }
            y[(size_t)iz * nx + ix] = acc;
        }
}
/* Transpose of orc_tidas_conv: r[z][j] = sum_t h_z[t] * y[z][j + t - center]. */
void orc_tidas_conv_adjoint(int nz, int nx, int taps, int center, const double* kernels,
                            const double* y, double* r) {
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < nz; ++iz)
        for (int j = 0; j < nx; ++j) {
            double acc = 0.0;
            for (int t = 0; t < taps; ++t) {
                int ix = j + t - center;
                if (ix < 0 || ix >= nx) continue;
                acc += kernels[(size_t)iz * taps + t] * y[(size_t)iz * nx + ix];
            }
            r[(size_t)iz * nx + j] = acc;
        }
}

/* 2D band kernels (the PSF's axial extent kept): kernels[j][u][t] is the image
 * of a unit scatterer on row j at output row j + u - cz, column offset
 * t - cx from the scatterer.  Superposing the images of all pixels of r:
 *   y[i][x] = sum_{u, t} kernels[j][u][t] * r[j][x - t + cx],  j = i - u + cz,
 * rows j outside [0, nz) and columns outside [0, nx) contributing nothing.
 * kz = 1, cz = 0 is the row-wise convolution orc_tidas_conv. */
void orc_tidas_conv2d(int nz, int nx, int kz, int taps, int cz, int cx, const double* kernels,
                      const double* r, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nz; ++i)
        for (int x = 0; x < nx; ++x) {
            double acc = 0.0;
            for (int u = 0; u < kz; ++u) {
                int j = i - u + cz;
                if (j < 0 || j >= nz) continue;
                for (int t = 0; t < taps; ++t) {
                    int xs = x - t + cx;
                    if (xs < 0 || xs >= nx) continue;
                    acc += kernels[((size_t)j * kz + u) * taps + t] * r[(size_t)j * nx + xs];
                }
            }
            y[(size_t)i * nx + x] = acc;
        }
}
/* Transpose of orc_tidas_conv2d:
 *   r[j][xs] = sum_{u, t} kernels[j][u][t] * y[j + u - cz][xs + t - cx]. */
void orc_tidas_conv2d_adjoint(int nz, int nx, int kz, int taps, int cz, int cx,
                              const double* kernels, const double* y, double* r) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nz; ++j)
        for (int xs = 0; xs < nx; ++xs) {
            double acc = 0.0;
            for (int u = 0; u < kz; ++u) {
                int i = j + u - cz;
                if (i < 0 || i >= nz) continue;
                for (int t = 0; t < taps; ++t) {
                    int x = xs + t - cx;
                    if (x < 0 || x >= nx) continue;
                    acc += kernels[((size_t)j * kz + u) * taps + t] * y[(size_t)i * nx + x];
                }
            }
            r[(size_t)j * nx + xs] = acc;
        }
}

/* Spatially varying kernels (Eq. (2.13) with the kernel of every pixel its
 * own single-scatterer image, Eq. (2.6)-(2.7)): kernels[j][s][u][t] is the
 * image of a unit scatterer on pixel (row j, column s) at output row
 * j + u - cz, column s + t - cx.  Born superposition (Eq. (2.1) is linear in
 * the reflectivity, Eq. (2.2) is linear in the data) adds the images of all
 * pixels of r, each scaled by its reflectivity:
 *   y[i][x] = sum_{u, t} kernels[j][s][u][t] * r[j][s],
 *             j = i - u + cz,  s = x - t + cx,
 * rows and columns outside the grid contributing nothing.  The kernel is the
 * one of the INPUT pixel (j, s), the scatterer.  kz = 1, cz = 0 is the
 * row-wise form; with kernels equal along every row it is orc_tidas_conv2d
 * term for term (same loop order). */
void orc_tidas_conv_varying(int nz, int nx, int kz, int taps, int cz, int cx,
                            const double* kernels, const double* r, double* y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nz; ++i)
        for (int x = 0; x < nx; ++x) {
            double acc = 0.0;
            for (int u = 0; u < kz; ++u) {
                int j = i - u + cz;
                if (j < 0 || j >= nz) continue;
                for (int t = 0; t < taps; ++t) {
                    int s = x - t + cx;
                    if (s < 0 || s >= nx) continue;
                    acc += kernels[(((size_t)j * nx + s) * kz + u) * taps + t] *
                           r[(size_t)j * nx + s];
                }
            }
            y[(size_t)i * nx + x] = acc;
        }
}
/* Transpose of orc_tidas_conv_varying: every pixel correlates the output with
 * its own kernel,
 *   r[j][s] = sum_{u, t} kernels[j][s][u][t] * y[j + u - cz][s + t - cx]. */
void orc_tidas_conv_varying_adjoint(int nz, int nx, int kz, int taps, int cz, int cx,
                                    const double* kernels, const double* y, double* r) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nz; ++j)
        for (int s = 0; s < nx; ++s) {
            double acc = 0.0;
            for (int u = 0; u < kz; ++u) {
                int i = j + u - cz;
                if (i < 0 || i >= nz) continue;
                for (int t = 0; t < taps; ++t) {
                    int x = s + t - cx;
                    if (x < 0 || x >= nx) continue;
                    acc += kernels[(((size_t)j * nx + s) * kz + u) * taps + t] *
                           y[(size_t)i * nx + x];
                }
            }
            r[(size_t)j * nx + s] = acc;
        }
}

/* =========================================================================
 * Single-line experiment of Section 3 (focused transmit, one image line on
 * the array axis), in the channel domain of Eq. (2.8) -- Eq. (2.13).
 *
 * Geometry: the linear array above; the line is x = 0 with n_depths points
 * z_i = z_first + (z_last - z_first) i / (n_depths - 1) (Section 3.1: 600
 * points from 2 to 42 mm).  Scatterers sit on these points.
 *
 * Transmit (Section 3.1): focused on the axis at z_focus by the elements
 * with |x_m| <= a_tx, where Kossoff's criterion with parameter kappa fixes
 * the normalised focal distance z_focus / (a_tx^2 / lambda) = kappa, i.e.
 * a_tx = sqrt(z_focus lambda / kappa), lambda = c / f0.  Element m fires at
 * (z_focus - sqrt(x_m^2 + z_focus^2)) / c, so every wavelet reaches the
 * focus at z_focus / c.  Receive: the elements with |x_n| <= z / (2 F#) of
 * the depth z being focused (rectangular aperture, F# = fnum_rx).
 *
 * Channel data of a unit scatterer at (0, z_r), Eq. (2.1) / (2.6):
 *   S_n(t_k) = sum_{m active} p(t_k - fire_m - |r - x_m| / c - |r - x_n| / c),
 * t_k = k / fs, p the real pulse (envelope times cos), no spreading (R3).
 * ========================================================================= */
typedef struct {
    int32_t n_elem;
    double pitch, f0, fs, c, frac_bw;
    int32_t n_samples;
    int32_t n_depths;
    double z_first, z_last;
    double z_focus, kossoff, fnum_rx;
    int32_t interp; /* 0 linear, 1 cubic (Keys, a = -0.5) */
} orc_line;

static double line_alpha(const orc_line* L) {
    double half_bw = 0.5 * L->frac_bw * L->f0;
    return M_PI * M_PI * half_bw * half_bw / log(pow(10.0, 6.0 / 20.0));
}
static double line_thalf(const orc_line* L) {
    return sqrt(log(pow(10.0, 60.0 / 20.0)) / line_alpha(L));
}
double orc_line_elem_x(const orc_line* L, int n) {
    return ((double)n - 0.5 * (double)(L->n_elem - 1)) * L->pitch;
}
double orc_line_depth(const orc_line* L, int i) {
    return L->z_first + (L->z_last - L->z_first) * (double)i / (double)(L->n_depths - 1);
}
double orc_line_tx_radius(const orc_line* L) {
    return sqrt(L->z_focus * (L->c / L->f0) / L->kossoff);
}
int orc_line_tx_active(const orc_line* L, int m) {
    return fabs(orc_line_elem_x(L, m)) <= orc_line_tx_radius(L);
}
double orc_line_fire(const orc_line* L, int m) {
    double xm = orc_line_elem_x(L, m);
    return (L->z_focus - sqrt(xm * xm + L->z_focus * L->z_focus)) / L->c;
}
int orc_line_rx_active(const orc_line* L, int n, double z) {
    return fabs(orc_line_elem_x(L, n)) <= z / (2.0 * L->fnum_rx);
}
/* Eq. (2.3): receive delay of element n for the on-axis point at depth z */
double orc_line_delay(const orc_line* L, int n, double z) {
    double xn = orc_line_elem_x(L, n);
    return (z - sqrt(xn * xn + z * z)) / L->c;
}
/* echo arrival of the on-axis point at depth z on element n, with the
 * transmit arrival z / c of the focused beam on its axis */
double orc_line_arrival(const orc_line* L, int n, double z) {
    double xn = orc_line_elem_x(L, n);
    return z / L->c + sqrt(xn * xn + z * z) / L->c;
}

/* S[n][k] of a unit scatterer on line point r; S is overwritten */
void orc_line_synth(const orc_line* L, int r, double* S) {
    double alpha = line_alpha(L), thalf = line_thalf(L);
    double zr = orc_line_depth(L, r);
#pragma omp parallel for schedule(static)
    for (int n = 0; n < L->n_elem; ++n) {
        double xn = orc_line_elem_x(L, n);
        double rx = sqrt(xn * xn + zr * zr) / L->c;
        double* out = S + (size_t)n * L->n_samples;
        for (int k = 0; k < L->n_samples; ++k) out[k] = 0.0;
        for (int m = 0; m < L->n_elem; ++m) {
            if (!orc_line_tx_active(L, m)) continue;
            double xm = orc_line_elem_x(L, m);
            double tau = orc_line_fire(L, m) + sqrt(xm * xm + zr * zr) / L->c + rx;
            for (int k = 0; k < L->n_samples; ++k) {
                double t = (double)k / L->fs - tau;
                if (fabs(t) > thalf) continue;
                out[k] += exp(-alpha * t * t) * cos(2.0 * M_PI * L->f0 * t);
            }
        }
    }
}

static double line_interp(const orc_line* L, const double* row, double u) {
    long fl = (long)floor(u);
    double phi = u - (double)fl, acc = 0.0;
    if (L->interp == 0) {
        if (fl >= 0 && fl < L->n_samples) acc += (1.0 - phi) * row[fl];
        if (fl + 1 >= 0 && fl + 1 < L->n_samples) acc += phi * row[fl + 1];
        return acc;
    }
    for (long m = fl - 1; m <= fl + 2; ++m)
        if (m >= 0 && m < L->n_samples) acc += orc_keys(u - (double)m) * row[m];
    return acc;
}

/* DAS line (Eq. (2.2) with dynamic receive focusing): for every line point
 * z_i, sum over the receive aperture of z_i of S_n at the echo arrival
 * time of z_i, i.e. the aligned time 2 z_i / c minus D_n(z_i) of Eq. (2.3) */
void orc_line_das(const orc_line* L, const double* S, double* g) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < L->n_depths; ++i) {
        double zi = orc_line_depth(L, i), acc = 0.0;
        for (int n = 0; n < L->n_elem; ++n) {
            if (!orc_line_rx_active(L, n, zi)) continue;
            double u = (2.0 * zi / L->c - orc_line_delay(L, n, zi)) * L->fs;
            acc += line_interp(L, S + (size_t)n * L->n_samples, u);
        }
        g[i] = acc;
    }
}

/* Window of Eq. (2.8): the samples of channel n whose time lies within eps
 * of the echo arrival of line point r on that channel (chi^r = 1_B) */
int orc_line_in_window(const orc_line* L, int r, double eps, int n, long k) {
    double t = (double)k / L->fs - orc_line_arrival(L, n, orc_line_depth(L, r));
    return fabs(t) <= eps;
}

/* Fixed-curve line of Eq. (2.8) / (2.13) without theta:
 *   a[i] = sum_{n in aperture(z_s)} S~_n(2 z_i / c - D_n(z_s)),
 * S~_n = S_n times the window of scatterer r (eps < 0: no window).  The
 * delay set and the aperture are those of line point s for every z_i. */
void orc_line_fixed(const orc_line* L, const double* S, int r, int s, double eps, double* a) {
    double zs = orc_line_depth(L, s);
    double* Sw = (double*)malloc(sizeof(double) * (size_t)L->n_elem * L->n_samples);
    for (int n = 0; n < L->n_elem; ++n)
        for (long k = 0; k < L->n_samples; ++k) {
            size_t q = (size_t)n * L->n_samples + k;
            Sw[q] = (eps < 0.0 || orc_line_in_window(L, r, eps, n, k)) ? S[q] : 0.0;
        }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < L->n_depths; ++i) {
        double zi = orc_line_depth(L, i), acc = 0.0;
        for (int n = 0; n < L->n_elem; ++n) {
            if (!orc_line_rx_active(L, n, zs)) continue;
            double u = (2.0 * zi / L->c - orc_line_delay(L, n, zs)) * L->fs;
            acc += line_interp(L, Sw + (size_t)n * L->n_samples, u);
        }
        a[i] = acc;
    }
    free(Sw);
}

/* Line model of Eq. (2.13) on channel data S[n_elem][n_samples] of a whole
 * line (any scatterers): for every line point i,
 *   L_i = theta[i] * sum_{n in aperture(z_s)} S~^(i)_n((2 z_i / c - D_n(z_s)) fs),
 * S~^(i)_n = the samples of channel n within eps of the echo arrival of point
 * i (the window of Eq. (2.8) for a scatterer on point i).  Plain loops over
 * the interpolation taps, each tested against the window. */
void orc_line_model(const orc_line* L, const double* S, int s, const double* theta, double eps,
                    double* out) {
    double zs = orc_line_depth(L, s);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < L->n_depths; ++i) {
        double zi = orc_line_depth(L, i), acc = 0.0;
        for (int n = 0; n < L->n_elem; ++n) {
            if (!orc_line_rx_active(L, n, zs)) continue;
            double u = (2.0 * zi / L->c - orc_line_delay(L, n, zs)) * L->fs;
            double t_i = orc_line_arrival(L, n, zi);
            long fl = (long)floor(u);
            double phi = u - (double)fl;
            const double* row = S + (size_t)n * L->n_samples;
            for (long m = fl - 1; m <= fl + 2; ++m) {
                if (m < 0 || m >= L->n_samples) continue;
                if (!(fabs((double)m / L->fs - t_i) <= eps)) continue;
                double w;
                if (L->interp == 0)
                    w = (m == fl) ? 1.0 - phi : (m == fl + 1) ? phi : 0.0;
                else
                    w = orc_keys(u - (double)m);
                acc += w * row[m];
            }
        }
        out[i] = theta[i] * acc;
    }
}
