"""Python face of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It wraps the C routines of tidas_oracle.c (plain loops in FP64)
and adds the parts that are naturally written with numpy: kernel fitting
(Section 2.2 single-scatterer PSF and the weight theta of Eq. (2.12)) and
error metrics.  Nothing here is shared with the GPU path.
"""
import ctypes
import os

import numpy as np

from .build_oracle import build_oracle
from tidas_workloads.presets import angles_rad

_lib = None


class Geom(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int32), ("pitch", ctypes.c_double), ("f0", ctypes.c_double),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("frac_bw", ctypes.c_double),
        ("n_angles", ctypes.c_int32), ("angles", ctypes.POINTER(ctypes.c_double)),
        ("n_samples", ctypes.c_int32), ("t0", ctypes.c_double),
        ("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("x0", ctypes.c_double), ("dx", ctypes.c_double),
        ("z0", ctypes.c_double), ("dz", ctypes.c_double),
        ("interp", ctypes.c_int32), ("fnum", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_G = ctypes.POINTER(Geom)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        sig = {
            "orc_elem_x": (ctypes.c_double, [_G, ctypes.c_int]),
            "orc_pix_x": (ctypes.c_double, [_G, ctypes.c_int]),
            "orc_pix_z": (ctypes.c_double, [_G, ctypes.c_int]),
            "orc_pulse_alpha": (ctypes.c_double, [_G]),
            "orc_pulse_halfwidth": (ctypes.c_double, [_G]),
            "orc_pulse": (None, [_G, _D, ctypes.c_int, _D, _D]),
            "orc_delay_samples": (ctypes.c_double, [_G, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_double, ctypes.c_double]),
            "orc_receive_delay_eq23": (ctypes.c_double, [_G, ctypes.c_int, ctypes.c_double]),
            "orc_delay_table": (None, [_G, ctypes.c_int, _I32, _D]),
            "orc_apod": (ctypes.c_double, [_G, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "orc_keys": (ctypes.c_double, [ctypes.c_double]),
            "orc_interp": (ctypes.c_double, [_G, _D, ctypes.c_double]),
            "orc_synthesize": (None, [_G, _D, _D, ctypes.c_int, _D]),
            "orc_synth_adjoint": (None, [_G, _D, _D]),
            "orc_das": (None, [_G, _D, _D]),
            "orc_das_pixels": (None, [_G, _D, _I64, ctypes.c_int64, _D]),
            "orc_das_adjoint": (None, [_G, _D, _D]),
            "orc_tidas_conv": (None, [ctypes.c_int] * 4 + [_D, _D, _D]),
            "orc_tidas_conv_adjoint": (None, [ctypes.c_int] * 4 + [_D, _D, _D]),
            "orc_tidas_conv2d": (None, [ctypes.c_int] * 6 + [_D, _D, _D]),
            "orc_tidas_conv2d_adjoint": (None, [ctypes.c_int] * 6 + [_D, _D, _D]),
            "orc_tidas_conv_varying": (None, [ctypes.c_int] * 6 + [_D, _D, _D]),
            "orc_tidas_conv_varying_adjoint": (None, [ctypes.c_int] * 6 + [_D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """FP64 reference for one acquisition geometry (a dict of presets.py form)."""

    def __init__(self, geom: dict):
        self.p = dict(geom)
        # the radian values come from the shared workload module, so both
        # sides hand identical doubles to sin() and cos()
        self._angles = _f64(angles_rad(geom))
        g = Geom()
        for k in ("n_elem", "n_samples", "nx", "nz", "interp"):
            setattr(g, k, int(geom[k]))
        for k in ("pitch", "f0", "fs", "c", "frac_bw", "t0", "x0", "dx", "z0", "dz", "fnum"):
            setattr(g, k, float(geom[k]))
        g.n_angles = len(self._angles)
        g.angles = _dp(self._angles)
        self.g = g
        self.L = lib()
        self.A, self.N, self.S = g.n_angles, g.n_elem, g.n_samples
        self.nx, self.nz = g.nx, g.nz

    # -- geometry ---------------------------------------------------------
    def elem_x(self, n):
        return self.L.orc_elem_x(ctypes.byref(self.g), int(n))

    def pix_x(self, ix):
        return self.L.orc_pix_x(ctypes.byref(self.g), int(ix))

    def pix_z(self, iz):
        return self.L.orc_pix_z(ctypes.byref(self.g), int(iz))

    def grid_xz(self):
        xs = np.array([self.pix_x(i) for i in range(self.nx)])
        zs = np.array([self.pix_z(i) for i in range(self.nz)])
        return xs, zs

    # -- pulse ------------------------------------------------------------
    def pulse_alpha(self):
        return self.L.orc_pulse_alpha(ctypes.byref(self.g))

    def pulse_halfwidth(self):
        return self.L.orc_pulse_halfwidth(ctypes.byref(self.g))

    def pulse(self, t):
        t = _f64(np.atleast_1d(t))
        re = np.empty_like(t)
        im = np.empty_like(t)
        self.L.orc_pulse(ctypes.byref(self.g), _dp(t), t.size, _dp(re), _dp(im))
        return re + 1j * im

    # -- delays / apodization / interpolation -----------------------------
    def delay_samples(self, a, n, x, z):
        return self.L.orc_delay_samples(ctypes.byref(self.g), int(a), int(n), float(x), float(z))

    def receive_delay_eq23(self, n, z):
        return self.L.orc_receive_delay_eq23(ctypes.byref(self.g), int(n), float(z))

    def delay_table(self, a):
        idx = np.empty((self.nz, self.nx, self.N), np.int32)
        frac = np.empty((self.nz, self.nx, self.N), np.float64)
        self.L.orc_delay_table(ctypes.byref(self.g), int(a), idx.ctypes.data_as(_I32), _dp(frac))
        return idx, frac

    def apod(self, n, x, z):
        return self.L.orc_apod(ctypes.byref(self.g), int(n), float(x), float(z))

    def keys(self, s):
        return self.L.orc_keys(float(s))

    def interp(self, row, u):
        row = _f64(row)
        assert row.size == self.S
        return self.L.orc_interp(ctypes.byref(self.g), _dp(row), float(u))

    # -- operators (one frame each; leading batch axes are looped) ---------
    def synthesize(self, pos, amp):
        """Channel data [A, N, S] of point scatterers, Eq. (2.1)."""
        pos = _f64(pos).reshape(-1, 2)
        amp = _f64(amp).reshape(-1, 2)
        rf = np.empty((self.A, self.N, self.S))
        self.L.orc_synthesize(ctypes.byref(self.g), _dp(pos), _dp(amp), pos.shape[0], _dp(rf))
        return rf

    def grid_positions(self):
        xs, zs = self.grid_xz()
        X, Z = np.meshgrid(xs, zs)
        return np.stack([X.ravel(), Z.ravel()], axis=1)

    def synth_grid(self, refl):
        """Channel data of real reflectivities sitting on the pixel centres."""
        refl = _f64(refl)
        if refl.ndim == 3:
            return np.stack([self.synth_grid(r) for r in refl])
        amp = np.zeros((refl.size, 2))
        amp[:, 0] = refl.ravel()
        return self.synthesize(self.grid_positions(), amp)

    def synth_adjoint(self, rf):
        rf = _f64(rf)
        if rf.ndim == 4:
            return np.stack([self.synth_adjoint(r) for r in rf])
        out = np.empty((self.nz, self.nx))
        self.L.orc_synth_adjoint(ctypes.byref(self.g), _dp(rf), _dp(out))
        return out

    def das(self, rf):
        """Delay and Sum image [nz, nx], Eq. (2.2)."""
        rf = _f64(rf)
        if rf.ndim == 4:
            return np.stack([self.das(r) for r in rf])
        assert rf.shape == (self.A, self.N, self.S)
        img = np.empty((self.nz, self.nx))
        self.L.orc_das(ctypes.byref(self.g), _dp(rf), _dp(img))
        return img

    def das_pixels(self, rf, flat_idx):
        rf = _f64(rf)
        flat_idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
        out = np.empty(flat_idx.size)
        self.L.orc_das_pixels(ctypes.byref(self.g), _dp(rf), flat_idx.ctypes.data_as(_I64),
                              flat_idx.size, _dp(out))
        return out

    def das_adjoint(self, img):
        img = _f64(img)
        if img.ndim == 3:
            return np.stack([self.das_adjoint(i) for i in img])
        rf = np.empty((self.A, self.N, self.S))
        self.L.orc_das_adjoint(ctypes.byref(self.g), _dp(img), _dp(rf))
        return rf

    # -- tiDAS kernel fitting (Sections 2.2-2.3, Eq. (2.12)) ---------------
    def center_column(self):
        return self.nx // 2

    def psf_rows(self, taps, rows=None, ic=None):
        """Exact single-scatterer PSF of every row iz: a unit scatterer on pixel
        (ic, iz) is synthesised (Eq. (2.1)) and beamformed (Eq. (2.2)); the
        row iz is returned at columns ic + k - taps//2, k = 0..taps-1
        (zero outside the grid)."""
        ic = self.center_column() if ic is None else ic
        rows = range(self.nz) if rows is None else rows
        half = taps // 2
        out = []
        for iz in rows:
            rf = self.synthesize([[self.pix_x(ic), self.pix_z(iz)]], [[1.0, 0.0]])
            cols = np.arange(ic - half, ic - half + taps)
            ok = (cols >= 0) & (cols < self.nx)
            vals = np.zeros(taps)
            vals[ok] = self.das_pixels(rf, iz * self.nx + cols[ok])
            out.append(vals)
        return np.array(out)

    def psf_patches(self, kz, taps, rows=None, ic=None):
        """2D band kernels: for every row j, the exact image of a unit scatterer
        on pixel (ic, j) (Eq. (2.1) then Eq. (2.2)) over output rows
        j + u - kz//2 (u = 0..kz-1, also outside the grid) and columns
        ic + t - taps//2 (zero outside the grid): kernels[j][u][t]."""
        ic = self.center_column() if ic is None else ic
        rows = range(self.nz) if rows is None else rows
        cz, half = kz // 2, taps // 2
        cols = np.arange(ic - half, ic - half + taps)
        ok = (cols >= 0) & (cols < self.nx)
        out = []
        for j in rows:
            rf = self.synthesize([[self.pix_x(ic), self.pix_z(j)]], [[1.0, 0.0]])
            # a grid of kz rows x taps columns centred on the scatterer
            patch = dict(self.p, nz=kz, z0=self.p["z0"] + (j - cz) * self.p["dz"],
                         nx=taps, x0=self.p["x0"] + (ic - half) * self.p["dx"])
            img = Oracle(patch).das(rf)
            img[:, ~ok] = 0.0
            out.append(img)
        return np.array(out)

    def fit_kernels(self, taps, ref_stride=1, rows=None):
        """Per-row kernels.  ref_stride == 1: the PSF row itself.  ref_stride > 1:
        rows share the PSF of a reference row s (the middle row of each block of
        ref_stride rows), scaled by the least-squares weight of Eq. (2.12)."""
        psf = self.psf_rows(taps, rows=range(self.nz))
        if ref_stride <= 1:
            return psf, np.ones(self.nz)
        kern = np.empty_like(psf)
        theta = np.empty(self.nz)
        for iz in range(self.nz):
            s = reference_row(iz, ref_stride, self.nz)
            theta[iz] = theta_ls(psf[s], psf[iz])
            kern[iz] = theta[iz] * psf[s]
        return kern, theta


def reference_row(iz, ref_stride, nz):
    """Middle row of the block of ref_stride rows that contains iz."""
    s = (iz // ref_stride) * ref_stride + ref_stride // 2
    return min(s, nz - 1)


def theta_ls(a, b):
    """Weight theta minimising ||theta a - b||^2, Eq. (2.12): by Plancherel the
    frequency-domain ratio Int Re(conj(a) b) / Int |a|^2 equals the
    time-domain ratio <a, b> / <a, a> for real signals."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.dot(a, b) / np.dot(a, a))


def theta_ls_freq(a, b):
    """Eq. (2.12) evaluated literally in the frequency domain (first line)."""
    A = np.fft.fft(np.asarray(a, np.float64))
    B = np.fft.fft(np.asarray(b, np.float64))
    num = np.sum(np.conj(A) * B + A * np.conj(B)).real
    den = 2.0 * np.sum(np.abs(A) ** 2)
    return float(num / den)


def tidas_conv(kernels, r, center=None):
    """Eq. (2.13) row-wise lateral convolution for [nz, nx] or [B, nz, nx] inputs."""
    kernels = _f64(kernels)
    r = _f64(r)
    nz, taps = kernels.shape
    center = taps // 2 if center is None else center
    if r.ndim == 3:
        return np.stack([tidas_conv(kernels, x, center) for x in r])
    y = np.empty_like(r)
    lib().orc_tidas_conv(nz, r.shape[1], taps, center, _dp(kernels), _dp(r), _dp(y))
    return y


def tidas_conv_adjoint(kernels, y, center=None):
    kernels = _f64(kernels)
    y = _f64(y)
    nz, taps = kernels.shape
    center = taps // 2 if center is None else center
    if y.ndim == 3:
        return np.stack([tidas_conv_adjoint(kernels, x, center) for x in y])
    r = np.empty_like(y)
    lib().orc_tidas_conv_adjoint(nz, y.shape[1], taps, center, _dp(kernels), _dp(y), _dp(r))
    return r


def tidas_conv2d(kernels, r):
    """2D band form of Eq. (2.13): every pixel of r adds its row's
    single-scatterer image kernels[j] (kz rows x taps columns, centred)."""
    kernels = _f64(kernels)
    r = _f64(r)
    nz, kz, taps = kernels.shape
    if r.ndim == 3:
        return np.stack([tidas_conv2d(kernels, x) for x in r])
    y = np.empty_like(r)
    lib().orc_tidas_conv2d(nz, r.shape[1], kz, taps, kz // 2, taps // 2, _dp(kernels), _dp(r),
                           _dp(y))
    return y


def tidas_conv2d_adjoint(kernels, y):
    kernels = _f64(kernels)
    y = _f64(y)
    nz, kz, taps = kernels.shape
    if y.ndim == 3:
        return np.stack([tidas_conv2d_adjoint(kernels, x) for x in y])
    r = np.empty_like(y)
    lib().orc_tidas_conv2d_adjoint(nz, y.shape[1], kz, taps, kz // 2, taps // 2, _dp(kernels),
                                   _dp(y), _dp(r))
    return r


def _varying_shape(kernels):
    """[nz, nx, taps] (row kernels) or [nz, nx, kz, taps] (band kernels) ->
    the 4-D array and its sizes."""
    kernels = _f64(kernels)
    if kernels.ndim == 3:
        kernels = kernels[:, :, None, :]
    nz, nx, kz, taps = kernels.shape
    return np.ascontiguousarray(kernels), nz, nx, kz, taps


def tidas_conv_varying(kernels, r):
    """Eq. (2.13) with a kernel per pixel: every pixel (j, s) of r adds r[j][s]
    times its own single-scatterer image kernels[j][s] (taps columns, or kz
    rows x taps columns, centred on the pixel).  [nz, nx] or [B, nz, nx]."""
    k, nz, nx, kz, taps = _varying_shape(kernels)
    r = _f64(r)
    if r.ndim == 3:
        return np.stack([tidas_conv_varying(k, x) for x in r])
    assert r.shape == (nz, nx)
    y = np.empty_like(r)
    lib().orc_tidas_conv_varying(nz, nx, kz, taps, kz // 2, taps // 2, _dp(k), _dp(r), _dp(y))
    return y


def tidas_conv_varying_adjoint(kernels, y):
    """Transpose of tidas_conv_varying: each pixel correlates y with its own kernel."""
    k, nz, nx, kz, taps = _varying_shape(kernels)
    y = _f64(y)
    if y.ndim == 3:
        return np.stack([tidas_conv_varying_adjoint(k, x) for x in y])
    assert y.shape == (nz, nx)
    r = np.empty_like(y)
    lib().orc_tidas_conv_varying_adjoint(nz, nx, kz, taps, kz // 2, taps // 2, _dp(k), _dp(y),
                                         _dp(r))
    return r


# -- metrics ----------------------------------------------------------------
def nrmse(y, ref):
    """||y - ref||_2 / ||ref||_2 in FP64."""
    y = np.asarray(y, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


def fwhm(profile, spacing=1.0):
    """Full width at half maximum of |profile| around its peak, with linear
    interpolation of the half-maximum crossings."""
    p = np.abs(np.asarray(profile, np.float64))
    k = int(np.argmax(p))
    half = 0.5 * p[k]
    lo = k
    while lo > 0 and p[lo - 1] > half:
        lo -= 1
    hi = k
    while hi < p.size - 1 and p[hi + 1] > half:
        hi += 1
    left = lo - 1 + (half - p[lo - 1]) / (p[lo] - p[lo - 1]) if lo > 0 else float(lo)
    right = hi + (p[hi] - half) / (p[hi] - p[hi + 1]) if hi < p.size - 1 else float(hi)
    return (right - left) * spacing
