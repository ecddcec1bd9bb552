"""Single-line experiment of Section 3 -- TEST INFRASTRUCTURE ONLY.

FP64 oracle of the channel-domain tiDAS of Section 2.3 (Eq. (2.8), (2.12),
(2.13)) on one image line under a focused transmit (Section 3.1):
  - channel data of a unit scatterer on each line point (Eq. (2.1), (2.6));
  - the DAS line with dynamic receive focusing (Eq. (2.2), (2.3), (2.7));
  - the fixed-curve line of Eq. (2.8): the windowed channels aligned with
    the delay set of one line point s and summed;
  - the weight theta of Eq. (2.12) (first line, reading R13) and the local
    and global errors of Section 3.3 for every (delay curve s, scatterer r).
The C routines in tidas_oracle.c are plain loops; the metrics below are
plain sums.  Nothing here is shared with the GPU path.

Readings (the paper leaves these open):
  - Kossoff's criterion with parameter 0.6 sets the transmit half-aperture
    a_tx from z_focus / (a_tx^2 / lambda) = 0.6;
  - the window of Eq. (2.8) keeps, on each channel, the samples within eps
    of the scatterer's echo arrival on that channel;
  - eps = FWHM / 2 of the DAS PSF at the focal point.  There the transmit and
    receive delays align every contribution, so the PSF's time profile is
    the pulse itself and eps = sqrt(ln 2 / alpha) (closed form);
  - the local error of Section 3.3 uses the line points within c eps / 2 of
    the scatterer (the same window in depth), the global error all points;
    both are relative to the DAS line's energy in the same region;
  - the fixed-curve line uses the receive aperture of its own line point s.
"""
import ctypes

import numpy as np

from .core import _dp, _f64, lib as _core_lib


class LineParams(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int32), ("pitch", ctypes.c_double), ("f0", ctypes.c_double),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("frac_bw", ctypes.c_double),
        ("n_samples", ctypes.c_int32), ("n_depths", ctypes.c_int32),
        ("z_first", ctypes.c_double), ("z_last", ctypes.c_double),
        ("z_focus", ctypes.c_double), ("kossoff", ctypes.c_double),
        ("fnum_rx", ctypes.c_double), ("interp", ctypes.c_int32),
    ]


_P = ctypes.POINTER(LineParams)
_D = ctypes.POINTER(ctypes.c_double)
_SIG = {
    "orc_line_elem_x": (ctypes.c_double, [_P, ctypes.c_int]),
    "orc_line_depth": (ctypes.c_double, [_P, ctypes.c_int]),
    "orc_line_tx_radius": (ctypes.c_double, [_P]),
    "orc_line_tx_active": (ctypes.c_int, [_P, ctypes.c_int]),
    "orc_line_fire": (ctypes.c_double, [_P, ctypes.c_int]),
    "orc_line_rx_active": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "orc_line_delay": (ctypes.c_double, [_P, ctypes.c_int, ctypes.c_double]),
    "orc_line_arrival": (ctypes.c_double, [_P, ctypes.c_int, ctypes.c_double]),
    "orc_line_synth": (None, [_P, ctypes.c_int, _D]),
    "orc_line_das": (None, [_P, _D, _D]),
    "orc_line_in_window": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_long]),
    "orc_line_fixed": (None, [_P, _D, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]),
    "orc_line_model": (None, [_P, _D, ctypes.c_int, _D, ctypes.c_double, _D]),
}
_lib = None


def lib():
    global _lib
    if _lib is None:
        L = _core_lib()
        for name, (res, args) in _SIG.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class LineOracle:
    """The line experiment for one set of parameters (a dict with the
    LineParams fields)."""

    def __init__(self, p: dict):
        self.p = dict(p)
        self.P = LineParams(**{k: self.p[k] for k, _ in LineParams._fields_})
        self.L = lib()
        self.N, self.S, self.D = self.P.n_elem, self.P.n_samples, self.P.n_depths

    def _p(self):
        return ctypes.byref(self.P)

    # -- geometry -------------------------------------------------------------
    def elem_x(self, n):
        return self.L.orc_line_elem_x(self._p(), int(n))

    def depth(self, i):
        return self.L.orc_line_depth(self._p(), int(i))

    def depths(self):
        return np.array([self.depth(i) for i in range(self.D)])

    def tx_radius(self):
        return self.L.orc_line_tx_radius(self._p())

    def tx_active(self):
        return np.array([bool(self.L.orc_line_tx_active(self._p(), m)) for m in range(self.N)])

    def fire(self, m):
        return self.L.orc_line_fire(self._p(), int(m))

    def rx_active(self, n, z):
        return bool(self.L.orc_line_rx_active(self._p(), int(n), float(z)))

    def delay(self, n, z):
        """Eq. (2.3) for the on-axis point at depth z."""
        return self.L.orc_line_delay(self._p(), int(n), float(z))

    def arrival(self, n, z):
        return self.L.orc_line_arrival(self._p(), int(n), float(z))

    def alpha(self):
        half_bw = 0.5 * self.P.frac_bw * self.P.f0
        return np.pi ** 2 * half_bw ** 2 / np.log(10.0 ** (6.0 / 20.0))

    def eps(self):
        """Half the FWHM of the focal-point PSF, i.e. of the pulse envelope."""
        return float(np.sqrt(np.log(2.0) / self.alpha()))

    # -- signals --------------------------------------------------------------
    def synth(self, r):
        """Channel data [n_elem, n_samples] of a unit scatterer on point r."""
        out = np.empty((self.N, self.S))
        self.L.orc_line_synth(self._p(), int(r), _dp(out))
        return out

    def das_line(self, S):
        S = _f64(S)
        assert S.shape == (self.N, self.S)
        g = np.empty(self.D)
        self.L.orc_line_das(self._p(), _dp(S), _dp(g))
        return g

    def in_window(self, r, eps, n, k):
        return bool(self.L.orc_line_in_window(self._p(), int(r), float(eps), int(n), int(k)))

    def fixed_line(self, S, r, s, eps):
        """Fixed-curve line of curve s on the channels of scatterer r,
        windowed with half-width eps (eps < 0: no window)."""
        S = _f64(S)
        a = np.empty(self.D)
        self.L.orc_line_fixed(self._p(), _dp(S), int(r), int(s), float(eps), _dp(a))
        return a

    def line_data(self, amps):
        """Channel data of a line of scatterers: amps[r] on point r (Eq. (2.1)
        is linear in the reflectivity)."""
        S = np.zeros((self.N, self.S))
        for r in np.nonzero(amps)[0]:
            S += amps[r] * self.synth(r)
        return S

    def model_line(self, S, s, theta, eps):
        """Eq. (2.13): the line model with delay curve s and weights theta[i]."""
        S = _f64(S)
        th = _f64(theta)
        assert th.size == self.D
        out = np.empty(self.D)
        self.L.orc_line_model(self._p(), _dp(S), int(s), _dp(th), float(eps), _dp(out))
        return out

    def mainlobe_halfwidth(self):
        """Half-width in depth of a scatterer's main lobe: where the pulse
        envelope is 20 dB down, t = sqrt(ln 10 / alpha), two-way: c t / 2."""
        return self.P.c * np.sqrt(np.log(10.0) / self.alpha()) / 2.0

    # -- Eq. (2.12) and the errors of Section 3.3 -----------------------------
    def local_points(self, r, eps):
        z = self.depths()
        return np.abs(z - z[r]) <= self.P.c * eps / 2.0

    def sweep_pair(self, S, g, r, s, eps):
        """(theta, local error, global error) of delay curve s for scatterer r,
        S its channel data and g its DAS line."""
        a = self.fixed_line(S, r, s, eps)
        b = self.fixed_line(S, r, r, eps)
        aa = float(np.dot(a, a))
        theta = float(np.dot(a, b) / aa) if aa > 0.0 else 0.0
        d = theta * a - g
        w = self.local_points(r, eps)
        gl = float(np.dot(g[w], g[w]))
        e_loc = float(np.dot(d[w], d[w]) / gl) if gl > 0.0 else 0.0
        e_glob = float(np.dot(d, d) / np.dot(g, g))
        return theta, e_loc, e_glob


# the experiment's parameters and scenes are inputs, shared with the GPU side
from tidas_workloads.line_scenarios import paper_line, scenarios as line_scenarios  # noqa: E402,F401


# -- line-reconstruction metrics (Section 3.4, Table 3.1) -----------------------
def envelope(x):
    """|analytic signal| of a real sequence: the spectrum's negative
    frequencies removed, the positive ones doubled (discrete Hilbert
    transform)."""
    x = np.asarray(x, np.float64)
    n = x.size
    h = np.zeros(n)
    h[0] = 1.0
    if n % 2 == 0:
        h[n // 2] = 1.0
        h[1:n // 2] = 2.0
    else:
        h[1:(n + 1) // 2] = 2.0
    return np.abs(np.fft.ifft(np.fft.fft(x) * h))


def sidelobe_level_db(env, z, points, halfwidth):
    """Mean side-lobe level (dB): the mean envelope over the line points
    outside every scatterer's main lobe (|z - z_j| > halfwidth), relative to
    the envelope's maximum."""
    env = np.asarray(env, np.float64)
    z = np.asarray(z, np.float64)
    side = np.ones(z.size, bool)
    for j in points:
        side &= np.abs(z - z[j]) > halfwidth
    return float(20.0 * np.log10(env[side].mean() / env.max()))
