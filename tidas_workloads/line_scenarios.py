"""Inputs of the single-line experiment of Section 3 (no method arithmetic).

The line parameters follow Section 3.1: 600 points from 2 to 42 mm on the
axis, a transmit focus on it, Kossoff 0.6 transmit aperture and F# 1
receive; the array is 192 elements at 0.3 mm pitch sampled at 40 MHz.  The
line scenes follow Section 3.4, whose positions and amplitudes the paper
does not give.
"""
import numpy as np


def paper_line(f0=5e6, z_focus=25e-3, n_depths=600, n_elem=192, n_samples=2560):
    return dict(n_elem=n_elem, pitch=0.3e-3, f0=f0, fs=40e6, c=1540.0, frac_bw=0.6,
                n_samples=n_samples, n_depths=n_depths, z_first=2e-3, z_last=42e-3,
                z_focus=z_focus, kossoff=0.6, fnum_rx=1.0, interp=1)


def scenarios(n_depths=600):
    """Amplitude per line point: five unit scatterers at 10, 17.5, 25, 32.5
    and 40 mm; the same five with amplitudes 1..5 increasing with depth; 100
    unit scatterers on every 6th point from the first."""
    z = 2e-3 + 40e-3 * np.arange(n_depths) / (n_depths - 1)
    five = [int(np.argmin(np.abs(z - d))) for d in (10e-3, 17.5e-3, 25e-3, 32.5e-3, 40e-3)]
    out = {}
    a = np.zeros(n_depths)
    a[five] = 1.0
    out["5_uniform"] = a
    a = np.zeros(n_depths)
    a[five] = np.arange(1, 6, dtype=np.float64)
    out["5_increasing"] = a
    a = np.zeros(n_depths)
    a[0:n_depths:6] = 1.0
    out["100_uniform"] = a
    return out
