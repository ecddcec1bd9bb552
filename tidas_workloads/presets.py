"""Acquisition geometries of the benchmark workloads (parameters only).

Units are SI (metres, seconds, hertz).  Grid extents: the 64-element case
covers x in [-9.6, 9.6] mm, z in [5, 35] mm; the 128-element cases cover
x in [-19.2, 19.2] mm, z in [5, 60] mm.  Pixel centres are at
x0 + (i + 1/2) dx and z0 + (j + 1/2) dz.
"""
import math

_COMMON = dict(pitch=0.3e-3, f0=5.0e6, fs=40.0e6, c=1540.0, frac_bw=0.6, t0=0.0, fnum=1.5)

GEOMETRIES = {
    # 64 elements, one 0 degree plane wave, 128 x 256 pixels, linear interpolation
    "pw64_single": dict(_COMMON, n_elem=64, angles_deg=[0.0], n_samples=2048,
                        nx=128, nz=256, x0=-9.6e-3, dx=19.2e-3 / 128, z0=5.0e-3,
                        dz=30.0e-3 / 256, interp=0),
    # 128 elements, 11 plane waves -10..+10 degrees, 512 x 1024 pixels, cubic
    "pw128_compound": dict(_COMMON, n_elem=128, angles_deg=[-10.0 + 2.0 * a for a in range(11)],
                           n_samples=4096, nx=512, nz=1024, x0=-19.2e-3, dx=38.4e-3 / 512,
                           z0=5.0e-3, dz=55.0e-3 / 1024, interp=1),
    # same array on a 1024 x 1024 reflectivity / image grid (deconvolution)
    "pw128_deconv": dict(_COMMON, n_elem=128, angles_deg=[-10.0 + 2.0 * a for a in range(11)],
                         n_samples=4096, nx=1024, nz=1024, x0=-19.2e-3, dx=38.4e-3 / 1024,
                         z0=5.0e-3, dz=55.0e-3 / 1024, interp=1),
}


def angles_rad(geom: dict):
    return [a * math.pi / 180.0 for a in geom["angles_deg"]]


def geometry(name: str, **overrides) -> dict:
    """Copy of a named geometry with fields overridden (e.g. interp=0, nz=64)."""
    g = dict(GEOMETRIES[name])
    g.update(overrides)
    return g


def toy(n_elem=8, nx=6, nz=6, n_samples=128, angles_deg=(0.0,), interp=1, fnum=0.0, **kw) -> dict:
    """Tiny geometry for brute-force checks: a short array over a shallow grid."""
    g = dict(_COMMON, n_elem=n_elem, angles_deg=list(angles_deg), n_samples=n_samples,
             nx=nx, nz=nz, x0=-0.6e-3, dx=0.2e-3, z0=1.0e-3, dz=0.1e-3, interp=interp, fnum=fnum)
    g.update(kw)
    return g
