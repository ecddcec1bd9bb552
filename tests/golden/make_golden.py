"""Write the stored expected values under tests/golden from the FP64 oracle.

Run from the repository root:  python tests/golden/make_golden.py
Only oracle/ and the input recipes in tidas_workloads are called.  The
files hold small cases, each with the passage of the paper its values
follow; tests/test_golden.py checks that the oracle still reproduces them and
that the GPU path matches them within its tolerances.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.line import LineOracle  # noqa: E402
from tidas_workloads import presets  # noqa: E402


def das_case():
    # 16 elements, two plane waves (-5, 5 degrees), 12 x 10 pixels, cubic, F# 1.5;
    # three point scatterers with real and complex amplitudes
    g = presets.toy(n_elem=16, nx=12, nz=10, n_samples=256, angles_deg=(-5.0, 5.0), fnum=1.5,
                    z0=3.0e-3, dz=0.15e-3, dx=0.15e-3, x0=-0.9e-3)
    O = oracle.Oracle(g)
    pos = np.array([[-0.3e-3, 3.6e-3], [0.2e-3, 4.1e-3], [0.05e-3, 3.25e-3]])
    amp = np.array([[1.0, 0.0], [-0.6, 0.3], [0.8, -0.5]])
    rf = O.synthesize(pos, amp)
    img = O.das(rf.astype(np.float32).astype(np.float64))
    idx, frac = O.delay_table(1)
    return {
        "cite": "Eq. (2.1) synthesis, Eq. (2.2) DAS, Eq. (2.3) delays generalised to steered "
                "plane waves",
        "geometry": g, "pos": pos.tolist(), "amp": amp.tolist(),
        "delay_index_angle1": idx.tolist(),
        "das_image_of_fp32_rounded_data": img.tolist(),
        "rf_row_a0_n5": rf[0, 5].tolist(),
    }


def kernel_case():
    # row kernels (Section 2.2: the PSF row of a unit scatterer) on a shallow grid
    g = presets.toy(n_elem=16, nx=24, nz=6, n_samples=256, angles_deg=(0.0,), fnum=1.5,
                    z0=3.0e-3, dz=0.2e-3, dx=0.1e-3, x0=-1.2e-3)
    O = oracle.Oracle(g)
    return {"cite": "Eq. (2.6)-(2.7): exact single-scatterer PSF rows as 9-tap kernels",
            "geometry": g, "taps": 9, "kernels": O.psf_rows(9).tolist()}


def line_case():
    # the single-line experiment of Section 3 on a 41-point line
    p = dict(n_elem=64, pitch=0.3e-3, f0=5e6, fs=40e6, c=1540.0, frac_bw=0.6, n_samples=1536,
             n_depths=41, z_first=5e-3, z_last=25e-3, z_focus=15e-3, kossoff=0.6, fnum_rx=1.0,
             interp=1)
    O = LineOracle(p)
    eps = O.eps()
    rows = []
    for r in (8, 20, 33):
        S = O.synth(r)
        g = O.das_line(S.astype(np.float32).astype(np.float64))
        for s in (r - 3, r, r + 3, 20):
            th, el, eg = O.sweep_pair(S.astype(np.float32).astype(np.float64), g, r, s, eps)
            rows.append({"r": r, "s": s, "theta": th, "err_local": el, "err_global": eg})
    return {"cite": "Eq. (2.8) windowed fixed-curve line, Eq. (2.12) theta, Section 3.3 errors",
            "params": p, "eps": eps, "pairs": rows}


def band_case():
    # 2D band kernels (the PSF's axial extent kept, the paper's 2D outlook of
    # Section 4) and the band form of Eq. (2.13) on a small seeded map
    from tidas_workloads import generators
    g = presets.toy(n_elem=16, nx=24, nz=8, n_samples=256, angles_deg=(0.0,), fnum=1.5,
                    z0=3.0e-3, dz=0.1e-3, dx=0.1e-3, x0=-1.2e-3)
    O = oracle.Oracle(g)
    kz, taps = 3, 9
    k = O.psf_patches(kz, taps)
    refl = generators.bernoulli_normal((g["nz"], g["nx"]), 0.3, (9,))
    y = oracle.tidas_conv2d(k.astype(np.float32).astype(np.float64), refl)
    return {"cite": "Eq. (2.6)-(2.7) PSF of a unit scatterer kept over kz rows; Eq. (2.13) "
                    "summed over the band rows",
            "geometry": g, "kz": kz, "taps": taps, "kernels": k.tolist(),
            "refl": refl.tolist(), "band_conv_of_fp32_rounded_kernels": y.tolist()}


def main():
    for name, fn in (("das_toy", das_case), ("row_kernels_toy", kernel_case),
                     ("line_sweep_toy", line_case), ("band_toy", band_case)):
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(fn(), f, indent=1)
        print("wrote", name)


if __name__ == "__main__":
    main()
