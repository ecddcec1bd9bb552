"""Stored expected values (tests/golden, written by tests/golden/make_golden.py
from the FP64 oracle alone): the oracle must keep reproducing them, and the GPU
path must match them within its tolerances without running the oracle."""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name + ".json")) as f:
        return json.load(f)


# ------------------------------------------------------------------ oracle
def test_oracle_reproduces_stored_das_case():
    import oracle
    G = load("das_toy")
    O = oracle.Oracle(G["geometry"])
    rf = O.synthesize(np.array(G["pos"]), np.array(G["amp"]))
    np.testing.assert_allclose(rf[0, 5], G["rf_row_a0_n5"], rtol=1e-13, atol=1e-15)
    np.testing.assert_array_equal(O.delay_table(1)[0], np.array(G["delay_index_angle1"]))
    img = O.das(rf.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(img, G["das_image_of_fp32_rounded_data"], rtol=1e-12, atol=1e-14)


def test_oracle_reproduces_stored_kernels_and_line_pairs():
    import oracle
    from oracle.line import LineOracle
    K = load("row_kernels_toy")
    np.testing.assert_allclose(oracle.Oracle(K["geometry"]).psf_rows(K["taps"]), K["kernels"],
                               rtol=1e-12, atol=1e-15)
    L = load("line_sweep_toy")
    O = LineOracle(L["params"])
    assert O.eps() == L["eps"]
    for row in L["pairs"][:4]:
        S = O.synth(row["r"]).astype(np.float32).astype(np.float64)
        g = O.das_line(S)
        th, el, eg = O.sweep_pair(S, g, row["r"], row["s"], L["eps"])
        assert th == pytest.approx(row["theta"], rel=1e-10)
        assert el == pytest.approx(row["err_local"], rel=1e-9, abs=1e-14)
        assert eg == pytest.approx(row["err_global"], rel=1e-9, abs=1e-14)


def test_oracle_reproduces_stored_band_kernels_and_convolution():
    import oracle
    B = load("band_toy")
    k = oracle.Oracle(B["geometry"]).psf_patches(B["kz"], B["taps"])
    np.testing.assert_allclose(k, B["kernels"], rtol=1e-12, atol=1e-15)
    y = oracle.tidas_conv2d(np.array(B["kernels"], np.float32).astype(np.float64),
                            np.array(B["refl"]))
    np.testing.assert_allclose(y, B["band_conv_of_fp32_rounded_kernels"], rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------- GPU
@pytest.mark.gpu
def test_gpu_matches_stored_das_case():
    from .gpu_helpers import host, rel_l2, require_gpu, torch
    require_gpu()
    from paper_2507_15464_gb300.ops import DasPlan
    G = load("das_toy")
    P = DasPlan(G["geometry"])
    pos = torch.tensor(G["pos"], dtype=torch.float64, device="cuda")[None]
    amp = torch.tensor(G["amp"], dtype=torch.float32, device="cuda")[None]
    rf = P.synthesize(pos, amp)
    # the stored row is FP64; the GPU rounds amplitudes and sums to FP32
    assert rel_l2(host(rf)[0, 0, 5], np.array(G["rf_row_a0_n5"])) <= 1e-5
    np.testing.assert_array_equal(host(P.delay_table(1)[0]), np.array(G["delay_index_angle1"]))
    assert rel_l2(host(P.forward(rf))[0], np.array(G["das_image_of_fp32_rounded_data"])) <= 1e-5


@pytest.mark.gpu
def test_gpu_matches_stored_kernels_and_line_pairs():
    from .gpu_helpers import host, rel_l2, require_gpu
    require_gpu()
    from paper_2507_15464_gb300.ops import DasPlan, LineExperiment
    K = load("row_kernels_toy")
    k, _ = DasPlan(K["geometry"]).fit_kernels(K["taps"])
    assert rel_l2(host(k), np.array(K["kernels"])) <= 1e-5
    L = load("line_sweep_toy")
    E = LineExperiment(L["params"])
    assert E.window() == pytest.approx(L["eps"], rel=1e-15)
    rf = E.synthesize()
    g = E.das_lines(rf)
    th, el, eg = (host(t) for t in E.sweep(rf, g, L["eps"]))
    for row in L["pairs"]:
        r, s = row["r"], row["s"]
        assert th[s, r] == pytest.approx(row["theta"], rel=1e-4)
        assert el[s, r] == pytest.approx(row["err_local"], abs=1e-4)
        assert eg[s, r] == pytest.approx(row["err_global"], abs=1e-4)


@pytest.mark.gpu
def test_gpu_matches_stored_band_kernels_and_convolution():
    from .gpu_helpers import host, rel_l2, require_gpu, torch
    require_gpu()
    from paper_2507_15464_gb300 import capi, ops
    from paper_2507_15464_gb300.ops import DasPlan
    B = load("band_toy")
    k = DasPlan(B["geometry"]).fit_kernels_2d(B["kz"], B["taps"])
    assert rel_l2(host(k), np.array(B["kernels"])) <= 1e-5
    kern = torch.tensor(B["kernels"], dtype=torch.float32, device="cuda")
    refl = torch.tensor(B["refl"], dtype=torch.float32, device="cuda")[None]
    y = ops.tidas_forward_2d(kern, refl, variant=capi.VARIANT_DIRECT)
    assert rel_l2(host(y)[0], np.array(B["band_conv_of_fp32_rounded_kernels"])) <= 1e-5
