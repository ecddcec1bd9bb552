"""GPU parity of the DAS family (delay tables, synthesis, DAS, transposes, PSF
kernel fit) against the FP64 oracle, through the C ABI.

Tolerances: integer delay indices bit-exact; FP32 paths relative L2 <= 1e-5
against the oracle on identical input values; FP16 channel data <= 5e-3
against the oracle on the unquantised FP32 data; adjoint identities
<= 1e-6 relative with FP64 dot products.
"""
import numpy as np
import pytest

from tidas_workloads import generators, presets

from .gpu_helpers import dot64, dot_test, host, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def plan(geom, dtype=None):
    from paper_2507_15464_gb300.ops import DasPlan
    return DasPlan(geom, rf_dtype=dtype or torch.float32)


def oracle(geom):
    import oracle as orc
    return orc.Oracle(geom)


# ------------------------------------------------------------ delay tables
@pytest.mark.parametrize("name,angles", [("pw64_single", [0]), ("pw128_compound", [0, 3, 10])])
def test_delay_table_bit_exact(name, angles):
    g = presets.geometry(name)
    P, O = plan(g), oracle(g)
    for a in angles:
        idx, frac = P.delay_table(a)
        oi, of = O.delay_table(a)
        assert np.array_equal(host(idx), oi)
        assert np.array_equal(host(frac), of.astype(np.float32))


# --------------------------------------------------------------- synthesis
def test_synthesize_single_frame_real():
    g = presets.geometry("pw64_single")
    P, O = plan(g), oracle(g)
    pos, amp = generators.single_frame_speckle(0)
    rf = P.synthesize(to_dev(pos[None]), to_dev(amp[None]))
    ref = O.synthesize(pos, amp)
    assert rel_l2(host(rf)[0], ref) <= TOL32


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_synthesize_zero_scatterers_gives_zero_data(dtype):
    # the empty scene: no scatterer, every channel sample overwritten with 0
    g = presets.geometry("pw64_single")
    P = plan(g, dtype)
    pos = torch.zeros((2, 0, 2), dtype=torch.float64, device="cuda")
    amp = torch.zeros((2, 0, 2), dtype=torch.float32, device="cuda")
    out = torch.full(P.rf_shape(2), 7.0, dtype=dtype, device="cuda")
    rf = host(P.synthesize(pos, amp, out=out))
    assert rf.shape == (2, 1, 64, g["n_samples"]) and not rf.any()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_synthesize_compound_complex(dtype):
    g = presets.geometry("pw128_compound")
    P = plan(g, torch.float16 if dtype == "f16" else torch.float32)
    O = oracle(g)
    pos, amp = generators.point_scatterers(400, (-19.2e-3, 19.2e-3), (5e-3, 60e-3), (11, 0),
                                           real=False)
    pos2, amp2 = generators.point_scatterers(400, (-19.2e-3, 19.2e-3), (5e-3, 60e-3), (11, 1),
                                             real=False)
    rf = P.synthesize(to_dev(np.stack([pos, pos2])), to_dev(np.stack([amp, amp2])))
    out = host(rf)
    tol = TOL16 if dtype == "f16" else TOL32
    assert rel_l2(out[0], O.synthesize(pos, amp)) <= tol
    assert rel_l2(out[1], O.synthesize(pos2, amp2)) <= tol


# --------------------------------------------------------------------- DAS
def test_das_single_angle_linear_full_image():
    g = presets.geometry("pw64_single")
    P, O = plan(g), oracle(g)
    pos, amp = generators.single_frame_speckle(0)
    rf64 = O.synthesize(pos, amp)
    rf32 = rf64.astype(np.float32)
    img = host(P.forward(to_dev(rf32[None])))[0]
    ref = O.das(rf32)
    assert rel_l2(img, ref) <= TOL32
    # error against the FP64 channel data is reported alongside
    assert rel_l2(img, O.das(rf64)) <= TOL32


def _compound_rf_frames(O, nframes, n_scat=1500):
    out = []
    for f in range(nframes):
        pos, amp = generators.point_scatterers(n_scat, (-19.2e-3, 19.2e-3), (5e-3, 60e-3),
                                               (1, f), real=False)
        out.append(O.synthesize(pos, amp))
    return np.stack(out)


@pytest.mark.parametrize("nf", [1, 3])
def test_das_compound_cubic_fp32_sampled(nf):
    g = presets.geometry("pw128_compound")
    P, O = plan(g), oracle(g)
    rf = _compound_rf_frames(O, nf).astype(np.float32)
    img = host(P.forward(to_dev(rf)))
    rng = np.random.default_rng(7)
    for f in range(nf):
        pix = rng.choice(g["nx"] * g["nz"], 3000, replace=False)
        ref = O.das_pixels(rf[f], pix)
        assert rel_l2(img[f].ravel()[pix], ref) <= TOL32


def test_das_compound_fp16_channel_data():
    g = presets.geometry("pw128_compound")
    P16, O = plan(g, torch.float16), oracle(g)
    rf32 = _compound_rf_frames(O, 2).astype(np.float32)
    rf16 = rf32.astype(np.float16)
    img = host(P16.forward(to_dev(rf16)))
    rng = np.random.default_rng(8)
    for f in range(2):
        pix = rng.choice(g["nx"] * g["nz"], 3000, replace=False)
        same_input = O.das_pixels(rf16[f].astype(np.float64), pix)
        assert rel_l2(img[f].ravel()[pix], same_input) <= TOL32
        assert rel_l2(img[f].ravel()[pix], O.das_pixels(rf32[f], pix)) <= TOL16


# The tensor-core path (>= 16 FP16 frames) rounds the apodized interpolation
# weights to FP16: relative error <= 2^-11 per weight, ~2^-11/sqrt(3) = 2.8e-4
# rms over the ~650 terms of a pixel; bound 1e-3 against the oracle on the
# same channel data (and 5e-3 against unquantised data).
TOL_TC = 1e-3


def test_das_full_batch_fp16_sampled_frames():
    # the benchmark's launch configuration: 64 frames of FP16 channel data
    g = presets.geometry("pw128_compound")
    P16, O = plan(g, torch.float16), oracle(g)
    B = 64
    rf = np.empty((B, 11, 128, 4096), np.float16)
    for f in range(B):
        rf[f] = generators.standard_normal((11, 128, 4096), (21, f), np.float16)
    x = to_dev(rf)
    img = host(P16.forward(x))            # tensor cores
    P16.set_tensor_cores(False)
    img_cc = host(P16.forward(x))         # CUDA cores
    assert not np.array_equal(img, img_cc)
    rng = np.random.default_rng(9)
    for f in (0, 37, B - 1):
        pix = rng.choice(g["nx"] * g["nz"], 600, replace=False)
        ref = O.das_pixels(rf[f].astype(np.float64), pix)
        assert rel_l2(img[f].ravel()[pix], ref) <= TOL_TC
        assert rel_l2(img_cc[f].ravel()[pix], ref) <= TOL32
    assert rel_l2(img, img_cc) <= TOL_TC


@pytest.mark.parametrize("name,nf,over", [
    ("pw128_compound", 16, {}), ("pw128_compound", 20, {}),
    ("pw64_single", 16, {}), ("pw64_single", 17, dict(nx=100, nz=77, n_samples=1104)),
    ("pw64_single", 33, dict(interp=1, nx=64, nz=40, z0=6e-3)),
    ("pw128_compound", 64, dict(angles_deg=[-8.0, 0.0, 8.0], nx=80, nz=61, n_samples=2048))])
def test_das_tensor_core_path(name, nf, over):
    # ragged pixel tiles, ragged frame tiles, out-of-record windows (zero
    # margins), linear and cubic interpolation; one, three and eleven angles,
    # so that a round of two pairs spans one or several elements
    g = presets.geometry(name, **over)
    P16, O = plan(g, torch.float16), oracle(g)
    S = g["n_samples"]
    rf = generators.standard_normal((nf, len(g["angles_deg"]), g["n_elem"], S), (29, nf),
                                    np.float16)
    x = to_dev(rf)
    img = host(P16.forward(x))
    P16.set_tensor_cores(False)
    img_cc = host(P16.forward(x))
    assert rel_l2(img, img_cc) <= TOL_TC
    # FP16 weights against FP32 ones: equal images would mean no tensor cores ran
    assert not np.array_equal(img, img_cc)
    rng = np.random.default_rng(10)
    for f in (0, nf - 1):
        pix = rng.choice(g["nx"] * g["nz"], min(800, g["nx"] * g["nz"]), replace=False)
        ref = O.das_pixels(rf[f].astype(np.float64), pix)
        assert rel_l2(img[f].ravel()[pix], ref) <= TOL_TC


@pytest.mark.parametrize("interp", [0, 1])
def test_das_ragged_grid_and_out_of_record_taps(interp):
    # grid not a multiple of the 32 x 8 pixel tile, frames not a multiple of
    # the frame batch, and a record too short for the deepest pixels (their
    # taps read zeros outside the record)
    g = presets.geometry("pw64_single", nx=100, nz=77, interp=interp, n_samples=1100)
    P, O = plan(g), oracle(g)
    rf = generators.standard_normal((5, 1, 64, 1100), (22,), np.float32)
    img = host(P.forward(to_dev(rf)))
    for f in (0, 4):
        assert rel_l2(img[f], O.das(rf[f])) <= TOL32


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("interp", [0, 1])
def test_das_small_batches(dtype, interp):
    # batches of 2 .. 20 frames take every CUDA-core path: per-interval
    # coefficients with 1, 2 or 4 frames per thread (up to 6 FP32 / 4 FP16
    # frames), FP16 frames restaged innermost and read as frame vectors
    # (tiles of 8 or 16 frames, the last one ragged), and FP32 gathers in
    # place; a ragged grid whose deepest taps leave the record exercises the
    # bounds-checked variants.  Every frame must equal the single-frame path
    # (rounding order differs between the paths) and the oracle.
    g = presets.geometry("pw64_single", nx=100, nz=77, interp=interp, n_samples=1100)
    tdt = torch.float32 if dtype == "f32" else torch.float16
    P, O = plan(g, tdt), oracle(g)
    for nf in (2, 3, 4, 5, 6, 8, 9, 13, 20):
        rf = generators.standard_normal((nf, 1, 64, 1100), (23, nf), np.float32)
        x = to_dev(rf, tdt)
        img = host(P.forward(x))
        xs = host(x)  # the values the GPU sees (FP16-rounded for f16)
        for f in sorted({0, nf // 2, nf - 1}):
            one = host(P.forward(x[f:f + 1].contiguous()))[0]
            assert rel_l2(img[f], one) <= 1e-6, (nf, f)
            assert rel_l2(img[f], O.das(xs[f])) <= TOL32, (nf, f)


def test_das_full_aperture_no_fnum():
    # whole array, unit weights: receive excess paths reach ~360 samples, where
    # the FP32 split delay is least accurate; band-limited channel data
    g = presets.geometry("pw64_single", fnum=0.0, nz=64)
    P, O = plan(g), oracle(g)
    pos, amp = generators.single_frame_speckle(3)
    rf = np.stack([O.synthesize(pos, amp), O.synthesize(pos[::-1] * [[-1, 1]], amp)])
    rf = rf.astype(np.float32)
    img = host(P.forward(to_dev(rf)))
    for f in range(2):
        assert rel_l2(img[f], O.das(rf[f])) <= TOL32


# --------------------------------------------------------------- adjoints
@pytest.mark.parametrize("interp", [0, 1])
def test_das_adjoint_matches_oracle_and_identity(interp):
    g = presets.geometry("pw64_single", interp=interp, nz=96, n_samples=1500)
    P, O = plan(g), oracle(g)
    y = generators.standard_normal((2, 96, 128), (24,), np.float32)
    x = generators.standard_normal((2, 1, 64, 1500), (25,), np.float32)
    bty = host(P.adjoint(to_dev(y)))
    for f in range(2):
        assert rel_l2(bty[f], O.das_adjoint(y[f])) <= TOL32
    bx = host(P.forward(to_dev(x)))
    dot_test(bx, y, x, bty)


def test_das_adjoint_identity_compound():
    g = presets.geometry("pw128_compound", nz=160)
    P = plan(g)
    y = generators.standard_normal((1, 160, 512), (26,), np.float32)
    x = generators.standard_normal((1, 11, 128, 4096), (27,), np.float32)
    bx = host(P.forward(to_dev(x)))
    bty = host(P.adjoint(to_dev(y)))
    dot_test(bx, y, x, bty)


def test_synthesis_grid_and_adjoint():
    g = presets.geometry("pw64_single", nx=40, nz=24, z0=12e-3, n_samples=1600)
    P, O = plan(g), oracle(g)
    refl = generators.bernoulli_normal((2, 24, 40), 0.2, (28,))
    rf = host(P.synthesize_grid(to_dev(refl)))
    for f in range(2):
        assert rel_l2(rf[f], O.synth_grid(refl[f])) <= TOL32
    y = generators.standard_normal((2, 1, 64, 1600), (29,), np.float32)
    aty = host(P.synthesize_adjoint(to_dev(y)))
    for f in range(2):
        assert rel_l2(aty[f], O.synth_adjoint(y[f])) <= TOL32
    dot_test(rf, y, refl, aty)


def test_synthesis_grid_sparse_maps():
    # the gather stages only the nonzero pixels of each column and packs
    # consecutive columns up to nz pixels per pass: an all-zero frame, a
    # sparse frame with empty columns, a frame whose nonzeros fill some columns
    # completely (groups of one full column next to partial ones), and a dense
    # frame must each match the oracle; the all-zero frame gives exact zeros
    g = presets.geometry("pw64_single", nx=40, nz=24, z0=12e-3, n_samples=1600)
    P, O = plan(g), oracle(g)
    refl = np.zeros((4, 24, 40), np.float32)
    refl[1] = generators.bernoulli_normal((24, 40), 0.03, (41,))
    refl[1][:, 5:17] = 0.0  # empty columns
    mixed = generators.bernoulli_normal((24, 40), 0.4, (42,))
    mixed[:, 3] = generators.standard_normal((24,), (43,), np.float32)  # full columns
    mixed[:, 30] = generators.standard_normal((24,), (44,), np.float32)
    refl[2] = mixed
    refl[3] = generators.standard_normal((24, 40), (45,), np.float32)
    rf = host(P.synthesize_grid(to_dev(refl)))
    assert not rf[0].any()
    for f in (1, 2, 3):
        assert rel_l2(rf[f], O.synth_grid(refl[f])) <= TOL32, f


# ------------------------------------------------------------- kernel fit
def test_fit_kernels_single_angle_all_rows():
    g = presets.geometry("pw64_single")
    P, O = plan(g), oracle(g)
    k, th = P.fit_kernels(31)
    ref = O.psf_rows(31)
    assert rel_l2(host(k), ref) <= TOL32
    assert np.all(host(th) == 1.0)


def test_fit_kernels_shared_reference_theta():
    import oracle as orc
    g = presets.geometry("pw64_single", nz=40)
    P, O = plan(g), oracle(g)
    k, th = P.fit_kernels(31, ref_stride=8)
    rk, rth = O.fit_kernels(31, ref_stride=8)
    assert rel_l2(host(k), rk) <= TOL32
    np.testing.assert_allclose(host(th), rth, rtol=1e-5)
    assert orc.reference_row(12, 8, 40) == 12 and host(th)[12] == 1.0


def test_fit_kernels_compound_sampled_rows():
    g = presets.geometry("pw128_compound")
    P, O = plan(g), oracle(g)
    k = host(P.fit_kernels(63)[0])
    rows = list(range(0, 1024, 97)) + [1023]
    ref = O.psf_rows(63, rows=rows)
    assert rel_l2(k[rows], ref) <= TOL32


def test_streamer_overlapped_batches_equal_plain_forward():
    # the serving form: uploads / read-backs overlap the beamforming on
    # separate streams; every image equals the plain call on the same batch
    from paper_2507_15464_gb300.ops import DasStreamer
    g = presets.geometry("pw64_single", nz=64, z0=10e-3)
    P = plan(g, torch.float16)
    nf = 16
    batches = [torch.from_numpy(generators.standard_normal(P.rf_shape(nf), (50 + k,), np.float32))
               .to(torch.float16).pin_memory() for k in range(5)]
    outs = [torch.empty(P.img_shape(nf), dtype=torch.float32).pin_memory() for _ in range(5)]
    S = DasStreamer(P, nf)
    done = [S.submit(b, o) for b, o in zip(batches, outs)]
    done[-1].synchronize()
    torch.cuda.synchronize()
    for b, o in zip(batches, outs):
        np.testing.assert_array_equal(o.numpy(), host(P.forward(b.cuda())))


@pytest.mark.parametrize("big", [6.0e4, np.nan])
@pytest.mark.parametrize("dtype,nf", [("f16", 16), ("f16", 6), ("f16", 3), ("f32", 2), ("f32", 8)])
def test_read_window_holds_every_weighted_sample(dtype, nf, big):
    # samples outside the plan's read window, set to huge finite values or to
    # NaN (and infinities), leave the image bit for bit unchanged on every
    # path: the tensor cores (16 FP16 frames, whose repack zeroes every sample
    # outside the window), the per-interval coefficients (3 FP16 and 2 FP32
    # frames, which count samples outside the window as zero), and the
    # frames-innermost (6 FP16 frames) and in-place (8 FP32 frames) gathers,
    # which read none of them; and the windowed upload gives the same image as
    # a full one
    from paper_2507_15464_gb300 import capi
    g = presets.geometry("pw128_compound", nz=96, z0=20e-3)
    tdt = torch.float16 if dtype == "f16" else torch.float32
    P = plan(g, tdt)
    first, count = P.read_window()
    S = g["n_samples"]
    assert 0 < first and first + count < S  # a strict sub-window for this grid
    rf = generators.standard_normal(P.rf_shape(nf), (31, nf), np.float32)
    inside = rf.copy()
    inside[..., :first] = 0.0
    inside[..., first + count:] = 0.0
    outside = rf.copy()
    outside[..., :first] = big
    outside[..., first + count:] = -big if np.isfinite(big) else np.inf
    a = host(P.forward(to_dev(inside, tdt)))
    b = host(P.forward(to_dev(outside, tdt)))
    np.testing.assert_array_equal(a, b)
    host_rf = torch.from_numpy(outside).to(tdt).pin_memory()
    dev = torch.zeros(P.rf_shape(nf), dtype=tdt, device="cuda")
    capi.call("das_upload_window", P.handle, host_rf.data_ptr(), dev.data_ptr(), nf,
              torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(host(P.forward(dev)), a)
