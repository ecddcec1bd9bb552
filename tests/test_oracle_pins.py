"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed-form geometry (Pythagorean triples), the paper's delay identities
(Eq. (2.3), Eq. (2.5)), textbook kernel values, library routines (numpy's
FFT, interp, convolve, least squares), invariants (symmetry, linearity,
adjoint identities) and brute-force explicit matrices on toy problems.
"""
import math

import numpy as np
import pytest

from tidas_workloads import presets, generators

C, FS = 1540.0, 40.0e6
L = C / FS  # one sample of path length


def O(geom):
    import oracle
    return oracle.Oracle(geom)


# ----------------------------------------------------------------- pulse
def test_pulse_spectrum_is_6db_down_at_band_edges():
    o = O(presets.geometry("pw64_single"))
    dt = 1.0 / 2.0e9
    t = np.arange(-4096, 4096) * dt
    p = o.pulse(t).real
    spec = np.abs(np.fft.rfft(p, n=1 << 17))
    f = np.fft.rfftfreq(1 << 17, dt)
    s = lambda fq: np.interp(fq, f, spec)
    f0 = 5.0e6
    assert abs(f[np.argmax(spec)] - f0) < 0.02e6
    for edge in (0.7 * f0, 1.3 * f0):
        db = 20 * np.log10(s(edge) / s(f0))
        assert abs(db + 6.0) < 0.05, db


def test_pulse_centre_and_truncation():
    o = O(presets.geometry("pw64_single"))
    th = o.pulse_halfwidth()
    assert o.pulse(0.0)[0] == pytest.approx(1.0, abs=1e-15)
    env_edge = abs(o.pulse(th * (1 - 1e-9))[0])
    assert env_edge == pytest.approx(1e-3, rel=1e-6)  # -60 dB envelope
    assert o.pulse(th * (1 + 1e-6))[0] == 0
    assert o.pulse(-th * (1 + 1e-6))[0] == 0
    # even real part, odd imaginary part (zero-phase pulse)
    t = np.linspace(-th, th, 101)
    v = o.pulse(t)
    np.testing.assert_allclose(v.real, v.real[::-1], atol=1e-13)
    np.testing.assert_allclose(v.imag, -v.imag[::-1], atol=1e-13)


# ---------------------------------------------------------------- delays
def _one_pixel(n_elem, pitch, x, z, angles_deg=(0.0,), fnum=0.0, n_samples=64, interp=1):
    return dict(presets.toy(), n_elem=n_elem, pitch=pitch, nx=1, nz=1, dx=L, dz=L,
                x0=x - L / 2, z0=z - L / 2, angles_deg=list(angles_deg), fnum=fnum,
                n_samples=n_samples, interp=interp)


def test_delay_pythagorean_unsteered():
    # elements at +-3L, point at (0, 4L): transmit 4L + receive 5L = 9 samples
    o = O(_one_pixel(2, 6 * L, 0.0, 4 * L))
    assert o.elem_x(0) == pytest.approx(-3 * L) and o.elem_x(1) == pytest.approx(3 * L)
    for n in range(2):
        assert o.delay_samples(0, n, 0.0, 4 * L) == pytest.approx(9.0, abs=1e-12)
    # 5-12-13: elements at +-12L, point at (0, 5L) -> 5 + 13 = 18
    o = O(_one_pixel(2, 24 * L, 0.0, 5 * L))
    assert o.delay_samples(0, 1, 0.0, 5 * L) == pytest.approx(18.0, abs=1e-12)


def test_delay_pythagorean_steered():
    # sin(theta) = 0.6, cos(theta) = 0.8; point (3L, 4L): transmit path 5L.
    th = math.degrees(math.asin(0.6))
    o = O(_one_pixel(2, 6 * L, 3 * L, 4 * L, angles_deg=(th, -th)))
    # element at +3L sits right above the point: receive path 4L
    assert o.delay_samples(0, 1, 3 * L, 4 * L) == pytest.approx(9.0, abs=1e-12)
    # element at -3L: receive sqrt(36 + 16) L
    assert o.delay_samples(0, 0, 3 * L, 4 * L) == pytest.approx(5 + math.sqrt(52), abs=1e-12)
    # the opposite steering angle: transmit path 0.8*4 - 0.6*3 = 1.4 L
    assert o.delay_samples(1, 1, 3 * L, 4 * L) == pytest.approx(1.4 + 4.0, abs=1e-12)


def test_delay_mirror_symmetry():
    g = presets.geometry("pw128_compound")
    o = O(g)
    A, N = o.A, o.N
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, n = rng.integers(A), rng.integers(N)
        x, z = rng.uniform(-19e-3, 19e-3), rng.uniform(5e-3, 60e-3)
        u1 = o.delay_samples(a, n, x, z)
        u2 = o.delay_samples(A - 1 - a, N - 1 - n, -x, z)
        assert u1 == pytest.approx(u2, rel=1e-13)


def test_receive_delay_matches_eq23_on_axis():
    o = O(presets.geometry("pw128_compound", angles_deg=[0.0]))
    for z in (5e-3, 20e-3, 55e-3):
        for n in (0, 17, 64, 127):
            # absolute round trip for x = 0: z/c + tau_rx; Eq. (2.3): D_n = z/c - tau_rx
            u = o.delay_samples(0, n, 0.0, z)
            d_eq23 = o.receive_delay_eq23(n, z)
            assert 2 * z / C - u / FS == pytest.approx(d_eq23, rel=1e-12, abs=1e-18)


def test_delay_taylor_relative_variation_eq25():
    o = O(presets.geometry("pw128_compound", angles_deg=[0.0]))
    for z0 in (10e-3, 30e-3):
        for n in (0, 30, 100):
            xn = o.elem_x(n)
            if abs(xn) < 1e-9:
                continue
            h = 1e-6
            rel = (o.receive_delay_eq23(n, z0 + h) - o.receive_delay_eq23(n, z0)) / \
                o.receive_delay_eq23(n, z0)
            pred = -h / math.sqrt(xn ** 2 + z0 ** 2)
            assert rel == pytest.approx(pred, rel=1e-3)


def test_delay_flattens_with_depth():
    # Section 2.1: delay curves flatten as depth grows
    o = O(presets.geometry("pw128_compound", angles_deg=[0.0]))
    spread = [o.receive_delay_eq23(0, z) - o.receive_delay_eq23(63, z) for z in (5e-3, 20e-3, 60e-3)]
    assert abs(spread[0]) > abs(spread[1]) > abs(spread[2])


def test_delay_table_floor_and_fraction():
    o = O(presets.toy(nx=5, nz=4, n_elem=6, angles_deg=(-10.0, 7.0)))
    for a in range(2):
        idx, frac = o.delay_table(a)
        assert np.all(frac >= 0) and np.all(frac < 1)
        iz, ix, n = 3, 2, 4
        u = o.delay_samples(a, n, o.pix_x(ix), o.pix_z(iz))
        assert idx[iz, ix, n] == math.floor(u) and frac[iz, ix, n] == u - math.floor(u)


# ------------------------------------------------------------ apodization
def test_apodization_hann_aperture():
    o = O(presets.geometry("pw128_compound"))
    z = 30e-3
    xn = o.elem_x(40)
    assert o.apod(40, xn, z) == pytest.approx(1.0)
    # |x - xn| F# / z = 1/4 -> cos^2(pi/4) = 1/2
    assert o.apod(40, xn + 0.25 * z / 1.5, z) == pytest.approx(0.5, abs=1e-14)
    assert o.apod(40, xn - 0.25 * z / 1.5, z) == pytest.approx(0.5, abs=1e-14)
    assert o.apod(40, xn + 0.51 * z / 1.5, z) == 0.0
    # active aperture is z / F# wide: about 10 mm / 0.3 mm elements at z = 15 mm
    act = sum(o.apod(n, 0.0, 15e-3) > 0 for n in range(128))
    assert act in (33, 34)


# ---------------------------------------------------------- interpolation
def test_keys_kernel_textbook_values():
    o = O(presets.toy())
    assert o.keys(0.0) == 1.0
    for s in (1.0, -1.0, 2.0, -2.0, 2.5):
        assert o.keys(s) == pytest.approx(0.0, abs=1e-15)
    assert o.keys(0.5) == pytest.approx(0.5625)   # Catmull-Rom: 9/16
    assert o.keys(1.5) == pytest.approx(-0.0625)  # -1/16


def test_interpolation_reproduces_polynomials():
    g = presets.toy(n_samples=64)
    k = np.arange(64, dtype=np.float64)
    cub = O(g)
    lin = O(dict(g, interp=0))
    quad = 0.3 * k ** 2 - 2.0 * k + 5.0
    line = -1.5 * k + 4.0
    for u in (10.0, 10.25, 31.5, 40.9):
        assert cub.interp(quad, u) == pytest.approx(0.3 * u * u - 2.0 * u + 5.0, rel=1e-13)
        assert lin.interp(line, u) == pytest.approx(-1.5 * u + 4.0, rel=1e-13)
    rng = np.random.default_rng(0)
    row = rng.standard_normal(64)
    for u in (0.2, 7.7, 60.4):
        assert lin.interp(row, u) == pytest.approx(np.interp(u, k, row), rel=1e-13)
    # outside the record the samples are zero
    assert cub.interp(row, -3.5) == 0.0 and cub.interp(row, 66.0) == 0.0


# ------------------------------------------------------ synthesis and DAS
def test_point_on_sample_grid_beamforms_to_sum_of_weights():
    # 3-4-5 geometry: both echoes arrive exactly on sample 9, so DAS returns
    # sum_n w_n * p(0) = 2 exactly, for linear and cubic interpolation.
    for interp in (0, 1):
        o = O(_one_pixel(2, 6 * L, 0.0, 4 * L, interp=interp))
        rf = o.synthesize([[0.0, 4 * L]], [[1.0, 0.0]])
        assert np.argmax(rf[0, 0]) == 9 and np.argmax(rf[0, 1]) == 9
        assert o.das(rf)[0, 0] == pytest.approx(2.0, abs=1e-12)


def test_steered_point_beamforms_to_one_with_aperture():
    # only the element above the point lies inside the F# = 1 aperture
    th = math.degrees(math.asin(0.6))
    o = O(_one_pixel(2, 6 * L, 3 * L, 4 * L, angles_deg=(th,), fnum=1.0))
    assert o.apod(0, 3 * L, 4 * L) == 0.0 and o.apod(1, 3 * L, 4 * L) == 1.0
    rf = o.synthesize([[3 * L, 4 * L]], [[1.0, 0.0]])
    assert np.argmax(rf[0, 1]) == 9
    assert o.das(rf)[0, 0] == pytest.approx(1.0, abs=1e-12)


def test_complex_amplitude_shifts_carrier_phase():
    o = O(_one_pixel(2, 6 * L, 0.0, 4 * L))
    rf_re = o.synthesize([[0.0, 4 * L]], [[1.0, 0.0]])
    rf_im = o.synthesize([[0.0, 4 * L]], [[0.0, 1.0]])
    t = (np.arange(o.S) - 9) / FS
    p = o.pulse(t)
    np.testing.assert_allclose(rf_re[0, 0], p.real, atol=1e-14)
    np.testing.assert_allclose(rf_im[0, 0], -p.imag, atol=1e-14)  # Re(i p) = -Im p


@pytest.mark.parametrize("name,iz", [("pw64_single", 60), ("pw64_single", 200)])
def test_single_scatterer_focuses_on_its_pixel(name, iz):
    g = presets.geometry(name)
    o = O(g)
    ic = o.nx // 2 + 7
    rf = o.synthesize([[o.pix_x(ic), o.pix_z(iz)]], [[1.0, 0.0]])
    img = o.das(rf)
    win = np.abs(img[iz - 10:iz + 11, ic - 10:ic + 11])
    assert np.unravel_index(np.argmax(win), win.shape) == (10, 10)


def test_das_linear_matches_numpy_interp():
    g = presets.geometry("pw64_single", nz=24, z0=15e-3)
    o = O(g)
    pos, amp = generators.single_frame_speckle(0, n=30)
    pos[:, 1] = np.clip(pos[:, 1], 15e-3, 17.5e-3)
    rf = o.synthesize(pos, amp)
    img = o.das(rf)
    k = np.arange(o.S)
    for iz, ix in ((3, 10), (12, 64), (20, 120)):
        x, z = o.pix_x(ix), o.pix_z(iz)
        ref = sum(o.apod(n, x, z) * np.interp(o.delay_samples(0, n, x, z), k, rf[0, n])
                  for n in range(o.N))
        assert img[iz, ix] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_linearity_in_amplitudes():
    g = presets.toy(nx=5, nz=5, n_elem=6, angles_deg=(-5.0, 5.0))
    o = O(g)
    pos = np.array([[0.1e-3, 1.2e-3], [-0.3e-3, 1.45e-3]])
    a1 = np.array([[1.0, 0.5], [-0.2, 0.0]])
    a2 = np.array([[0.3, -1.0], [2.0, 0.7]])
    lhs = o.das(o.synthesize(pos, 2.0 * a1 - 3.0 * a2))
    rhs = 2.0 * o.das(o.synthesize(pos, a1)) - 3.0 * o.das(o.synthesize(pos, a2))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(lhs)


# --------------------------------------------------------------- adjoints
@pytest.mark.parametrize("interp", [0, 1])
def test_das_adjoint_identity(interp):
    g = presets.geometry("pw64_single", nz=40, z0=10e-3, interp=interp, n_samples=1024)
    o = O(g)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((o.A, o.N, o.S))
    y = rng.standard_normal((o.nz, o.nx))
    lhs = np.vdot(o.das(x), y)
    rhs = np.vdot(x, o.das_adjoint(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_synthesis_adjoint_identity():
    g = presets.toy(nx=6, nz=5, n_elem=4, angles_deg=(-8.0, 0.0, 8.0))
    o = O(g)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((o.nz, o.nx))
    y = rng.standard_normal((o.A, o.N, o.S))
    lhs = np.vdot(o.synth_grid(x), y)
    rhs = np.vdot(x, o.synth_adjoint(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("interp", [0, 1])
def test_explicit_das_matrix_transpose(interp):
    # brute force: columns of H from unit channel samples, rows of H^T from unit pixels
    g = presets.toy(nx=6, nz=6, n_elem=8, n_samples=128, interp=interp, fnum=1.0)
    o = O(g)
    S = o.A * o.N * o.S
    H = np.zeros((o.nz * o.nx, S))
    for k in range(S):
        e = np.zeros(S)
        e[k] = 1.0
        H[:, k] = o.das(e.reshape(o.A, o.N, o.S)).ravel()
    Ht = np.zeros((S, o.nz * o.nx))
    for p in range(o.nz * o.nx):
        e = np.zeros(o.nz * o.nx)
        e[p] = 1.0
        Ht[:, p] = o.das_adjoint(e.reshape(o.nz, o.nx)).ravel()
    np.testing.assert_allclose(Ht, H.T, atol=1e-14)
    # every pixel row holds <= 4 (cubic) or 2 (linear) taps per active element
    taps = 4 if interp else 2
    assert (np.count_nonzero(H, axis=1) <= taps * o.N).all()


def test_explicit_synthesis_matrix_transpose():
    g = presets.toy(nx=3, nz=3, n_elem=3, n_samples=128)
    o = O(g)
    P = o.nz * o.nx
    A = np.stack([o.synth_grid(np.eye(P)[p].reshape(o.nz, o.nx)).ravel() for p in range(P)], 1)
    S = o.A * o.N * o.S
    At = np.zeros((P, S))
    for k in range(S):
        e = np.zeros(S)
        e[k] = 1.0
        At[:, k] = o.synth_adjoint(e.reshape(o.A, o.N, o.S)).ravel()
    np.testing.assert_allclose(At, A.T, atol=1e-14)


# ------------------------------------------------------------- theta fit
def test_theta_least_squares_eq212():
    import oracle
    rng = np.random.default_rng(3)
    a = rng.standard_normal(63)
    b = 0.7 * a + 0.1 * rng.standard_normal(63)
    th = oracle.theta_ls(a, b)
    ref = np.linalg.lstsq(a[:, None], b, rcond=None)[0][0]
    assert th == pytest.approx(ref, rel=1e-13)
    # Plancherel: frequency-domain form of Eq. (2.12) equals the time-domain one
    assert oracle.theta_ls_freq(a, b) == pytest.approx(th, rel=1e-12)
    # the normal-equation residual is orthogonal to a; theta = 1 for b = a
    assert abs(np.dot(th * a - b, a)) < 1e-12 * np.dot(a, a)
    assert oracle.theta_ls(a, a) == pytest.approx(1.0, rel=1e-15)


# ------------------------------------------------------------ tiDAS conv
@pytest.mark.parametrize("taps", [31, 63, 4])
def test_tidas_conv_matches_numpy_convolve(taps):
    import oracle
    rng = np.random.default_rng(4)
    nz, nx = 5, 40
    h = rng.standard_normal((nz, taps))
    r = rng.standard_normal((nz, nx))
    y = oracle.tidas_conv(h, r)
    c = taps // 2
    for iz in range(nz):
        full = np.convolve(r[iz], h[iz])
        np.testing.assert_allclose(y[iz], full[c:c + nx], rtol=1e-13, atol=1e-13)
    # adjoint identity
    v = rng.standard_normal((nz, nx))
    lhs = np.vdot(y, v)
    rhs = np.vdot(r, oracle.tidas_conv_adjoint(h, v))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_tidas_kernel_reproduces_exact_psf_row():
    # by construction (Section 2.3): the fitted kernel convolved with the
    # fitting scatterer returns the exact DAS row through that scatterer
    import oracle
    g = presets.geometry("pw64_single")
    o = O(g)
    taps = 31
    rows = [40, 150]
    psf = o.psf_rows(taps, rows=rows)
    ic = o.center_column()
    for i, iz in enumerate(rows):
        rf = o.synthesize([[o.pix_x(ic), o.pix_z(iz)]], [[1.0, 0.0]])
        das_row = o.das_pixels(rf, iz * o.nx + np.arange(o.nx))
        r = np.zeros((1, o.nx))
        r[0, ic] = 1.0
        y = oracle.tidas_conv(psf[i:i + 1], r)[0]
        sl = slice(ic - taps // 2, ic + taps // 2 + 1)
        np.testing.assert_allclose(y[sl], das_row[sl], rtol=1e-13, atol=1e-13)
        assert np.all(y[:sl.start] == 0) and np.all(y[sl.stop:] == 0)


# ---------------------------------------------- 2D band kernels (axial x lateral)
def test_tidas_conv2d_kz1_is_the_rowwise_convolution():
    import oracle
    rng = np.random.default_rng(7)
    h = rng.standard_normal((6, 1, 9))
    r = rng.standard_normal((2, 6, 30))
    np.testing.assert_allclose(oracle.tidas_conv2d(h, r), oracle.tidas_conv(h[:, 0], r),
                               rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("kz,taps", [(5, 7), (4, 3), (16, 31)])
def test_tidas_conv2d_matches_scattered_convolutions(kz, taps):
    # scatter form, written independently of the oracle's gather loop: every
    # input row j, convolved laterally with slice u of its own kernel, lands on
    # output row j + u - kz//2
    import oracle
    rng = np.random.default_rng(8)
    nz, nx = 11, 37
    h = rng.standard_normal((nz, kz, taps))
    r = rng.standard_normal((nz, nx))
    want = np.zeros((nz, nx))
    cz, cx = kz // 2, taps // 2
    for j in range(nz):
        for u in range(kz):
            i = j + u - cz
            if 0 <= i < nz:
                want[i] += np.convolve(r[j], h[j, u])[cx:cx + nx]
    np.testing.assert_allclose(oracle.tidas_conv2d(h, r), want, rtol=1e-12, atol=1e-12)
    # a unit reflector reproduces its row's kernel, centred on it
    e = np.zeros((nz, nx))
    e[5, 18] = 1.0
    y = oracle.tidas_conv2d(h, e)
    for u in range(kz):
        i = 5 + u - cz
        if 0 <= i < nz:
            np.testing.assert_array_equal(y[i, 18 - cx:18 - cx + taps], h[5, u])
    # adjoint identity
    v = rng.standard_normal((nz, nx))
    lhs = np.vdot(oracle.tidas_conv2d(h, r), v)
    rhs = np.vdot(r, oracle.tidas_conv2d_adjoint(h, v))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_psf_patch_reproduces_exact_image():
    # the 2D kernel of row j convolved with the fitting scatterer returns the
    # exact DAS image of that scatterer over the whole patch; its centre row
    # is the 1D kernel of the same row
    import oracle
    g = presets.geometry("pw64_single")
    o = O(g)
    kz, taps = 9, 31
    rows = [40, 150]
    pat = o.psf_patches(kz, taps, rows=rows)
    psf = o.psf_rows(taps, rows=rows)
    ic = o.center_column()
    for n, j in enumerate(rows):
        rf = o.synthesize([[o.pix_x(ic), o.pix_z(j)]], [[1.0, 0.0]])
        img = o.das(rf)
        k = np.zeros((o.nz, kz, taps))
        k[j] = pat[n]
        r = np.zeros((o.nz, o.nx))
        r[j, ic] = 1.0
        y = oracle.tidas_conv2d(k, r)
        rs = slice(j - kz // 2, j - kz // 2 + kz)
        cs = slice(ic - taps // 2, ic - taps // 2 + taps)
        # the patch grid rounds its own pixel coordinates (x0 + (i + 1/2) dx with
        # a shifted x0), so delays differ in the last bits: ~1e-12 of the peak
        peak = np.abs(img).max()
        np.testing.assert_allclose(y[rs, cs], img[rs, cs], rtol=0, atol=1e-10 * peak)
        np.testing.assert_allclose(pat[n][kz // 2], psf[n], rtol=1e-13, atol=1e-13)


# ------------------------------------------ spatially varying (per-pixel) kernels
def test_tidas_conv_varying_with_equal_kernels_is_the_shift_invariant_form():
    # the same kernel at every pixel of a row: term for term the row-wise and
    # the band convolutions (same loop order, so bit for bit)
    import oracle
    rng = np.random.default_rng(20)
    nz, nx = 7, 33
    h1 = rng.standard_normal((nz, 9))
    h2 = rng.standard_normal((nz, 5, 9))
    r = rng.standard_normal((2, nz, nx))
    k1 = np.ascontiguousarray(np.broadcast_to(h1[:, None, :], (nz, nx, 9)))
    k2 = np.ascontiguousarray(np.broadcast_to(h2[:, None], (nz, nx, 5, 9)))
    np.testing.assert_array_equal(oracle.tidas_conv_varying(k1, r), oracle.tidas_conv(h1, r))
    np.testing.assert_array_equal(oracle.tidas_conv_varying(k2, r), oracle.tidas_conv2d(h2, r))


@pytest.mark.parametrize("kz,taps", [(1, 7), (1, 8), (5, 7), (4, 6)])
def test_tidas_conv_varying_superposes_each_pixels_own_kernel(kz, taps):
    # Born superposition written independently of the oracle's loop: every
    # input pixel (j, s) adds r[j][s] times ITS OWN kernel, placed with its
    # centre on the pixel.  A unit reflector returns exactly its kernel, so the
    # kernel of the output pixel (the other possible reading) would fail.
    import oracle
    rng = np.random.default_rng(21)
    nz, nx = 9, 23
    k = rng.standard_normal((nz, nx, kz, taps))
    r = rng.standard_normal((nz, nx))
    cz, cx = kz // 2, taps // 2
    want = np.zeros((nz + 2 * kz, nx + 2 * taps))  # padded canvas
    for j in range(nz):
        for s in range(nx):
            i0, x0 = j - cz + kz, s - cx + taps
            want[i0:i0 + kz, x0:x0 + taps] += r[j, s] * k[j, s]
    want = want[kz:kz + nz, taps:taps + nx]
    got = oracle.tidas_conv_varying(k if kz > 1 else k[:, :, 0], r)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    e = np.zeros((nz, nx))
    e[4, 11] = 1.0
    y = oracle.tidas_conv_varying(k, e)
    for u in range(kz):
        np.testing.assert_array_equal(y[4 + u - cz, 11 - cx:11 - cx + taps], k[4, 11, u])
    mask = np.ones((nz, nx), bool)
    mask[4 - cz:4 - cz + kz, 11 - cx:11 - cx + taps] = False
    assert not y[mask].any()
    # adjoint identity
    v = rng.standard_normal((nz, nx))
    lhs = np.vdot(oracle.tidas_conv_varying(k, r), v)
    rhs = np.vdot(r, oracle.tidas_conv_varying_adjoint(k, v))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_exact_per_pixel_psfs_reproduce_das():
    # Eq. (2.1) and Eq. (2.2) are linear, so with every pixel's exact
    # single-scatterer image as its kernel (support covering the whole grid),
    # the varying convolution of a reflectivity map IS the DAS image of its
    # synthesised channel data.  A steered wave and a finite F# make the
    # images differ from pixel to pixel.
    import oracle
    g = presets.toy(n_elem=10, nx=6, nz=5, n_samples=160, angles_deg=(7.0,), fnum=1.2)
    o = O(g)
    kz, taps = 2 * g["nz"] - 1, 2 * g["nx"] - 1
    cz, cx = kz // 2, taps // 2
    k = np.zeros((g["nz"], g["nx"], kz, taps))
    for j in range(g["nz"]):
        for s in range(g["nx"]):
            img = o.das(o.synthesize([[o.pix_x(s), o.pix_z(j)]], [[1.0, 0.0]]))
            k[j, s, cz - j:cz - j + g["nz"], cx - s:cx - s + g["nx"]] = img
    # the images do vary across the grid
    assert np.abs(k[0, 0] - k[4, 5]).max() > 0.1 * np.abs(k).max()
    r = np.random.default_rng(22).standard_normal((g["nz"], g["nx"]))
    das = o.das(o.synth_grid(r))
    y = oracle.tidas_conv_varying(k, r)
    np.testing.assert_allclose(y, das, rtol=0, atol=1e-12 * np.abs(das).max())


def test_fwhm_of_gaussian():
    import oracle
    x = np.arange(-50, 51, dtype=np.float64)
    sig = 7.3
    g = np.exp(-0.5 * (x / sig) ** 2)
    assert oracle.fwhm(g) == pytest.approx(2 * math.sqrt(2 * math.log(2)) * sig, rel=2e-3)
