"""Pins of the single-line oracle (Section 3, Eq. (2.8), (2.12), (2.13)):
each check ties it to something other than itself -- the plane-wave oracle
(pinned separately), Eq. (2.3), closed forms of the transmit focus and of the
pulse envelope, and identities between the DAS and fixed-curve lines."""
import numpy as np
import pytest

import oracle
from oracle.line import LineOracle, paper_line


def small_line(**kw):
    # 64 elements, 41 points from 5 to 25 mm (0.5 mm apart: the 15 mm focus is point 20)
    p = dict(n_elem=64, pitch=0.3e-3, f0=5e6, fs=40e6, c=1540.0, frac_bw=0.6, n_samples=1536,
             n_depths=41, z_first=5e-3, z_last=25e-3, z_focus=15e-3, kossoff=0.6, fnum_rx=1.0,
             interp=1)
    p.update(kw)
    return LineOracle(p)


def test_kossoff_aperture_and_focus_timing():
    O = LineOracle(paper_line(z_focus=25e-3))
    # a_tx = sqrt(z_f lambda / 0.6) = 3.582 mm: elements at +-(0.15 + 0.3 j) mm, j <= 11
    a = np.sqrt(25e-3 * (1540.0 / 5e6) / 0.6)
    assert O.tx_radius() == pytest.approx(a, rel=1e-15)
    act = O.tx_active()
    assert act.sum() == 24 == 2 * int(np.floor(a / 0.3e-3 + 0.5))
    # every active element's wavelet reaches the focus at z_f / c
    for m in np.nonzero(act)[0]:
        xm = O.elem_x(m)
        assert O.fire(m) + np.hypot(xm, 25e-3) / 1540.0 == pytest.approx(25e-3 / 1540.0,
                                                                          abs=1e-18)


def test_receive_delay_is_eq23_of_the_plane_wave_oracle():
    O = small_line()
    g = dict(n_elem=64, pitch=0.3e-3, f0=5e6, fs=40e6, c=1540.0, frac_bw=0.6, t0=0.0, fnum=1.0,
             angles_deg=[0.0], n_samples=1536, nx=4, nz=4, x0=-0.3e-3, dx=0.15e-3, z0=5e-3,
             dz=1e-3, interp=1)
    P = oracle.Oracle(g)
    for n in (0, 13, 31, 32, 63):
        for z in (5e-3, 11.3e-3, 25e-3):
            assert O.delay(n, z) == P.receive_delay_eq23(n, z)


def test_channel_data_at_the_focus_is_the_aligned_pulse_sum():
    # at the focus all transmit wavelets coincide: the data equal |Tx| times
    # the single-wave data of the plane-wave oracle (0 degrees, same scatterer)
    O = small_line()
    r = 20
    assert O.depth(r) == pytest.approx(15e-3, abs=1e-15)
    S = O.synth(r)
    g = dict(n_elem=64, pitch=0.3e-3, f0=5e6, fs=40e6, c=1540.0, frac_bw=0.6, t0=0.0, fnum=1.0,
             angles_deg=[0.0], n_samples=1536, nx=4, nz=4, x0=-0.3e-3, dx=0.15e-3, z0=5e-3,
             dz=1e-3, interp=1)
    ref = oracle.Oracle(g).synthesize(np.array([[0.0, O.depth(r)]]), np.array([[1.0, 0.0]]))[0]
    ntx = O.tx_active().sum()
    np.testing.assert_allclose(S, ntx * ref, rtol=0, atol=1e-11 * ntx)


def test_das_line_peaks_on_the_scatterer():
    O = small_line()
    for r in (3, 20, 37):
        g = O.das_line(O.synth(r))
        assert int(np.argmax(np.abs(g))) == r


def test_fixed_curve_of_the_scatterer_equals_das_on_its_point():
    # Eq. (2.8) with D_n = D_n^r and no window is Eq. (2.7) at z_r
    O = small_line()
    for r in (4, 20, 33):
        S = O.synth(r)
        g = O.das_line(S)
        a = O.fixed_line(S, r, r, -1.0)
        assert a[r] == g[r]


def test_window_limits_and_the_envelope_fwhm():
    O = small_line()
    # eps is half the FWHM of the pulse envelope exp(-alpha t^2)
    t = np.linspace(-1e-6, 1e-6, 2000001)
    env = np.exp(-O.alpha() * t * t)
    above = t[env >= 0.5]
    assert above[-1] - above[0] == pytest.approx(2 * O.eps(), rel=1e-5)
    r = 12
    S = O.synth(r)
    # a window wider than the echo changes nothing
    np.testing.assert_array_equal(O.fixed_line(S, r, 25, 5e-6), O.fixed_line(S, r, 25, -1.0))
    # a window of half a sample keeps one sample per channel
    n = 40
    k_t = O.arrival(n, O.depth(r)) * 40e6
    kept = [k for k in range(1536) if O.in_window(r, 0.49 / 40e6, n, k)]
    assert kept == [int(np.rint(k_t))]


def test_theta_of_the_own_curve_is_one_and_matches_the_frequency_form():
    O = small_line()
    r = 26
    S = O.synth(r)
    g = O.das_line(S)
    eps = O.eps()
    th, el, eg = O.sweep_pair(S, g, r, r, eps)
    assert th == 1.0
    assert 0.0 <= el and 0.0 <= eg
    # Eq. (2.12) in the frequency domain (Plancherel) gives the same weight
    for s in (20, 30):
        a = O.fixed_line(S, r, s, eps)
        b = O.fixed_line(S, r, r, eps)
        th_s = O.sweep_pair(S, g, r, s, eps)[0]
        assert th_s == pytest.approx(oracle.theta_ls_freq(a, b), rel=1e-10)
        # theta minimises ||theta a - b||: the residual is orthogonal to a
        assert abs(np.dot(th_s * a - b, a)) <= 1e-10 * np.dot(b, b)


def test_errors_are_relative_energies_of_the_difference():
    O = small_line()
    r, s = 18, 23
    S = O.synth(r)
    g = O.das_line(S)
    eps = O.eps()
    th, el, eg = O.sweep_pair(S, g, r, s, eps)
    a = O.fixed_line(S, r, s, eps)
    # global error by expansion of ||theta a - g||^2
    expand = (th * th * np.dot(a, a) - 2 * th * np.dot(a, g) + np.dot(g, g)) / np.dot(g, g)
    assert eg == pytest.approx(expand, rel=1e-9)
    # the local points are the scatterer's own neighbourhood in depth
    w = O.local_points(r, eps)
    assert w[r] and w.sum() >= 1 and np.all(np.abs(np.nonzero(w)[0] - r) <= 1)


def test_line_model_at_a_scatterer_is_its_windowed_fixed_curve_line():
    # Eq. (2.13) with theta = 1 on the data of one scatterer r reads, at point
    # r, the windowed fixed-curve line of Eq. (2.8) for that scatterer
    O = small_line()
    eps = O.eps()
    for r, s in ((12, 12), (12, 16), (30, 25)):
        S = O.synth(r)
        m = O.model_line(S, s, np.ones(41), eps)
        assert m[r] == pytest.approx(O.fixed_line(S, r, s, eps)[r], rel=1e-12, abs=1e-15)


def test_line_model_is_linear_and_scaled_by_theta():
    O = small_line()
    eps = O.eps()
    amps = np.zeros(41)
    amps[[8, 22]] = [1.0, -0.5]
    S = O.line_data(amps)
    np.testing.assert_allclose(S, O.synth(8) - 0.5 * O.synth(22), rtol=0, atol=1e-12)
    th = np.linspace(0.5, 2.0, 41)
    m = O.model_line(S, 20, th, eps)
    m1 = O.model_line(O.synth(8), 20, np.ones(41), eps)
    m2 = O.model_line(O.synth(22), 20, np.ones(41), eps)
    np.testing.assert_allclose(m, th * (m1 - 0.5 * m2), rtol=1e-12, atol=1e-14)


def test_envelope_of_pure_and_modulated_tones():
    from oracle.line import envelope
    n = 600
    k = np.arange(n)
    np.testing.assert_allclose(envelope(np.cos(2 * np.pi * 37 * k / n + 0.3)), 1.0, atol=1e-12)
    # a narrow-band Gaussian burst: the envelope is the Gaussian
    g = np.exp(-((k - 300) / 40.0) ** 2)
    np.testing.assert_allclose(envelope(g * np.cos(2 * np.pi * 0.2 * k)), g, atol=1e-6)


def test_sidelobe_level_and_main_lobes():
    from oracle.line import line_scenarios, sidelobe_level_db
    z = np.arange(100) * 1e-4
    env = np.full(100, 0.1)
    env[[20, 60]] = 1.0
    assert sidelobe_level_db(env, z, [20, 60], 2.5e-4) == pytest.approx(-20.0, abs=1e-12)
    sc = line_scenarios()
    assert (sc["5_uniform"] > 0).sum() == 5 and (sc["100_uniform"] > 0).sum() == 100
    np.testing.assert_array_equal(np.nonzero(sc["5_increasing"])[0], np.nonzero(sc["5_uniform"])[0])
    O = LineOracle(paper_line())
    # main lobe: the pulse envelope 20 dB down, two-way depth
    t20 = O.mainlobe_halfwidth() * 2 / 1540.0
    assert np.exp(-O.alpha() * t20 ** 2) == pytest.approx(0.1, rel=1e-12)
