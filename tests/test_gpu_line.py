"""GPU parity of the single-line experiment of Section 3 (focused transmit,
DAS lines, and the Eq. (2.8) / (2.12) sweep over every (delay curve,
scatterer) pair) against the FP64 oracle, through the C ABI.

Tolerances: channel data and DAS lines relative L2 <= 1e-5 (FP32 pulse and
sums; the sample indices and the apertures are taken in FP64 on both
sides).  theta relative <= 1e-4 where the fixed-curve line carries at least
1e-6 of the largest energy over the curves (elsewhere theta is a ratio of
vanishing sums); errors absolute <= 1e-4 (FP32 sums of the lines).
"""
import functools

import numpy as np
import pytest

from .gpu_helpers import host, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def small_params(**kw):
    p = dict(n_elem=64, pitch=0.3e-3, f0=5e6, fs=40e6, c=1540.0, frac_bw=0.6, n_samples=1536,
             n_depths=41, z_first=5e-3, z_last=25e-3, z_focus=15e-3, kossoff=0.6, fnum_rx=1.0,
             interp=1)
    p.update(kw)
    return p


def experiment(p):
    from paper_2507_15464_gb300.ops import LineExperiment
    return LineExperiment(p)


def line_oracle(p):
    from oracle.line import LineOracle
    return LineOracle(p)


@pytest.mark.parametrize("interp", [0, 1])
def test_synthesis_and_das_lines_match_oracle(interp):
    p = small_params(interp=interp)
    E, O = experiment(p), line_oracle(p)
    rf = E.synthesize()
    rf_h = host(rf)
    for r in (0, 7, 20, 40):
        assert rel_l2(rf_h[r], O.synth(r)) <= 1e-5
    g = host(E.das_lines(rf))
    for r in (0, 7, 20, 40):
        assert rel_l2(g[r], O.das_line(rf_h[r].astype(np.float64))) <= 1e-5


def _compare_sweep(O, rf_h, g_h, th, el, eg, rs, ss, eps, r_first=0):
    for r in rs:
        S = rf_h[r - r_first].astype(np.float64)
        g = g_h[r - r_first].astype(np.float64)
        ref = [O.sweep_pair(S, g, r, s, eps) for s in ss]
        aa = np.array([np.dot(a, a) for a in (O.fixed_line(S, r, s, eps) for s in ss)])
        for j, s in enumerate(ss):
            t_ref, el_ref, eg_ref = ref[j]
            got = th[s, r - r_first], el[s, r - r_first], eg[s, r - r_first]
            if aa[j] >= 1e-6 * aa.max():
                assert got[0] == pytest.approx(t_ref, rel=1e-4, abs=1e-6), (r, s)
            assert got[1] == pytest.approx(el_ref, abs=1e-4), (r, s)
            assert got[2] == pytest.approx(eg_ref, abs=1e-4), (r, s)


@pytest.mark.parametrize("interp", [0, 1])
def test_sweep_matches_oracle_on_every_curve(interp):
    p = small_params(interp=interp)
    E, O = experiment(p), line_oracle(p)
    rf = E.synthesize()
    g = E.das_lines(rf)
    eps = O.eps()
    th, el, eg = (host(t) for t in E.sweep(rf, g, eps))
    assert th.shape == (41, 41)
    _compare_sweep(O, host(rf), host(g), th, el, eg, (0, 3, 20, 33, 40), range(41), eps)
    # every scatterer's own curve reproduces b exactly: theta = 1
    np.testing.assert_allclose(np.diag(th), 1.0, rtol=1e-6)


def test_sweep_of_a_scatterer_subset_equals_the_full_sweep():
    p = small_params()
    E, O = experiment(p), line_oracle(p)
    rf = E.synthesize()
    g = E.das_lines(rf)
    eps = O.eps()
    full = [host(t) for t in E.sweep(rf, g, eps)]
    part = [host(t) for t in E.sweep(rf[10:25].contiguous(), g[10:25].contiguous(), eps,
                                      r_first=10)]
    for f, q in zip(full, part):
        np.testing.assert_allclose(q, f[:, 10:25], rtol=1e-6, atol=1e-7)
    # the subset's own channel data (synthesised from point 10 on) are the same
    np.testing.assert_array_equal(host(E.synthesize(10, 15)), host(rf[10:25]))


def test_too_wide_window_is_refused():
    from paper_2507_15464_gb300 import capi
    p = small_params()
    E = experiment(p)
    rf = E.synthesize(0, 2)
    g = E.das_lines(rf)
    with pytest.raises(capi.TidasError):
        E.sweep(rf, g, 14.0 / 40e6)


@functools.lru_cache(maxsize=1)
def _paper_run():
    from oracle.line import paper_line
    p = paper_line(f0=5e6, z_focus=25e-3)
    E, O = experiment(p), line_oracle(p)
    rf = E.synthesize()
    g = E.das_lines(rf)
    eps = O.eps()
    th, el, eg = (host(t) for t in E.sweep(rf, g, eps))
    return p, O, host(rf), host(g), th, el, eg, eps


def test_paper_line_600_by_600_sampled_pairs():
    # 600 line points from 2 to 42 mm, 192 elements, focus 25 mm: every
    # (curve, scatterer) pair is computed, sampled pairs are checked
    p, O, rf_h, g_h, th, el, eg, eps = _paper_run()
    assert th.shape == (600, 600)
    rs = (0, 1, 150, 344, 599)
    for r in rs:
        assert rel_l2(rf_h[r], O.synth(r)) <= 1e-5
        assert rel_l2(g_h[r], O.das_line(rf_h[r].astype(np.float64))) <= 1e-5
    _compare_sweep(O, rf_h, g_h, th, el, eg, rs, (0, 10, 100, 300, 343, 344, 345, 598, 599), eps)
    np.testing.assert_allclose(np.diag(th), 1.0, rtol=1e-6)
    assert np.all(np.isfinite(th)) and np.all(el >= 0) and np.all(eg >= -1e-6)


# ------------------------------------------------------ line reconstruction
def test_line_data_and_model_match_oracle():
    p = small_params()
    E, O = experiment(p), line_oracle(p)
    rf = E.synthesize()
    amps = np.zeros(41, np.float32)
    amps[[6, 19, 31]] = [1.0, -0.7, 2.5]
    S = E.combine(rf, to_dev(amps))
    S_h = host(S)
    assert rel_l2(S_h, O.line_data(amps.astype(np.float64))) <= 1e-5
    eps = O.eps()
    rng = np.random.default_rng(7)
    for s in (5, 20, 35):
        th = rng.uniform(0.5, 2.0, 41).astype(np.float32)
        got = host(E.model(S, s, to_dev(th), eps))
        ref = O.model_line(S_h.astype(np.float64), s, th.astype(np.float64), eps)
        assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("n", [600, 41, 257])
def test_envelope_matches_oracle(n):
    from oracle.line import envelope as env_ref
    from paper_2507_15464_gb300.ops import envelope
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)).astype(np.float32)
    k = np.arange(n)
    x[1] = (np.exp(-((k - n / 2) / (n / 12)) ** 2) * np.cos(2 * np.pi * 0.23 * k)).astype(np.float32)
    got = host(envelope(to_dev(x)))
    for j in range(3):
        assert rel_l2(got[j], env_ref(x[j].astype(np.float64))) <= 1e-5


def test_paper_line_reconstruction_matches_oracle():
    # five unit scatterers, delay curve of the 25 mm point, theta from the sweep
    from oracle.line import line_scenarios
    p, O, rf_h, g_h, th, el, eg, eps = _paper_run()
    E = experiment(p)
    s = int(np.argmin(np.abs(O.depths() - 25e-3)))
    amps = line_scenarios()["5_uniform"].astype(np.float32)
    rf = to_dev(rf_h)
    S = E.combine(rf, to_dev(amps))
    S_h = host(S).astype(np.float64)
    das = host(E.das_lines(S.reshape(1, *S.shape)))[0]
    assert rel_l2(das, O.das_line(S_h)) <= 1e-5
    got = host(E.model(S, s, to_dev(np.ascontiguousarray(th[s])), eps))
    assert rel_l2(got, O.model_line(S_h, s, th[s].astype(np.float64), eps)) <= 1e-5


def test_fixed_lines_match_oracle():
    # the tiDAS reconstruction of each scatterer under one delay curve
    p = small_params()
    E, O = experiment(p), line_oracle(p)
    rf = E.synthesize()
    eps = O.eps()
    rf_h = host(rf)
    for s in (20, 9):
        got = host(E.fixed_lines(rf, s, eps))
        assert got.shape == (41, 41)
        for r in (3, 18, 20, 35):
            S = rf_h[r].astype(np.float64)
            a = O.fixed_line(S, r, s, eps)
            th = O.sweep_pair(S, O.das_line(S), r, s, eps)[0]
            ref = th * a
            if np.linalg.norm(ref) > 0:
                assert rel_l2(got[r], ref) <= 1e-4, (r, s)
