"""Seeded random inputs (numpy PCG64 via SeedSequence; portable across hosts).

Every function returns plain arrays in the dtype the consumer uploads, so the
oracle and the GPU path read identical values.  Random numbers that an
algorithm itself draws (power-iteration start, network initialisation,
training-set sampling, measurement noise) are produced here as well and
passed in as inputs.
"""
import numpy as np


def _rng(*seed):
    return np.random.default_rng(list(seed))


def point_scatterers(n, x_range, z_range, seed, real=True):
    """n scatterers uniform in a box; amplitudes N(0,1) (real) or CN(0,1).

    Returns pos [n, 2] float64 (x, z) and amp [n, 2] float32 (Re, Im)."""
    rng = _rng(*seed)
    x = rng.uniform(x_range[0], x_range[1], n)
    z = rng.uniform(z_range[0], z_range[1], n)
    pos = np.stack([x, z], axis=1).astype(np.float64)
    amp = np.zeros((n, 2), np.float32)
    if real:
        amp[:, 0] = rng.standard_normal(n)
    else:
        amp[:, 0] = rng.standard_normal(n) * np.sqrt(0.5)
        amp[:, 1] = rng.standard_normal(n) * np.sqrt(0.5)
    return pos, amp


def single_frame_speckle(seed=0, n=200):
    """64-element workload: 200 real N(0,1) scatterers in a 19 mm x 30 mm box."""
    return point_scatterers(n, (-9.5e-3, 9.5e-3), (5.0e-3, 35.0e-3), (seed,), real=True)


def compound_speckle_frame(frame, n_speckle=100_000, seed=1):
    """128-element workload, one frame: complex-Gaussian speckle plus ten bright
    point targets 20 dB above the speckle RMS on the axis at z = 10..55 mm."""
    pos, amp = point_scatterers(n_speckle, (-19.2e-3, 19.2e-3), (5.0e-3, 60.0e-3),
                                (seed, frame), real=False)
    rng = _rng(seed, frame, 7)
    tz = np.arange(10, 60, 5, dtype=np.float64) * 1e-3
    tpos = np.stack([np.zeros_like(tz), tz], axis=1)
    phase = rng.uniform(0.0, 2.0 * np.pi, tz.size)
    tamp = np.stack([10.0 * np.cos(phase), 10.0 * np.sin(phase)], axis=1).astype(np.float32)
    return np.concatenate([pos, tpos]), np.concatenate([amp, tamp])


def compound_speckle_batch(n_frames, n_speckle=100_000, seed=1):
    """[B, n, 2] positions and amplitudes, frame f drawn from seed (seed, f)."""
    ps, am = zip(*[compound_speckle_frame(f, n_speckle, seed) for f in range(n_frames)])
    return np.stack(ps), np.stack(am)


def sparse_reflectivity(n_frames, nz, nx, p=0.02, seed=2, dtype=np.float32):
    """Bernoulli(p) support times N(0,1) amplitudes, [B, nz, nx]."""
    rng = _rng(seed)
    out = np.empty((n_frames, nz, nx), dtype)
    for f in range(n_frames):
        mask = rng.random((nz, nx)) < p
        out[f] = (mask * rng.standard_normal((nz, nx))).astype(dtype)
    return out


def standard_normal(shape, seed, dtype=np.float32):
    return _rng(*seed).standard_normal(shape).astype(dtype)


def uniform(shape, lo, hi, seed, dtype=np.float64):
    return _rng(*seed).uniform(lo, hi, shape).astype(dtype)


def bernoulli_normal(shape, p, seed, dtype=np.float32):
    rng = _rng(*seed)
    mask = rng.random(shape) < p
    return (mask * rng.standard_normal(shape)).astype(dtype)
