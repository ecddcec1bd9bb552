"""GPU parity of spatially varying tiDAS (Eq. (2.13) with a kernel per pixel,
each pixel adding its own single-scatterer image) and of its transpose
against the FP64 oracle, through the C ABI.

FP32 CUDA-core path: relative L2 <= 1e-5 against the oracle on identical
inputs (FP32 FMA chains of at most kz x taps terms); a unit reflector
returns its own kernel bit for bit (one product by 1.0, the other terms
exact zeros).  tcgen05 GEMM path: <= 5e-3 against the oracle on the same
BF16 input values (the kernels are rounded to BF16, unit roundoff 2^-8;
FP32 sums).
"""
import numpy as np
import pytest

from tidas_workloads import generators

from .gpu_helpers import dot_test, host, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def ops():
    from paper_2507_15464_gb300 import ops as o
    return o


def _case(nf, nz, nx, kz, taps, seed):
    shape = (nz, nx, taps) if kz == 1 else (nz, nx, kz, taps)
    k = generators.standard_normal(shape, (seed, 1), np.float32)
    dens = 0.02 if nz * nx >= 65536 else 0.3
    r = generators.bernoulli_normal((nf, nz, nx), dens, (seed, 2)).astype(np.float32)
    return k, r


# (frames, rows, columns, kz, taps): ragged column tiles (nx not a multiple
# of 128, wider than 512), frame counts across the 8-frame register groups
# and the 64-frame block chunks, taps 1 / odd / even / 64, band kernels
CASES = [(3, 6, 700, 1, 63), (70, 3, 37, 1, 64), (2, 5, 129, 1, 1), (9, 4, 300, 1, 31),
         (2, 11, 150, 5, 7), (3, 9, 64, 4, 6), (1, 20, 200, 16, 63), (65, 7, 90, 3, 64)]


@pytest.mark.parametrize("nf,nz,nx,kz,taps", CASES)
def test_varying_forward_and_adjoint_match_oracle(nf, nz, nx, kz, taps):
    import oracle
    o = ops()
    k, r = _case(nf, nz, nx, kz, taps, 70 + nx + kz)
    kd = to_dev(k)
    y = host(o.tidas_forward_varying(kd, to_dev(r)))
    assert rel_l2(y, oracle.tidas_conv_varying(k, r)) <= 1e-5
    v = generators.standard_normal((nf, nz, nx), (71, nx), np.float32)
    a = host(o.tidas_adjoint_varying(kd, to_dev(v)))
    assert rel_l2(a, oracle.tidas_conv_varying_adjoint(k, v)) <= 1e-5
    dot_test(y, v, r, a)


def test_varying_unit_reflectors_return_their_own_kernels():
    o = ops()
    nz, nx, kz, taps = 12, 300, 5, 63
    k, _ = _case(1, nz, nx, kz, taps, 72)
    cz, cx = kz // 2, taps // 2
    pts = [(0, 0), (6, 150), (11, 299), (3, 40)]
    r = np.zeros((len(pts), nz, nx), np.float32)
    for f, (j, s) in enumerate(pts):
        r[f, j, s] = 1.0
    y = host(o.tidas_forward_varying(to_dev(k), to_dev(r)))
    for f, (j, s) in enumerate(pts):
        for u in range(kz):
            i = j + u - cz
            if not 0 <= i < nz:
                continue
            t0, t1 = max(0, cx - s), min(taps, nx - s + cx)
            np.testing.assert_array_equal(y[f, i, s - cx + t0:s - cx + t1], k[j, s, u, t0:t1])


def test_varying_full_rows_sampled():
    # the workload's 1024 x 512 grid with 63-tap row kernels (16 frames);
    # rows are independent at kz = 1, so the oracle runs on sampled rows only
    import oracle
    o = ops()
    nf, nz, nx, taps = 16, 1024, 512, 63
    k, r = _case(nf, nz, nx, 1, taps, 73)
    y = host(o.tidas_forward_varying(to_dev(k), to_dev(r)))
    rows = [0, 1, 255, 511, 1022, 1023]
    ref = oracle.tidas_conv_varying(k[rows], r[:, rows])
    assert rel_l2(y[:, rows], ref) <= 1e-5


def test_varying_band_full_width_slab():
    # 16 x 63 band kernels on full 512-column rows; the oracle runs on a slab
    # of rows and only the rows whose whole band lies in the slab are compared
    import oracle
    o = ops()
    nf, nz, nx, kz, taps = 4, 96, 512, 16, 63
    k, r = _case(nf, nz, nx, kz, taps, 74)
    y = host(o.tidas_forward_varying(to_dev(k), to_dev(r)))
    lo, hi = 30, 70
    ref = oracle.tidas_conv_varying(k[lo:hi], r[:, lo:hi])
    inner = slice(kz, hi - lo - kz)
    assert rel_l2(y[:, lo:hi][:, inner], ref[:, inner]) <= 1e-5


def test_varying_rejects_unsupported_requests():
    from paper_2507_15464_gb300 import capi
    o = ops()
    k, r = _case(1, 4, 32, 1, 9, 75)
    with pytest.raises(capi.TidasError) as e:
        o.tidas_forward_varying(to_dev(k), to_dev(r), variant=capi.VARIANT_GEMM_RESID)
    assert e.value.code == capi.TIDAS_ERR_UNSUPPORTED
    big = np.zeros((4, 32, 65), np.float32)
    with pytest.raises(capi.TidasError) as e:
        o.tidas_forward_varying(to_dev(big), to_dev(r))
    assert e.value.code == capi.TIDAS_ERR_ARG


# (frames, rows, columns, kz, taps) of the GEMM path: one and three frame
# tiles (two per item, then a ragged one), partial column tiles, taps 1 / odd
# / 64, kz 1 .. 16
GEMM_CASES = [(3, 6, 256, 1, 63), (130, 5, 200, 4, 31), (257, 4, 64, 3, 64), (2, 20, 512, 8, 63),
              (1, 9, 136, 16, 7), (5, 3, 8, 2, 1)]


@pytest.mark.parametrize("nf,nz,nx,kz,taps", GEMM_CASES)
def test_varying_gemm_matches_oracle(nf, nz, nx, kz, taps):
    import oracle
    from paper_2507_15464_gb300 import capi
    o = ops()
    k, r = _case(nf, nz, nx, kz, taps, 76 + nx + kz)
    x16 = to_dev(r).to(torch.bfloat16)
    y = host(o.tidas_forward_varying(to_dev(k), x16, variant=capi.VARIANT_GEMM_BF16))
    frames = sorted({0, nf // 2, nf - 1})
    ref = oracle.tidas_conv_varying(k, host(x16)[frames])
    assert rel_l2(y[frames], ref) <= 5e-3
    # and close to the FP32 direct path on every frame
    yd = host(o.tidas_forward_varying(to_dev(k), x16.float()))
    assert rel_l2(y, yd) <= 5e-3
    # kernels at a 64-column pitch (read in place by the tensor copies) with
    # garbage in the columns past the taps: the same image
    kp = np.full(k.shape[:-1] + (64,), 1e3, np.float32)
    kp[..., :taps] = k
    yp = host(o.tidas_forward_varying(to_dev(kp), x16, variant=capi.VARIANT_GEMM_BF16, taps=taps))
    np.testing.assert_array_equal(yp, y)


def test_varying_gemm_full_width_band_slab():
    # the workload's 512-column rows with 8 x 63 band kernels and 256 frames
    # (two frame tiles per item); the oracle runs on a slab of rows for the
    # first and last frames, and the rows whose band lies in the slab compare
    import oracle
    from paper_2507_15464_gb300 import capi
    o = ops()
    nf, nz, nx, kz, taps = 256, 64, 512, 8, 63
    k, r = _case(nf, nz, nx, kz, taps, 77)
    x16 = to_dev(r).to(torch.bfloat16)
    y = host(o.tidas_forward_varying(to_dev(k), x16, variant=capi.VARIANT_GEMM_BF16))
    lo, hi = 20, 50
    xs = host(x16)[[0, nf - 1]][:, lo:hi]
    ref = oracle.tidas_conv_varying(k[lo:hi], xs)
    inner = slice(kz, hi - lo - kz)
    assert rel_l2(y[[0, nf - 1]][:, lo:hi][:, inner], ref[:, inner]) <= 5e-3


@pytest.mark.parametrize("nf,nz,nx,kz,taps", GEMM_CASES)
def test_varying_gemm_bf16_kernels_bit_identical(nf, nz, nx, kz, taps):
    # BF16 per-pixel kernels (tidas_forward_varying_2d_bf16k): the builders
    # otherwise round the FP32 kernels to BF16 (nearest even), so kernels
    # rounded the same way give the same image bit for bit, at the taps' own
    # pitch (padded copy when not a multiple of 8) and at a 64-column pitch
    # with garbage past the taps
    from paper_2507_15464_gb300 import capi
    o = ops()
    k, r = _case(nf, nz, nx, kz, taps, 78 + nx + kz)
    x16 = to_dev(r).to(torch.bfloat16)
    kd = to_dev(k)
    y = host(o.tidas_forward_varying(kd, x16, variant=capi.VARIANT_GEMM_BF16))
    y16 = host(o.tidas_forward_varying(kd.to(torch.bfloat16), x16, variant=capi.VARIANT_GEMM_BF16))
    np.testing.assert_array_equal(y16, y)
    kp = torch.full(tuple(k.shape[:-1]) + (64,), 3e4, dtype=torch.bfloat16, device="cuda")
    kp[..., :taps] = kd.to(torch.bfloat16)
    yp = host(o.tidas_forward_varying(kp, x16, variant=capi.VARIANT_GEMM_BF16, taps=taps))
    np.testing.assert_array_equal(yp, y)
    with pytest.raises(ValueError):
        o.tidas_forward_varying(kd.to(torch.bfloat16), x16.float())
