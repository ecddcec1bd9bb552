"""CPU-only checks of the C ABI boundary: the library builds, loads without a
GPU and exports every function include/tidas.h declares; host-side argument
validation rejects bad plans before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2507_15464_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("das_plan_create", "das_forward", "das_adjoint", "tidas_fit_kernels",
                 "tidas_forward", "tidas_adjoint", "tidas_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = capi.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(capi.EXPORTED) <= set(declared_functions())


def test_params_struct_layout_matches_header():
    # the ctypes mirror must follow the header's field order
    text = open(os.path.join(ROOT, "include", "tidas.h")).read()
    body = text[text.index("typedef struct {") + len("typedef struct {"):text.index("} das_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    flat = re.findall(r"(\w+)\s*[,;]", body)
    assert flat == [f[0] for f in capi.das_params._fields_]
    start = text.index("} das_params;")
    body = text[text.index("typedef struct {", start) + len("typedef struct {"):
                text.index("} tidas_line_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    assert re.findall(r"(\w+)\s*[,;]", body) == [f[0] for f in capi.line_params._fields_]


def _line(**kw):
    vals = dict(n_elem=64, pitch=3e-4, f0=5e6, fs=4e7, c=1540.0, frac_bw=0.6, n_samples=1024,
                n_depths=41, z_first=5e-3, z_last=25e-3, z_focus=15e-3, kossoff=0.6,
                fnum_rx=1.0, interp=1)
    vals.update(kw)
    return capi.line_params(**vals)


@pytest.mark.parametrize("bad", [dict(n_elem=0), dict(n_depths=1), dict(z_first=0.0),
                                 dict(z_last=4e-3), dict(kossoff=0.0), dict(interp=2),
                                 dict(n_elem=2000)])
def test_line_calls_reject_bad_parameters(bad):
    # refused on the host by the parameter check itself (null outputs would be
    # refused after it, so the message tells which check fired)
    with pytest.raises(capi.TidasError) as e:
        capi.tidas_line_synthesize(_line(**bad), 0, 1, None)
    assert "null" not in str(e.value)
    with pytest.raises(capi.TidasError) as e:
        capi.tidas_line_das(_line(**bad), None, 1, None)
    assert "null" not in str(e.value)



def _params(**kw):
    p = capi.das_params()
    ang = (ctypes.c_double * 1)(0.0)
    vals = dict(n_elem=8, pitch=3e-4, f0=5e6, fs=4e7, c=1540.0, frac_bw=0.6, n_angles=1,
                n_samples=256, t0=0.0, nx=8, nz=8, x0=-1e-3, dx=2.5e-4, z0=5e-3, dz=2.5e-4,
                interp=1, fnum=1.5, rf_dtype=0)
    vals.update(kw)
    for k, v in vals.items():
        setattr(p, k, v)
    p.angles_rad = ctypes.cast(ang, ctypes.POINTER(ctypes.c_double))
    return p, ang


@pytest.mark.parametrize("bad", [dict(n_elem=0), dict(n_angles=17), dict(nx=0), dict(c=-1.0),
                                 dict(interp=3), dict(rf_dtype=7), dict(z0=-1.0),
                                 dict(frac_bw=0.0), dict(n_samples=2)])
def test_plan_rejects_bad_parameters(bad):
    p, keep = _params(**bad)
    with pytest.raises(capi.TidasError) as e:
        capi.das_plan_create(p)
    assert e.value.code == capi.TIDAS_ERR_ARG
    assert capi.tidas_last_error()


def test_null_arguments_are_rejected_before_any_launch():
    with pytest.raises(capi.TidasError) as e:
        capi.das_forward(None, 1, 1, 1)
    assert e.value.code == capi.TIDAS_ERR_ARG
    with pytest.raises(capi.TidasError) as e:
        capi.tidas_forward(None, 31, 8, 8, 1, 1, 1, 0)
    assert e.value.code == capi.TIDAS_ERR_ARG
    with pytest.raises(capi.TidasError) as e:  # unknown variant
        capi.tidas_forward(16, 31, 8, 8, 16, 16, 1, 9)
    assert e.value.code == capi.TIDAS_ERR_ARG
    with pytest.raises(capi.TidasError) as e:  # GEMM needs taps <= 63
        capi.tidas_forward(16, 65, 8, 8, 16, 16, 1, capi.VARIANT_GEMM_BF16)
    assert e.value.code == capi.TIDAS_ERR_ARG
    with pytest.raises(capi.TidasError) as e:  # GEMM needs 16-byte alignment
        capi.tidas_forward(16, 63, 8, 8, 18, 16, 1, capi.VARIANT_GEMM_BF16)
    assert e.value.code == capi.TIDAS_ERR_ARG


def test_zero_counts_are_argument_errors():
    # empty batches and grids are rejected before anything is enqueued (the
    # pointers below are never dereferenced: validation fails first)
    for args in ((16, 31, 8, 8, 16, 16, 0, capi.VARIANT_DIRECT),   # no frames
                 (16, 31, 0, 8, 16, 16, 1, capi.VARIANT_DIRECT),   # no rows
                 (16, 0, 8, 8, 16, 16, 1, capi.VARIANT_DIRECT)):   # no taps
        with pytest.raises(capi.TidasError) as e:
            capi.tidas_forward(*args)
        assert e.value.code == capi.TIDAS_ERR_ARG


def test_band_workspace_size():
    # (rows x frame tiles x (2 per column tile + 2) chunks) x 16 KB for the
    # GEMM variant of the 2D band calls; none for the direct variant
    assert capi.tidas_band_workspace_bytes(1024, 512, 256, capi.VARIANT_GEMM_BF16) == \
        1024 * 2 * 10 * 16384
    assert capi.tidas_band_workspace_bytes(3, 24, 1, capi.VARIANT_GEMM_BF16) == 3 * 1 * 4 * 16384
    assert capi.tidas_band_workspace_bytes(1024, 512, 256, capi.VARIANT_DIRECT) == 0
    assert capi.tidas_band_workspace_bytes(0, 512, 256, capi.VARIANT_GEMM_BF16) == 0


def test_line_window_is_half_the_envelope_fwhm():
    # host-side closed form, checked against the oracle's (itself pinned to a
    # numerical FWHM of the envelope)
    from oracle.line import LineOracle, paper_line
    for f0 in (5e6, 7e6):
        p = paper_line(f0=f0)
        eps = capi.tidas_line_window(capi.line_params(**p))
        assert eps == pytest.approx(LineOracle(p).eps(), rel=1e-15)


def test_tensor_api_refuses_host_tensors():
    # no CPU fallback: the torch-level wrappers hand device pointers to the C ABI
    # and raise on host tensors instead of computing anything on the CPU
    import torch
    from paper_2507_15464_gb300 import deconv, ops
    k = torch.zeros((8, 31), dtype=torch.float32)
    x = torch.zeros((1, 8, 16), dtype=torch.float32)
    with pytest.raises(ValueError, match="GPU"):
        ops.tidas_forward(k, x, out=torch.empty_like(x))
    k2 = torch.zeros((8, 3, 31), dtype=torch.float32)
    with pytest.raises(ValueError, match="GPU"):
        ops.tidas_forward_2d(k2, x, out=torch.empty_like(x))
    with pytest.raises(ValueError, match="GPU"):
        deconv.dot(x, x)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # without libtidas.so the bindings raise; nothing substitutes for the kernels
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi._build, "LIB", str(tmp_path / "libtidas.so"))
    with pytest.raises(OSError, match="not been built"):
        capi.load(build_if_missing=False)


def test_debug_options_are_validated_on_the_host():
    # the failure-path test hooks reject unknown options and values outside
    # their ranges before touching any device
    for opt, val in ((capi.DEBUG_WAIT_LIMIT_NS, 10), (capi.DEBUG_WAIT_LIMIT_NS, 10 ** 11),
                     (capi.DEBUG_SKIP_COPIES, 2), (99, 0)):
        with pytest.raises(capi.TidasError) as e:
            capi.tidas_set_debug_option(opt, val)
        assert e.value.code == capi.TIDAS_ERR_ARG


@pytest.mark.parametrize("entry", ["fp32_kernels", "bf16_kernels"])
def test_varying_calls_validate_arguments(entry):
    # the spatially varying band calls check their arguments on the host before
    # anything is enqueued; the integer "pointers" below are never dereferenced
    def call(kern=256, ld=64, kz=8, taps=63, nz=8, nx=64, refl=512, img=1024, nf=1,
             variant=capi.VARIANT_GEMM_BF16):
        if entry == "bf16_kernels":
            return capi.tidas_forward_varying_2d_bf16k(kern, ld, kz, taps, nz, nx, refl, img, nf)
        return capi.tidas_forward_varying_2d(kern, ld, kz, taps, nz, nx, refl, img, nf, variant)

    arg_errors = [dict(kern=None), dict(refl=None), dict(img=None),  # null pointers
                  dict(taps=0), dict(ld=62),                         # taps, leading dimension
                  dict(kz=0), dict(nz=0), dict(nx=0), dict(nf=0),    # empty shapes
                  dict(refl=520)]                                    # not 16-byte aligned
    for bad in arg_errors:
        with pytest.raises(capi.TidasError) as e:
            call(**bad)
        assert e.value.code == capi.TIDAS_ERR_ARG, bad
    with pytest.raises(capi.TidasError) as e:  # the GEMM needs nx % 8 == 0
        call(nx=60)
    assert e.value.code == capi.TIDAS_ERR_UNSUPPORTED
    if entry == "fp32_kernels":
        with pytest.raises(capi.TidasError) as e:  # no such variant
            call(variant=9)
        assert e.value.code == capi.TIDAS_ERR_UNSUPPORTED
