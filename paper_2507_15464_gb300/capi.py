"""ctypes binding of libtidas.so with the C ABI's names (argument marshalling only).

Every function takes raw device pointers (ints) and a stream handle, exactly
as declared in include/tidas.h, and raises TidasError on a non-zero status.
There is no fallback: if the library cannot be loaded the import fails.
"""
import ctypes
import os

from . import build as _build

TIDAS_OK, TIDAS_ERR_ARG, TIDAS_ERR_CUDA, TIDAS_ERR_TIMEOUT, TIDAS_ERR_UNSUPPORTED = 0, -1, -2, -3, -4
RF_F32, RF_F16 = 0, 1
INTERP_LINEAR, INTERP_CUBIC = 0, 1
VARIANT_DIRECT, VARIANT_GEMM_BF16, VARIANT_GEMM_RESID = 0, 1, 2
DEBUG_WAIT_LIMIT_NS, DEBUG_SKIP_COPIES = 1, 2


class TidasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("tidas status %d: %s" % (code, msg))
        self.code = code


class das_params(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int32), ("pitch", ctypes.c_double), ("f0", ctypes.c_double),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("frac_bw", ctypes.c_double),
        ("n_angles", ctypes.c_int32), ("angles_rad", ctypes.POINTER(ctypes.c_double)),
        ("n_samples", ctypes.c_int32), ("t0", ctypes.c_double),
        ("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("x0", ctypes.c_double), ("dx", ctypes.c_double),
        ("z0", ctypes.c_double), ("dz", ctypes.c_double),
        ("interp", ctypes.c_int32), ("fnum", ctypes.c_double), ("rf_dtype", ctypes.c_int32),
    ]


class line_params(ctypes.Structure):
    """Mirror of tidas_line_params (include/tidas.h), field for field."""
    _fields_ = [
        ("n_elem", ctypes.c_int32), ("pitch", ctypes.c_double), ("f0", ctypes.c_double),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("frac_bw", ctypes.c_double),
        ("n_samples", ctypes.c_int32), ("n_depths", ctypes.c_int32),
        ("z_first", ctypes.c_double), ("z_last", ctypes.c_double),
        ("z_focus", ctypes.c_double), ("kossoff", ctypes.c_double),
        ("fnum_rx", ctypes.c_double), ("interp", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int32
_S = ctypes.c_size_t
_SIG = {
    "das_plan_create": [ctypes.POINTER(das_params), ctypes.POINTER(ctypes.c_void_p)],
    "das_plan_destroy": [_P],
    "das_plan_set_option": [_P, _I, _I],
    "das_plan_read_window": [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "das_upload_window": [_P, _P, _P, _I, _P],
    "das_synthesize": [_P, _P, _P, _I, _I, _P, _P],
    "das_synthesize_grid": [_P, _P, _P, _I, _P],
    "das_synthesize_adjoint": [_P, _P, _P, _I, _P],
    "das_forward": [_P, _P, _P, _I, _P],
    "das_adjoint": [_P, _P, _P, _I, _P],
    "das_delay_table": [_P, _I, _P, _P, _P],
    "tidas_fit_kernels": [_P, _I, _I, _P, _P, _P],
    "tidas_forward": [_P, _I, _I, _I, _P, _P, _I, _I, _P],
    "tidas_adjoint": [_P, _I, _I, _I, _P, _P, _I, _I, _P],
    "tidas_device_status": [ctypes.POINTER(ctypes.c_int32)],
    "tidas_set_debug_option": [_I, ctypes.c_int64],
    "tidas_dot": [_P, _P, ctypes.c_int64, _P, _P],
    "tidas_dot_noalloc": [_P, _P, ctypes.c_int64, _P, _P],
    "tidas_asum": [_P, ctypes.c_int64, _P, _P],
    "tidas_fista_update": [_P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, _P],
    "tidas_axpby": [_P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, _P],
    "tidas_psf_batch": [_P, _P, _I, _I, _P, _I, _P, _P],
    "tidas_psf_batch_2d": [_P, _P, _I, _I, _I, _I, _P, _I, _P, _P],
    "tidas_apod_sum": [_P, _P, ctypes.c_int64, _P, _P],
    "tidas_gemm_bf16": [_P, _P, _I, _I, _I, _P, _I, _P, _P, _I, _P],
    "tidas_transpose_bf16": [_P, _I, _I, _P, _P],
    "tidas_relu_backward": [_P, _P, ctypes.c_int64, _P, _P, _P],
    "tidas_gather_rows": [_P, _P, ctypes.c_int64, _I, _P, _P],
    "tidas_colsum": [_P, _I, _I, _I, _P, _P],
    "tidas_adam": [_P, _P, _P, _P, _I, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                   ctypes.c_float, ctypes.c_float, _I, _P, _P, _P],
    "tidas_mse": [_P, _P, _I, _I, _I, _I, _P, _P, _P],
    "tidas_encode": [_P, _I, _P, _P, _P, _P],
    "tidas_mlp_infer": [_P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _I, _I, _P],
    "tidas_fit_kernels_2d": [_P, _I, _I, _P, _P],
    "tidas_forward_2d": [_P, _I, _I, _I, _I, _P, _P, _I, _I, _P, _S, _P],
    "tidas_adjoint_2d": [_P, _I, _I, _I, _I, _P, _P, _I, _I, _P, _S, _P],
    "tidas_forward_varying": [_P, _I, _I, _I, _I, _P, _P, _I, _P],
    "tidas_forward_varying_2d": [_P, _I, _I, _I, _I, _I, _P, _P, _I, _I, _P],
    "tidas_adjoint_varying_2d": [_P, _I, _I, _I, _I, _I, _P, _P, _I, _I, _P],
    "tidas_forward_varying_2d_bf16k": [_P, _I, _I, _I, _I, _I, _P, _P, _I, _P],
    "tidas_kernel_fallback": [_P, _I, _P, _I, ctypes.c_int64, _I, ctypes.c_float, _P, _I, _P, _P],
    "tidas_row_scale": [_P, _I, _P, ctypes.c_int64, _I, _P, _I, _P],
    "tidas_band_workspace_bytes": [_I, _I, _I, _I],
    "tidas_line_synthesize": [ctypes.POINTER(line_params), _I, _I, _P, _P],
    "tidas_line_das": [ctypes.POINTER(line_params), _P, _I, _P, _P],
    "tidas_line_sweep": [ctypes.POINTER(line_params), _P, _P, _I, _I, ctypes.c_double, _P, _P,
                         _P, _P],
    "tidas_line_window": [ctypes.POINTER(line_params), ctypes.POINTER(ctypes.c_double)],
    "tidas_line_combine": [ctypes.POINTER(line_params), _P, _I, _P, _P, _P],
    "tidas_line_model": [ctypes.POINTER(line_params), _P, _I, _P, ctypes.c_double, _P, _P],
    "tidas_line_envelope": [_I, _I, _P, _P, _P],
    "tidas_line_fixed": [ctypes.POINTER(line_params), _P, _I, _I, _I, ctypes.c_double, _P, _P],
}
_RESTYPE = {"tidas_band_workspace_bytes": _S}
EXPORTED = list(_SIG) + ["tidas_last_error"]

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libtidas.so (building it first if absent).  Raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        _build.build()  # no-op when the library is newer than its sources
    elif not os.path.exists(path):
        raise OSError("libtidas.so has not been built: run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, args in _SIG.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _RESTYPE.get(name, ctypes.c_int)
    L.tidas_last_error.argtypes = []
    L.tidas_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc):
    if rc != TIDAS_OK:
        msg = load().tidas_last_error().decode(errors="replace")
        raise TidasError(rc, msg)
    return rc


def das_plan_create(params: das_params):
    h = ctypes.c_void_p()
    _check(load().das_plan_create(ctypes.byref(params), ctypes.byref(h)))
    return h.value


def das_plan_destroy(plan):
    return _check(load().das_plan_destroy(plan))


def das_synthesize(plan, pos_xz, amp, n_scat, n_frames, rf, stream=0):
    return _check(load().das_synthesize(plan, pos_xz, amp, n_scat, n_frames, rf, stream))


def das_synthesize_grid(plan, refl, rf, n_frames, stream=0):
    return _check(load().das_synthesize_grid(plan, refl, rf, n_frames, stream))


def das_synthesize_adjoint(plan, rf, refl, n_frames, stream=0):
    return _check(load().das_synthesize_adjoint(plan, rf, refl, n_frames, stream))


def das_forward(plan, rf, img, n_frames, stream=0):
    return _check(load().das_forward(plan, rf, img, n_frames, stream))


def das_adjoint(plan, img, rf, n_frames, stream=0):
    return _check(load().das_adjoint(plan, img, rf, n_frames, stream))


def das_delay_table(plan, angle, idx, frac, stream=0):
    return _check(load().das_delay_table(plan, angle, idx, frac, stream))


def tidas_fit_kernels(plan, taps, ref_stride, kernels, theta, stream=0):
    return _check(load().tidas_fit_kernels(plan, taps, ref_stride, kernels, theta, stream))


def tidas_forward(kernels, taps, nz, nx, refl, img, n_frames, variant, stream=0):
    return _check(load().tidas_forward(kernels, taps, nz, nx, refl, img, n_frames, variant, stream))


def tidas_adjoint(kernels, taps, nz, nx, img, refl, n_frames, variant, stream=0):
    return _check(load().tidas_adjoint(kernels, taps, nz, nx, img, refl, n_frames, variant, stream))


def tidas_fit_kernels_2d(plan, kz, taps, kernels, stream=0):
    return _check(load().tidas_fit_kernels_2d(plan, kz, taps, kernels, stream))


def tidas_forward_2d(kernels, kz, taps, nz, nx, refl, img, n_frames, variant, workspace=None,
                     workspace_bytes=0, stream=0):
    return _check(load().tidas_forward_2d(kernels, kz, taps, nz, nx, refl, img, n_frames, variant,
                                          workspace, workspace_bytes, stream))


def tidas_adjoint_2d(kernels, kz, taps, nz, nx, img, refl, n_frames, variant, workspace=None,
                     workspace_bytes=0, stream=0):
    return _check(load().tidas_adjoint_2d(kernels, kz, taps, nz, nx, img, refl, n_frames, variant,
                                          workspace, workspace_bytes, stream))


def tidas_forward_varying_2d(kernels, ld, kz, taps, nz, nx, refl, img, n_frames, variant,
                             stream=0):
    return _check(load().tidas_forward_varying_2d(kernels, ld, kz, taps, nz, nx, refl, img,
                                                  n_frames, variant, stream))


def tidas_forward_varying_2d_bf16k(kernels16, ld, kz, taps, nz, nx, refl, img, n_frames,
                                   stream=0):
    return _check(load().tidas_forward_varying_2d_bf16k(kernels16, ld, kz, taps, nz, nx, refl,
                                                        img, n_frames, stream))


def tidas_adjoint_varying_2d(kernels, ld, kz, taps, nz, nx, img, refl, n_frames, variant,
                             stream=0):
    return _check(load().tidas_adjoint_varying_2d(kernels, ld, kz, taps, nz, nx, img, refl,
                                                  n_frames, variant, stream))


def tidas_line_synthesize(p, r_first, n_scat, rf, stream=0):
    return _check(load().tidas_line_synthesize(ctypes.byref(p), r_first, n_scat, rf, stream))


def tidas_line_das(p, rf, n_scat, lines, stream=0):
    return _check(load().tidas_line_das(ctypes.byref(p), rf, n_scat, lines, stream))


def tidas_line_sweep(p, rf, lines, r_first, n_scat, eps, theta, err_local, err_global, stream=0):
    return _check(load().tidas_line_sweep(ctypes.byref(p), rf, lines, r_first, n_scat, eps, theta,
                                          err_local, err_global, stream))


def tidas_line_window(p):
    eps = ctypes.c_double()
    _check(load().tidas_line_window(ctypes.byref(p), ctypes.byref(eps)))
    return eps.value


def tidas_line_combine(p, rf, n_scat, amps, rf_line, stream=0):
    return _check(load().tidas_line_combine(ctypes.byref(p), rf, n_scat, amps, rf_line, stream))


def tidas_line_model(p, rf_line, s, theta, eps, out, stream=0):
    return _check(load().tidas_line_model(ctypes.byref(p), rf_line, s, theta, eps, out, stream))


def tidas_line_fixed(p, rf, r_first, n_scat, s, eps, out, stream=0):
    return _check(load().tidas_line_fixed(ctypes.byref(p), rf, r_first, n_scat, s, eps, out,
                                          stream))


def tidas_line_envelope(n_rows, n, x, env, stream=0):
    return _check(load().tidas_line_envelope(n_rows, n, x, env, stream))


def tidas_band_workspace_bytes(nz, nx, n_frames, variant):
    return load().tidas_band_workspace_bytes(nz, nx, n_frames, variant)


def tidas_dot(a, b, n, out, stream=0):
    return _check(load().tidas_dot(a, b, n, out, stream))


def tidas_dot_noalloc(a, b, n, out, stream=0):
    return _check(load().tidas_dot_noalloc(a, b, n, out, stream))


def tidas_asum(a, n, out, stream=0):
    return _check(load().tidas_asum(a, n, out, stream))


def tidas_fista_update(x, y, grad, n, step, thresh, beta, stream=0):
    return _check(load().tidas_fista_update(x, y, grad, n, step, thresh, beta, stream))


def tidas_axpby(a, b, out, n, alpha, beta, stream=0):
    return _check(load().tidas_axpby(a, b, out, n, alpha, beta, stream))


def call(name, *args):
    """Call any exported entry point by name, raising TidasError on failure."""
    return _check(getattr(load(), name)(*args))


def tidas_device_status():
    v = ctypes.c_int32(0)
    _check(load().tidas_device_status(ctypes.byref(v)))
    return v.value


def tidas_last_error():
    return load().tidas_last_error().decode(errors="replace")


def tidas_set_debug_option(option, value):
    return _check(load().tidas_set_debug_option(option, value))


def das_plan_read_window(plan):
    first, count = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().das_plan_read_window(plan, ctypes.byref(first), ctypes.byref(count)))
    return first.value, count.value
