"""Torch-facing wrappers: allocate outputs as CUDA tensors, pass pointers and the
current stream to the C ABI.  Every operation runs in libtidas.so kernels;
torch only supplies device memory and streams.
"""
import ctypes
import math

import torch

from . import capi


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _need(t, dtype, shape, name):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError("%s: expected %s %s, got %s %s" % (name, dtype, tuple(shape), t.dtype,
                                                            tuple(t.shape)))


class DasPlan:
    """A das_plan for one geometry dict (tidas_workloads.presets form)."""

    def __init__(self, geom: dict, rf_dtype=torch.float32):
        self.geom = dict(geom)
        ang = geom.get("angles_rad")
        if ang is None:
            ang = [a * math.pi / 180.0 for a in geom["angles_deg"]]
        self._angles = (ctypes.c_double * len(ang))(*ang)
        p = capi.das_params()
        for k in ("n_elem", "n_samples", "nx", "nz", "interp"):
            setattr(p, k, int(geom[k]))
        for k in ("pitch", "f0", "fs", "c", "frac_bw", "t0", "x0", "dx", "z0", "dz", "fnum"):
            setattr(p, k, float(geom[k]))
        p.n_angles = len(ang)
        p.angles_rad = ctypes.cast(self._angles, ctypes.POINTER(ctypes.c_double))
        if rf_dtype not in (torch.float32, torch.float16):
            raise ValueError("rf_dtype must be float32 or float16")
        p.rf_dtype = capi.RF_F16 if rf_dtype == torch.float16 else capi.RF_F32
        self.rf_dtype = rf_dtype
        self.params = p
        self.handle = capi.das_plan_create(p)
        self.A, self.N, self.S = p.n_angles, p.n_elem, p.n_samples
        self.nx, self.nz = p.nx, p.nz

    def read_window(self):
        """(first sample, count) of the samples das_forward weights in every
        channel record; samples outside never change the image if finite."""
        return capi.das_plan_read_window(self.handle)

    def set_tensor_cores(self, on: bool):
        """Route batches of >= 16 FP16 frames to the tensor-core DAS (default) or not."""
        capi.call("das_plan_set_option", self.handle, 1, 1 if on else 0)

    def close(self):
        """Destroy the plan (frees its device tables; synchronises the device)."""
        if self.handle:
            capi.das_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes
    def rf_shape(self, nf):
        """Shape of nf frames of channel data: (frames, angles, elements, samples)."""
        return (nf, self.A, self.N, self.S)

    def img_shape(self, nf):
        """Shape of nf images or reflectivity maps: (frames, nz, nx)."""
        return (nf, self.nz, self.nx)

    # operations
    def synthesize(self, pos, amp, out=None):
        """pos [B, n, 2] float64, amp [B, n, 2] float32 (CUDA) -> rf [B, A, N, S]."""
        nf, n = pos.shape[0], pos.shape[1]
        _need(pos, torch.float64, (nf, n, 2), "pos")
        _need(amp, torch.float32, (nf, n, 2), "amp")
        out = out if out is not None else torch.empty(self.rf_shape(nf), dtype=self.rf_dtype,
                                                      device=pos.device)
        capi.das_synthesize(self.handle, _ptr(pos), _ptr(amp), n, nf, _ptr(out), _stream())
        return out

    def synthesize_grid(self, refl, out=None):
        """Eq. (2.1) for reflectivities on the pixel centres: refl [B, nz, nx] FP32 ->
        rf [B, A, N, S] FP32 (the forward operator of deconvolution)."""
        nf = refl.shape[0]
        _need(refl, torch.float32, self.img_shape(nf), "refl")
        out = out if out is not None else torch.empty(self.rf_shape(nf), dtype=torch.float32,
                                                      device=refl.device)
        capi.das_synthesize_grid(self.handle, _ptr(refl), _ptr(out), nf, _stream())
        return out

    def synthesize_adjoint(self, rf, out=None):
        """Transpose of synthesize_grid: rf [B, A, N, S] FP32 -> refl [B, nz, nx]."""
        nf = rf.shape[0]
        _need(rf, torch.float32, self.rf_shape(nf), "rf")
        out = out if out is not None else torch.empty(self.img_shape(nf), dtype=torch.float32,
                                                      device=rf.device)
        capi.das_synthesize_adjoint(self.handle, _ptr(rf), _ptr(out), nf, _stream())
        return out

    def forward(self, rf, out=None):
        """Eq. (2.2) Delay-and-Sum: rf [B, A, N, S] (the plan's dtype) -> img [B, nz, nx]
        FP32.  FP16 batches of >= 16 frames run on the tensor cores."""
        nf = rf.shape[0]
        _need(rf, self.rf_dtype, self.rf_shape(nf), "rf")
        out = out if out is not None else torch.empty(self.img_shape(nf), dtype=torch.float32,
                                                      device=rf.device)
        capi.das_forward(self.handle, _ptr(rf), _ptr(out), nf, _stream())
        return out

    def adjoint(self, img, out=None):
        """Transpose of forward for FP32 plans: img [B, nz, nx] -> rf [B, A, N, S]."""
        nf = img.shape[0]
        _need(img, torch.float32, self.img_shape(nf), "img")
        out = out if out is not None else torch.empty(self.rf_shape(nf), dtype=torch.float32,
                                                      device=img.device)
        capi.das_adjoint(self.handle, _ptr(img), _ptr(out), nf, _stream())
        return out

    def delay_table(self, angle, device="cuda"):
        """Bit-exact FP64 delay split of one angle: (idx int32, frac FP32), [nz, nx, N]."""
        idx = torch.empty((self.nz, self.nx, self.N), dtype=torch.int32, device=device)
        frac = torch.empty((self.nz, self.nx, self.N), dtype=torch.float32, device=device)
        capi.das_delay_table(self.handle, angle, _ptr(idx), _ptr(frac), _stream())
        return idx, frac

    def fit_kernels(self, taps, ref_stride=1, device="cuda"):
        """Row kernels of Eq. (2.13) from exact PSF rows (Eq. (2.6)-(2.7)) and their
        least-squares weights theta (Eq. (2.12)): (kernels [nz, taps], theta [nz])."""
        k = torch.empty((self.nz, taps), dtype=torch.float32, device=device)
        th = torch.empty((self.nz,), dtype=torch.float32, device=device)
        capi.tidas_fit_kernels(self.handle, taps, ref_stride, _ptr(k), _ptr(th), _stream())
        return k, th

    def fit_kernels_2d(self, kz, taps, device="cuda"):
        """2D band kernels [nz, kz, taps]: the image of a unit scatterer on each row."""
        k = torch.empty((self.nz, kz, taps), dtype=torch.float32, device=device)
        capi.tidas_fit_kernels_2d(self.handle, kz, taps, _ptr(k), _stream())
        return k


class DasStreamer:
    """Host batches through das_forward with the transfers overlapped.

    Two device batch buffers: while batch k is beamformed on the compute
    stream, batch k + 1 is uploaded on an upload stream and batch k - 1's
    image is read back on a download stream.  Every batch still makes its
    own host -> device and device -> host copy; events order the reuse of
    each buffer.  The upload copies the plan's read window of every record
    (das_upload_window: the samples DAS weights); the device buffers are
    zeroed once, so the samples outside stay finite and the images equal
    those of whole-record uploads.  There is a single compute stream, so the
    plan's staging buffer serves one batch at a time.  Destroying a plan
    synchronises the device (cudaFree), which drains the pipeline: keep plan
    lifetimes (and the garbage collector) out of the submission loop."""

    def __init__(self, plan: DasPlan, n_frames: int, device="cuda"):
        self.plan = plan
        self.n_frames = n_frames
        self.rf = [torch.zeros(plan.rf_shape(n_frames), dtype=plan.rf_dtype, device=device)
                   for _ in range(2)]
        first, count = plan.read_window()
        esize = self.rf[0].element_size()
        self.h2d_bytes = count * esize * (self.rf[0].numel() // plan.rf_shape(n_frames)[-1])
        self.img = [torch.empty(plan.img_shape(n_frames), dtype=torch.float32, device=device)
                    for _ in range(2)]
        self.up, self.comp, self.down = (torch.cuda.Stream() for _ in range(3))
        self.uploaded = [torch.cuda.Event() for _ in range(2)]
        self.computed = [torch.cuda.Event() for _ in range(2)]
        self.downloaded = [torch.cuda.Event() for _ in range(2)]
        self.used = [False, False]
        self.k = 0

    def submit(self, host_rf, host_img):
        """Queue one batch (pinned host tensors).  Returns the event after
        which host_img holds its image."""
        b = self.k & 1
        reuse = self.used[b]
        with torch.cuda.stream(self.up):
            if reuse:
                self.up.wait_event(self.computed[b])  # batch k - 2 has read rf[b]
            if not host_rf.is_pinned():
                raise ValueError("DasStreamer needs page-locked host batches")
            _need(host_rf, self.plan.rf_dtype, self.rf[b].shape, "host_rf")
            capi.call("das_upload_window", self.plan.handle, host_rf.data_ptr(),
                      _ptr(self.rf[b]), self.n_frames, self.up.cuda_stream)
            self.uploaded[b].record(self.up)
        with torch.cuda.stream(self.comp):
            self.comp.wait_event(self.uploaded[b])
            if reuse:
                self.comp.wait_event(self.downloaded[b])  # img[b] of batch k - 2 is out
            self.plan.forward(self.rf[b], out=self.img[b])
            self.computed[b].record(self.comp)
        with torch.cuda.stream(self.down):
            self.down.wait_event(self.computed[b])
            host_img.copy_(self.img[b], non_blocking=True)
            self.downloaded[b].record(self.down)
        self.used[b] = True
        self.k += 1
        return self.downloaded[b]


def _tidas(fn, kernels, x, variant, out=None):
    nz, taps = kernels.shape
    nf, nz2, nx = x.shape
    if nz2 != nz:
        raise ValueError("kernel rows and image rows differ")
    _need(kernels, torch.float32, (nz, taps), "kernels")
    want = torch.bfloat16 if variant == capi.VARIANT_GEMM_BF16 else torch.float32
    _need(x, want, (nf, nz, nx), "input")
    out = out if out is not None else torch.empty((nf, nz, nx), dtype=torch.float32,
                                                  device=x.device)
    fn(_ptr(kernels), taps, nz, nx, _ptr(x), _ptr(out), nf, variant, _stream())
    return out


def tidas_forward(kernels, refl, variant=capi.VARIANT_DIRECT, out=None):
    """Eq. (2.13) row-wise lateral convolution: refl [B, nz, nx] -> img [B, nz, nx]."""
    return _tidas(capi.tidas_forward, kernels, refl, variant, out)


def tidas_adjoint(kernels, img, variant=capi.VARIANT_DIRECT, out=None):
    """Transpose of tidas_forward (correlation with each row's kernel)."""
    return _tidas(capi.tidas_adjoint, kernels, img, variant, out)


def _tidas2d(fn, kernels, x, variant, out=None, workspace=None):
    nz, kz, taps = kernels.shape
    nf, nz2, nx = x.shape
    if nz2 != nz:
        raise ValueError("kernel rows and image rows differ")
    _need(kernels, torch.float32, (nz, kz, taps), "kernels")
    want = torch.bfloat16 if variant == capi.VARIANT_GEMM_BF16 else torch.float32
    _need(x, want, (nf, nz, nx), "input")
    out = out if out is not None else torch.empty((nf, nz, nx), dtype=torch.float32,
                                                  device=x.device)
    ws, wsb = None, 0
    if workspace is not None:
        ws, wsb = _ptr(workspace), workspace.numel() * workspace.element_size()
    fn(_ptr(kernels), kz, taps, nz, nx, _ptr(x), _ptr(out), nf, variant, ws, wsb, _stream())
    return out


def band_workspace(nz, nx, n_frames, variant, device="cuda"):
    """Scratch for the 2D band calls (None when the variant needs none)."""
    n = capi.tidas_band_workspace_bytes(nz, nx, n_frames, variant)
    return torch.empty((n,), dtype=torch.uint8, device=device) if n else None


def tidas_forward_2d(kernels, refl, variant=capi.VARIANT_DIRECT, out=None, workspace=None):
    """Eq. (2.13) with 2D band kernels: refl [B, nz, nx] -> img [B, nz, nx]."""
    return _tidas2d(capi.tidas_forward_2d, kernels, refl, variant, out, workspace)


def tidas_adjoint_2d(kernels, img, variant=capi.VARIANT_DIRECT, out=None, workspace=None):
    """Transpose of tidas_forward_2d: img [B, nz, nx] -> refl [B, nz, nx]."""
    return _tidas2d(capi.tidas_adjoint_2d, kernels, img, variant, out, workspace)


def _varying(fn, kernels, x, variant, out=None, taps=None):
    if kernels.dim() == 3:
        nz, nx, ld = kernels.shape
        kz = 1
    else:
        nz, nx, kz, ld = kernels.shape
    taps = ld if taps is None else taps
    nf = x.shape[0]
    k16 = kernels.dtype == torch.bfloat16
    if k16 and (fn is not capi.tidas_forward_varying_2d or variant != capi.VARIANT_GEMM_BF16):
        raise ValueError("BF16 kernels serve the forward tensor-core variant only")
    _need(kernels, torch.bfloat16 if k16 else torch.float32, tuple(kernels.shape), "kernels")
    want = torch.bfloat16 if variant == capi.VARIANT_GEMM_BF16 else torch.float32
    _need(x, want, (nf, nz, nx), "input")
    out = out if out is not None else torch.empty((nf, nz, nx), dtype=torch.float32,
                                                  device=x.device)
    if k16:
        capi.tidas_forward_varying_2d_bf16k(_ptr(kernels), ld, kz, taps, nz, nx, _ptr(x), _ptr(out),
                                            nf, _stream())
    else:
        fn(_ptr(kernels), ld, kz, taps, nz, nx, _ptr(x), _ptr(out), nf, variant, _stream())
    return out


def tidas_forward_varying(kernels, refl, variant=capi.VARIANT_DIRECT, out=None, taps=None):
    """Eq. (2.13) with a kernel per pixel (each pixel adds its own
    single-scatterer image): kernels [nz, nx, taps] (row form) or
    [nz, nx, kz, taps] (band form), refl [B, nz, nx] -> img [B, nz, nx].
    VARIANT_DIRECT: FP32 refl on CUDA cores; VARIANT_GEMM_BF16: BF16 refl on
    the tcgen05 tensor cores, with FP32 kernels or BF16 kernels (half the
    bytes; FP32 kernels rounded to BF16 give the same image).  The last
    kernel axis is the row pitch; taps (default: all of it) are the columns
    in use."""
    return _varying(capi.tidas_forward_varying_2d, kernels, refl, variant, out, taps)


def tidas_adjoint_varying(kernels, img, variant=capi.VARIANT_DIRECT, out=None, taps=None):
    """Transpose of tidas_forward_varying: img [B, nz, nx] -> refl [B, nz, nx]."""
    return _varying(capi.tidas_adjoint_varying_2d, kernels, img, variant, out, taps)


class LineExperiment:
    """The single-line experiment of Section 3 on the GPU: channel data of a
    unit scatterer on every line point, DAS lines, and the sweep of Eq. (2.8)
    / (2.12) over every (delay curve, scatterer) pair.  `p` is a dict with the
    tidas_line_params fields."""

    def __init__(self, p: dict):
        self.p = dict(p)
        self.P = capi.line_params(**{k: self.p[k] for k, _ in capi.line_params._fields_})
        self.N, self.S, self.D = self.P.n_elem, self.P.n_samples, self.P.n_depths

    def window(self):
        """Half the FWHM of the focal-point PSF (the window of Section 3.2)."""
        return capi.tidas_line_window(self.P)

    def depth(self, i):
        """Depth in metres of line point i (points evenly spaced from z_first to z_last)."""
        return self.P.z_first + (self.P.z_last - self.P.z_first) * i / (self.D - 1)

    def synthesize(self, r_first=0, n_scat=None, out=None, device="cuda"):
        """Channel data [n_scat, N, S] of a unit scatterer on each line point from
        r_first on, under the focused transmit (Eq. (2.1))."""
        n_scat = self.D - r_first if n_scat is None else n_scat
        out = out if out is not None else torch.empty((n_scat, self.N, self.S),
                                                      dtype=torch.float32, device=device)
        _need(out, torch.float32, (n_scat, self.N, self.S), "rf")
        capi.tidas_line_synthesize(self.P, r_first, n_scat, _ptr(out), _stream())
        return out

    def das_lines(self, rf, out=None):
        """DAS lines [n, n_depths] of channel data [n, N, S] (Eq. (2.7) with dynamic focus)."""
        n = rf.shape[0]
        _need(rf, torch.float32, (n, self.N, self.S), "rf")
        out = out if out is not None else torch.empty((n, self.D), dtype=torch.float32,
                                                      device=rf.device)
        capi.tidas_line_das(self.P, _ptr(rf), n, _ptr(out), _stream())
        return out

    def sweep(self, rf, lines, eps, r_first=0):
        """theta, local error, global error: [n_depths curves, n_scat scatterers]."""
        n = rf.shape[0]
        _need(rf, torch.float32, (n, self.N, self.S), "rf")
        _need(lines, torch.float32, (n, self.D), "lines")
        outs = [torch.empty((self.D, n), dtype=torch.float32, device=rf.device) for _ in range(3)]
        capi.tidas_line_sweep(self.P, _ptr(rf), _ptr(lines), r_first, n, float(eps),
                              *[_ptr(o) for o in outs], _stream())
        return tuple(outs)

    def fixed_lines(self, rf, s, eps, r_first=0, out=None):
        """theta a_s for every scatterer under delay curve s: [n_scat, n_depths]."""
        n = rf.shape[0]
        _need(rf, torch.float32, (n, self.N, self.S), "rf")
        out = out if out is not None else torch.empty((n, self.D), dtype=torch.float32,
                                                      device=rf.device)
        capi.tidas_line_fixed(self.P, _ptr(rf), r_first, n, int(s), float(eps), _ptr(out),
                              _stream())
        return out

    def combine(self, rf, amps, out=None):
        """Channel data of a line of scatterers, amps[r] on point r."""
        n = rf.shape[0]
        _need(rf, torch.float32, (n, self.N, self.S), "rf")
        _need(amps, torch.float32, (n,), "amps")
        out = out if out is not None else torch.empty((self.N, self.S), dtype=torch.float32,
                                                      device=rf.device)
        capi.tidas_line_combine(self.P, _ptr(rf), n, _ptr(amps), _ptr(out), _stream())
        return out

    def model(self, rf_line, s, theta, eps, out=None):
        """Eq. (2.13): the line model with delay curve s and weights theta."""
        _need(rf_line, torch.float32, (self.N, self.S), "rf_line")
        _need(theta, torch.float32, (self.D,), "theta")
        out = out if out is not None else torch.empty((self.D,), dtype=torch.float32,
                                                      device=rf_line.device)
        capi.tidas_line_model(self.P, _ptr(rf_line), int(s), _ptr(theta), float(eps), _ptr(out),
                              _stream())
        return out


def envelope(x, out=None):
    """Envelope of each row of x [rows, n] (modulus of the analytic signal)."""
    x2 = x.reshape(-1, x.shape[-1])
    _need(x2, torch.float32, tuple(x2.shape), "x")
    out = out if out is not None else torch.empty_like(x2)
    capi.tidas_line_envelope(x2.shape[0], x2.shape[1], _ptr(x2), _ptr(out), _stream())
    return out.reshape(x.shape)
