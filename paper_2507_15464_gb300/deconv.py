"""Differentiable DAS / tiDAS operators and FISTA deconvolution.

The convolutional model exists, in the paper's words, to make deconvolution
possible (abstract, introduction and conclusion): min_x 1/2 ||H x - b||^2 +
lambda ||x||_1 with H either the exact operator (DAS of the channel data that
the reflectivity x produces, das_forward o das_synthesize_grid) or tiDAS
(tidas_forward).  torch.autograd.Function wrappers give backward = adjoint,
computed by the hand-written transpose kernels.  Every arithmetic step of the
iteration runs in libtidas.so kernels; torch supplies tensors and streams.
"""
import ctypes
import math

import torch

from . import capi
from .ops import DasPlan, _ptr, _stream, tidas_adjoint, tidas_forward


# ---------------------------------------------------------------- autograd
class _DasFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rf, plan):
        ctx.plan = plan
        return plan.forward(rf.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint(g.contiguous()), None


class _SynthGridFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, refl, plan):
        ctx.plan = plan
        return plan.synthesize_grid(refl.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.synthesize_adjoint(g.contiguous()), None


class _TidasFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, refl, kernels, variant):
        ctx.kernels, ctx.variant = kernels, variant
        return tidas_forward(kernels, refl.contiguous(), variant=variant)

    @staticmethod
    def backward(ctx, g):
        return tidas_adjoint(ctx.kernels, g.contiguous(), variant=ctx.variant), None, None


def das(rf, plan: DasPlan):
    """Delay and Sum with autograd (backward = das_adjoint); FP32 plans."""
    return _DasFn.apply(rf, plan)


def synthesize_grid(refl, plan: DasPlan):
    """Eq. (2.1) on the pixel grid with autograd (backward = das_synthesize_adjoint)."""
    return _SynthGridFn.apply(refl, plan)


def exact_operator(refl, plan: DasPlan):
    """H x = DAS(A x): reflectivity on the pixel grid -> beamformed image."""
    return das(synthesize_grid(refl, plan), plan)


def tidas(refl, kernels, variant=capi.VARIANT_DIRECT):
    """tiDAS with autograd; FP32 variants (DIRECT, GEMM_RESID)."""
    if variant == capi.VARIANT_GEMM_BF16:
        raise ValueError("autograd needs an FP32-input variant (DIRECT or GEMM_RESID)")
    return _TidasFn.apply(refl, kernels, variant)


# ------------------------------------------------------------- operators
class TidasOperator:
    """H = tiDAS with row kernels (Eq. (2.13)) for FISTA: forward(x, out) and
    adjoint(y, out) on [B, nz, nx] FP32 tensors."""

    def __init__(self, kernels, variant=capi.VARIANT_DIRECT):
        self.kernels, self.variant = kernels, variant

    def forward(self, x, out):
        return tidas_forward(self.kernels, x, variant=self.variant, out=out)

    def adjoint(self, y, out):
        return tidas_adjoint(self.kernels, y, variant=self.variant, out=out)


class TidasBandOperator:
    """tiDAS with 2D band kernels [nz, kz, taps] (the PSF's axial extent kept)."""

    def __init__(self, kernels, variant=capi.VARIANT_DIRECT):
        if variant != capi.VARIANT_DIRECT:
            raise ValueError("the band operator in FISTA runs on FP32 iterates (DIRECT)")
        self.kernels, self.variant = kernels, variant

    def forward(self, x, out):
        from .ops import tidas_forward_2d
        return tidas_forward_2d(self.kernels, x, variant=self.variant, out=out)

    def adjoint(self, y, out):
        from .ops import tidas_adjoint_2d
        return tidas_adjoint_2d(self.kernels, y, variant=self.variant, out=out)


class ExactOperator:
    """H = DAS of the channel data a reflectivity map produces (das_forward o
    das_synthesize_grid), with its exact transpose; FP32 plans."""

    def __init__(self, plan: DasPlan, frames=1):
        if plan.rf_dtype != torch.float32:
            raise ValueError("the exact operator needs an FP32 plan")
        self.plan = plan
        self.rf = torch.empty(plan.rf_shape(frames), dtype=torch.float32, device="cuda")

    def forward(self, x, out):
        self.plan.synthesize_grid(x, out=self.rf)
        return self.plan.forward(self.rf, out=out)

    def adjoint(self, y, out):
        self.plan.adjoint(y, out=self.rf)
        return self.plan.synthesize_adjoint(self.rf, out=out)


# ------------------------------------------------------------ primitives
def dot(a, b):
    """FP64 <a, b> of two float32 CUDA tensors, computed on the GPU."""
    out = torch.empty((), dtype=torch.float64, device=a.device)
    capi.tidas_dot(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream())
    return out


def asum(a):
    """FP64 sum of |a| of a float32 CUDA tensor (the L1 norm in the objective)."""
    out = torch.empty((), dtype=torch.float64, device=a.device)
    capi.tidas_asum(_ptr(a), a.numel(), _ptr(out), _stream())
    return out


def axpby(alpha, a, beta, b, out):
    """out = alpha a + beta b on float32 CUDA tensors."""
    capi.tidas_axpby(_ptr(a), _ptr(b), _ptr(out), a.numel(), alpha, beta, _stream())
    return out


def power_iteration(op, v0, iters=30):
    """Largest eigenvalue of H^T H by the power method from v0 (the random
    start is an input).  Returns (estimate, last unit vector)."""
    v = v0.clone()
    w = torch.empty_like(v)
    hv = None
    n0 = math.sqrt(float(dot(v, v)))
    axpby(1.0 / n0, v, 0.0, v, v)
    lam = 0.0
    for _ in range(iters):
        hv = op.forward(v, hv)
        op.adjoint(hv, w)
        lam = math.sqrt(float(dot(w, w)))
        axpby(1.0 / lam, w, 0.0, w, v)
    return lam, v


def objective(op, x, b, lam):
    """1/2 ||H x - b||^2 + lam ||x||_1 (FP64 reductions on the GPU)."""
    r = op.forward(x, None)
    axpby(1.0, r, -1.0, b, r)
    return 0.5 * float(dot(r, r)) + lam * float(asum(x))


def fista(op, b, lam, L, iters=200, x0=None):
    """FISTA with the L1 prior: x = soft(y - grad / L, lam / L), Nesterov
    momentum t' = (1 + sqrt(1 + 4 t^2)) / 2, y = x + (t - 1) / t' (x - x_prev).
    The momentum schedule is host arithmetic; all array work is in kernels."""
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    y = x.clone()
    hy = torch.empty_like(b)
    g = torch.empty_like(x)
    t = 1.0
    step, thresh = 1.0 / L, lam / L
    for _ in range(iters):
        op.forward(y, hy)
        axpby(1.0, hy, -1.0, b, hy)       # residual H y - b
        op.adjoint(hy, g)                 # gradient H^T (H y - b)
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        capi.tidas_fista_update(_ptr(x), _ptr(y), _ptr(g), x.numel(), step, thresh,
                                (t - 1.0) / t_next, _stream())
        t = t_next
    return x
