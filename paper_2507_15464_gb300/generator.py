"""Learned tiDAS kernel generator: a 4-layer MLP (4 -> 256 -> 256 -> 256 -> 63,
or -> kz x 63 for band kernels) mapping (lateral x, depth z, receive
f-number, transmit angle) to the normalised row kernel (or the kz-row band
patch of the same PSF), trained on exact single-scatterer PSFs.

The paper's conclusion names learned scaling parameters as the way forward;
the network extends that to the whole kernel and to any (x, F#, angle).
Training runs in BF16 on tcgen05 tensor cores with FP32 master weights and
AdamW; every array operation is a libtidas.so kernel (tidas_gemm_bf16,
tidas_relu_backward, tidas_colsum, tidas_adam, tidas_mse, tidas_transpose_bf16,
tidas_gather_rows, tidas_encode).  torch supplies memory and streams; the
host only sequences calls and computes the learning-rate schedule.

Targets are PSF rows divided by the sum of the apodization weights at the
scatterer (so the centre tap is ~1); inference multiplies the network output
back by that sum (tidas_apod_sum, tidas_row_scale).  Where a learned kernel's
NRMSE against the exact kernel exceeds a threshold, the exact kernel is used
(tidas_kernel_fallback).
"""
import ctypes
import math

import numpy as np
import torch

from . import capi
from .ops import _ptr, _stream

TAPS = 63
SLOT = 64    # output columns per kernel row (column 63 of each row is padding)
OUT = SLOT   # padded output width of the row-kernel network
IN = 64      # padded input width (4 features)
HID = 256


def layers(kz=1):
    """(out, in) of the four linear layers; the output holds kz rows of SLOT."""
    return [(HID, IN), (HID, HID), (HID, HID), (kz * SLOT, HID)]


LAYERS = layers(1)
BOUNDS_LO = (-19.2e-3, 5e-3, 1.0, -math.radians(15.0))
BOUNDS_HI = (19.2e-3, 60e-3, 3.0, math.radians(15.0))


def init_params(seed=5, kz=1):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (seeded,
    drawn on the host by the shared generator module)."""
    from tidas_workloads import generators
    params = []
    lay = layers(kz)
    for li, (o, i) in enumerate(lay):
        fan_in = 4 if li == 0 else i
        bound = 1.0 / math.sqrt(fan_in)
        w = generators.uniform((o, i), -bound, bound, (seed, li), np.float32)
        if li == 0:
            w[:, 4:] = 0.0  # padded input columns
        if li == len(lay) - 1:
            w.reshape(kz, SLOT, i)[:, TAPS:, :] = 0.0  # padding column of each kernel row
        params.append((w, np.zeros(o, np.float32)))
    return params


def _bf16(shape):
    return torch.empty(shape, dtype=torch.bfloat16, device="cuda")


def _f32(shape):
    return torch.empty(shape, dtype=torch.float32, device="cuda")


class KernelMLP:
    """The kernel generator 4 -> 256 -> 256 -> 256 -> kz x 63 (ReLU between
    layers; kz = 1: the row kernel): FP32 master weights with BF16 copies for
    the tensor cores, AdamW training (fit), inference (infer: one fused launch
    for row kernels, the layer path for band kernels) and the layer-by-layer
    path (infer_layers).  The output row of a sample holds kz kernel rows of
    SLOT columns (the layout [kz][SLOT] of the varying tiDAS calls).
    `params` is a list of (W [out, in], b [out]) float32 arrays, seeded by
    init_params() when omitted."""

    def __init__(self, params=None, batch=256, kz=1):
        params = params or init_params(kz=kz)
        self.kz = kz
        self.out = kz * SLOT
        # loss columns: the 63 taps of a row kernel; every column of a band
        # patch (the padding columns' targets are zero)
        self.used = TAPS if kz == 1 else self.out
        self.B = batch
        self.W, self.b, self.W16, self.W16t, self.mW, self.vW, self.mb, self.vb = ([] for _ in range(8))
        for (w, b) in params:
            W = torch.from_numpy(np.ascontiguousarray(w)).cuda()
            self.W.append(W)
            self.b.append(torch.from_numpy(np.ascontiguousarray(b)).cuda())
            self.W16.append(_bf16(W.shape))
            self.W16t.append(_bf16((W.shape[1], W.shape[0])))
            for lst, shp in ((self.mW, W.shape), (self.vW, W.shape), (self.mb, b.shape),
                             (self.vb, b.shape)):
                lst.append(torch.zeros(shp, dtype=torch.float32, device="cuda"))
        self.lo = torch.tensor(BOUNDS_LO, dtype=torch.float32, device="cuda")
        self.hi = torch.tensor(BOUNDS_HI, dtype=torch.float32, device="cuda")
        self.step_count = 0
        self._refresh_bf16()
        self._alloc_train(batch)

    # copies of the master weights in BF16 (and transposed) via a zero-lr Adam pass
    def _refresh_bf16(self):
        zero = [torch.zeros_like(W) for W in self.W]
        for l, W in enumerate(self.W):
            o, i = W.shape
            m = torch.zeros_like(W)
            v = torch.zeros_like(W)
            capi.call("tidas_adam", _ptr(W), _ptr(m), _ptr(v), _ptr(zero[l]), o, i, 0.0, 0.9,
                      0.999, 1e-8, 0.0, 1, _ptr(self.W16[l]), _ptr(self.W16t[l]), _stream())

    def _alloc_train(self, B):
        self.x16, self.x16t = _bf16((B, IN)), _bf16((IN, B))
        self.h32 = [_f32((B, HID)) for _ in range(3)]
        self.h16 = [_bf16((B, HID)) for _ in range(3)]
        self.h16t = [_bf16((HID, B)) for _ in range(3)]
        O = self.out
        self.y32 = _f32((B, O))
        self.dy32, self.dy16, self.dy16t = _f32((B, O)), _bf16((B, O)), _bf16((O, B))
        self.dh32 = _f32((B, HID))
        self.dz32 = [_f32((B, HID)) for _ in range(3)]
        self.dz16 = [_bf16((B, HID)) for _ in range(3)]
        self.dz16t = [_bf16((HID, B)) for _ in range(3)]
        self.gW = [torch.empty_like(W) for W in self.W]
        self.gb = [torch.empty_like(b) for b in self.b]
        self.loss = torch.zeros((), dtype=torch.float64, device="cuda")
        self.tgt = _f32((B, O))

    # ------------------------------------------------------------ primitives
    def encode(self, samples, out16):
        """(x, z, F#, angle) samples [n, 4] float64 -> inputs [n, 64] BF16 in [-1, 1]
        (the four features, zero padding)."""
        capi.call("tidas_encode", _ptr(samples), samples.shape[0], _ptr(self.lo), _ptr(self.hi),
                  _ptr(out16), _stream())

    @staticmethod
    def gemm(A, B, M, N, K, bias, relu, c32, c16, ldc):
        """C = act(A B^T + bias) on the tensor cores, BF16 A [M, K] and B [N, K],
        FP32 (c32) and / or BF16 (c16) outputs with leading dimension ldc."""
        capi.call("tidas_gemm_bf16", _ptr(A), _ptr(B), M, N, K,
                  _ptr(bias) if bias is not None else None, 1 if relu else 0,
                  _ptr(c32) if c32 is not None else None,
                  _ptr(c16) if c16 is not None else None, ldc, _stream())

    def forward_into(self, x16, M, h32, h16, y32):
        """Forward pass of M encoded rows: hidden activations (BF16, and FP32
        when h32 is given, for training) and the FP32 output [M, 64]."""
        a = x16
        for l in range(3):
            self.gemm(a, self.W16[l], M, HID, a.shape[1], self.b[l], True,
                      h32[l] if h32 is not None else None, h16[l], HID)
            a = h16[l]
        self.gemm(a, self.W16[3], M, self.out, HID, self.b[3], False, y32, None, self.out)

    # --------------------------------------------------------------- training
    def train_step(self, x16, target, lr, wd=1e-4):
        """One AdamW step on a mini-batch (x16 [B, 64] BF16, target [B, out] FP32).
        Returns nothing; the batch loss is left in self.loss (device)."""
        B = self.B
        OUT = self.out
        st = _stream()
        self.forward_into(x16, B, self.h32, self.h16, self.y32)
        capi.call("tidas_mse", _ptr(self.y32), _ptr(target), B, self.used, OUT, OUT, _ptr(self.dy32),
                  _ptr(self.loss), st)
        # output layer
        capi.call("tidas_relu_backward", _ptr(self.dy32), None, B * OUT, None, _ptr(self.dy16), st)
        capi.call("tidas_transpose_bf16", _ptr(self.dy16), B, OUT, _ptr(self.dy16t), st)
        for l in range(3):
            capi.call("tidas_transpose_bf16", _ptr(self.h16[l]), B, HID, _ptr(self.h16t[l]), st)
        capi.call("tidas_transpose_bf16", _ptr(x16), B, IN, _ptr(self.x16t), st)
        self.gemm(self.dy16t, self.h16t[2], OUT, HID, B, None, False, self.gW[3], None, HID)
        capi.call("tidas_colsum", _ptr(self.dy32), B, OUT, OUT, _ptr(self.gb[3]), st)
        g16 = self.dy16
        for l in (2, 1, 0):
            # dH_l = dZ_{l+1} W_{l+1}  (B x 256)
            K = OUT if l == 2 else HID
            self.gemm(g16, self.W16t[l + 1], B, HID, K, None, False, self.dh32, None, HID)
            capi.call("tidas_relu_backward", _ptr(self.dh32), _ptr(self.h32[l]), B * HID,
                      _ptr(self.dz32[l]), _ptr(self.dz16[l]), st)
            capi.call("tidas_transpose_bf16", _ptr(self.dz16[l]), B, HID, _ptr(self.dz16t[l]), st)
            prev_t = self.h16t[l - 1] if l > 0 else self.x16t
            n_in = HID if l > 0 else IN
            self.gemm(self.dz16t[l], prev_t, HID, n_in, B, None, False, self.gW[l], None, n_in)
            capi.call("tidas_colsum", _ptr(self.dz32[l]), B, HID, HID, _ptr(self.gb[l]), st)
            g16 = self.dz16[l]
        self.step_count += 1
        t = self.step_count
        for l, W in enumerate(self.W):
            o, i = W.shape
            capi.call("tidas_adam", _ptr(W), _ptr(self.mW[l]), _ptr(self.vW[l]), _ptr(self.gW[l]),
                      o, i, lr, 0.9, 0.999, 1e-8, wd, t, _ptr(self.W16[l]), _ptr(self.W16t[l]), st)
            capi.call("tidas_adam", _ptr(self.b[l]), _ptr(self.mb[l]), _ptr(self.vb[l]),
                      _ptr(self.gb[l]), 1, o, lr, 0.9, 0.999, 1e-8, 0.0, t, None, None, st)

    def fit(self, x16_all, targets_all, epochs, perms, lr0=1e-3, log_every=0, first_epoch=0,
            total_epochs=None):
        """Mini-batch AdamW over the whole set for epochs first_epoch ..
        epochs - 1 of a run of total_epochs (default: epochs) with the given
        per-epoch permutations (int32 [>= epochs, n], an input), cosine
        schedule over the whole run.  first_epoch > 0 resumes a run restored
        by load_checkpoint."""
        n = x16_all.shape[0]
        steps_per_epoch = n // self.B
        total = (total_epochs or epochs) * steps_per_epoch
        xb, tb = _bf16((self.B, IN)), _f32((self.B, self.out))
        losses = []
        k = first_epoch * steps_per_epoch
        for e in range(first_epoch, epochs):
            perm = perms[e]
            for s in range(steps_per_epoch):
                idx = perm[s * self.B:(s + 1) * self.B]
                capi.call("tidas_gather_rows", _ptr(x16_all), _ptr(idx), self.B, IN * 2, _ptr(xb),
                          _stream())
                capi.call("tidas_gather_rows", _ptr(targets_all), _ptr(idx), self.B, self.out * 4,
                          _ptr(tb), _stream())
                lr = 0.5 * lr0 * (1.0 + math.cos(math.pi * k / total))
                self.train_step(xb, tb, lr)
                k += 1
            if log_every and (e % log_every == 0 or e == epochs - 1):
                losses.append((e, float(self.loss)))
        return losses

    # ------------------------------------------------------- checkpoint / resume
    def save_checkpoint(self, path):
        """Write the FP32 master weights and biases, the Adam moments and the
        step count to an .npz file: all the state a resumed run needs (the
        BF16 copies are rebuilt from the masters on load)."""
        arrays = {"step": np.array(self.step_count, np.int64), "kz": np.array(self.kz, np.int64)}
        for l in range(len(self.W)):
            for name, lst in (("W", self.W), ("b", self.b), ("mW", self.mW), ("vW", self.vW),
                              ("mb", self.mb), ("vb", self.vb)):
                arrays["%s%d" % (name, l)] = lst[l].cpu().numpy()
        np.savez(path, **arrays)

    @classmethod
    def load_checkpoint(cls, path, batch=256):
        """A network restored from save_checkpoint: masters, moments and step
        count as saved, BF16 copies rebuilt."""
        with np.load(path) as z:
            nl = len(LAYERS)
            params = [(z["W%d" % l], z["b%d" % l]) for l in range(nl)]
            net = cls(params, batch=batch, kz=int(z["kz"]) if "kz" in z else 1)
            for l in range(nl):
                for name, lst in (("mW", net.mW), ("vW", net.vW), ("mb", net.mb), ("vb", net.vb)):
                    lst[l].copy_(torch.from_numpy(z["%s%d" % (name, l)]))
            net.step_count = int(z["step"])
        return net

    # -------------------------------------------------------------- inference
    def infer(self, plan, samples, chunk=None):
        """Kernels [n, out] (63 taps per row of SLOT, kz rows for a band patch)
        for samples [n, 4] float64 on the GPU: one fused launch (encode, four
        BF16 layers, scale by the apodization sum) for 64, 128, 192, 256 or
        512 outputs; other band heights take the layer path."""
        if self.out not in (64, 128, 192, 256, 512):
            # band heights the fused kernel's output chunks do not cover
            return self.infer_layers(plan, samples)
        n = samples.shape[0]
        out = _f32((n, self.out))
        scale = _f32((n,))
        capi.call("tidas_apod_sum", plan.handle, _ptr(samples), n, _ptr(scale), _stream())
        lo = (ctypes.c_float * 4)(*BOUNDS_LO)
        hi = (ctypes.c_float * 4)(*BOUNDS_HI)
        w = (ctypes.c_void_p * 4)(*[_ptr(W) for W in self.W16])
        b = (ctypes.c_void_p * 4)(*[_ptr(v) for v in self.b])
        capi.call("tidas_mlp_infer", _ptr(samples), n, lo, hi, w, b, _ptr(scale), _ptr(out),
                  self.out, self.out, _stream())
        return out

    def infer_layers(self, plan, samples, chunk=131072):
        """The same kernels through the layer-by-layer GEMM (tidas_gemm_bf16):
        the reference path of the fused kernel."""
        n = samples.shape[0]
        out = _f32((n, self.out))
        scale = _f32((n,))
        capi.call("tidas_apod_sum", plan.handle, _ptr(samples), n, _ptr(scale), _stream())
        c = min(chunk, n)
        x16 = _bf16((c, IN))
        h16 = [_bf16((c, HID)) for _ in range(3)]
        for s0 in range(0, n, chunk):
            m = min(chunk, n - s0)
            self.encode(samples[s0:s0 + m], x16[:m])
            self.forward_into(x16[:m], m, None, [h[:m] for h in h16], out[s0:s0 + m])
        capi.call("tidas_row_scale", _ptr(out), self.out, _ptr(scale), n, self.used, _ptr(out),
                  self.out, _stream())
        return out


def exact_kernels(plan, samples, normalise=False, kz=1):
    """Exact PSF rows [n, 64] (kz = 1) or band patches [n, kz * 64] (rows of
    SLOT columns) for samples [n, 4] (float64, CUDA)."""
    n = samples.shape[0]
    out = _f32((n, kz * SLOT))
    norm = _f32((n,)) if normalise else None
    if kz == 1:
        capi.call("tidas_psf_batch", plan.handle, _ptr(samples), n, TAPS, _ptr(out), OUT,
                  _ptr(norm) if norm is not None else None, _stream())
    else:
        capi.call("tidas_psf_batch_2d", plan.handle, _ptr(samples), n, kz, TAPS, SLOT, _ptr(out),
                  kz * SLOT, _ptr(norm) if norm is not None else None, _stream())
    return (out, norm) if normalise else out


def training_set(plan, n=20000, seed=4, kz=1):
    """(samples, normalised exact targets) for n uniform draws of (x, z, F#,
    angle) over the generator's domain; band patches of kz rows for kz > 1."""
    from tidas_workloads import generators
    lo, hi = np.array(BOUNDS_LO), np.array(BOUNDS_HI)
    u = generators.uniform((n, 4), 0.0, 1.0, (seed,), np.float64)
    s = torch.from_numpy(lo + u * (hi - lo)).cuda()
    tgt, _ = exact_kernels(plan, s, normalise=True, kz=kz)
    return s, tgt


def grid_samples(geom, fnum, angle_rad):
    """(x, z, F#, angle) of every pixel of a grid geometry, row-major."""
    xs = geom["x0"] + (np.arange(geom["nx"]) + 0.5) * geom["dx"]
    zs = geom["z0"] + (np.arange(geom["nz"]) + 0.5) * geom["dz"]
    X, Z = np.meshgrid(xs, zs)
    s = np.stack([X.ravel(), Z.ravel(), np.full(X.size, fnum), np.full(X.size, angle_rad)], 1)
    return torch.from_numpy(np.ascontiguousarray(s)).cuda()
