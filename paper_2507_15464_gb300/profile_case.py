"""Run one kernel case a few times on synthetic inputs, for profilers.

python -m paper_2507_15464_gb300.profile_case das --frames 8 --dtype f16 --iters 3
python -m paper_2507_15464_gb300.profile_case tidas --variant 1 --frames 64 --iters 3
python -m paper_2507_15464_gb300.profile_case tidas2d --variant 1 --kz 16 --frames 256 --iters 3
python -m paper_2507_15464_gb300.profile_case line --iters 2
python -m paper_2507_15464_gb300.profile_case mlp --kernels 524288 --iters 3

Inputs are seeded random arrays of the benchmark's shapes (the kernels'
cost does not depend on the values); nothing is checked here.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["das", "das_adjoint", "tidas", "tidas_adjoint", "tidas2d",
                                        "tidas2d_adjoint", "line", "mlp"])
    ap.add_argument("--frames", type=int, default=8)
    ap.add_argument("--dtype", default="f16", choices=["f16", "f32"])
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--kz", type=int, default=16)
    ap.add_argument("--geom", default="pw128_compound")
    ap.add_argument("--kernels", type=int, default=524288)
    a = ap.parse_args()

    import torch
    from paper_2507_15464_gb300 import ops
    from tidas_workloads import presets
    g = presets.geometry(a.geom)
    gen = torch.Generator(device="cuda").manual_seed(0)
    if a.case == "mlp":
        # fused inference of the kernel generator (untrained weights): samples
        # uniform over its (x, z, F#, angle) domain
        from paper_2507_15464_gb300 import generator
        P = ops.DasPlan(g)
        net = generator.KernelMLP()
        lo = torch.tensor(generator.BOUNDS_LO, dtype=torch.float64, device="cuda")
        hi = torch.tensor(generator.BOUNDS_HI, dtype=torch.float64, device="cuda")
        u = torch.rand((a.kernels, 4), dtype=torch.float64, device="cuda", generator=gen)
        s = lo + u * (hi - lo)
        fn = lambda: net.infer(P, s)
    elif a.case == "line":
        # the single-line experiment: 600 points, 192 elements, focus 25 mm
        p = dict(n_elem=192, pitch=0.3e-3, f0=5e6, fs=40e6, c=1540.0, frac_bw=0.6,
                 n_samples=2560, n_depths=600, z_first=2e-3, z_last=42e-3, z_focus=25e-3,
                 kossoff=0.6, fnum_rx=1.0, interp=1)
        E = ops.LineExperiment(p)
        eps = E.window()
        rf = E.synthesize()
        lines = E.das_lines(rf)

        def fn():
            E.synthesize(out=rf)
            E.das_lines(rf, out=lines)
            E.sweep(rf, lines, eps)
    elif a.case in ("das", "das_adjoint"):
        dt = torch.float16 if (a.dtype == "f16" and a.case == "das") else torch.float32
        P = ops.DasPlan(g, rf_dtype=dt)
        if a.case == "das":
            x = torch.randn(P.rf_shape(a.frames), device="cuda", generator=gen).to(dt)
            fn = lambda: P.forward(x)
        else:
            x = torch.randn(P.img_shape(a.frames), device="cuda", generator=gen)
            fn = lambda: P.adjoint(x)
    else:
        nz, nx = g["nz"], g["nx"]
        band = a.case.startswith("tidas2d")
        k = torch.randn((nz, a.kz, 63) if band else (nz, 63), device="cuda", generator=gen)
        x = torch.randn((a.frames, nz, nx), device="cuda", generator=gen)
        if a.variant == 1:
            x = x.to(torch.bfloat16)
        if band:
            f = ops.tidas_forward_2d if a.case == "tidas2d" else ops.tidas_adjoint_2d
        else:
            f = ops.tidas_forward if a.case == "tidas" else ops.tidas_adjoint
        fn = lambda: f(k, x, variant=a.variant)
    for _ in range(a.iters):
        fn()
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
