"""Throughput benchmark: exact compounded-plane-wave DAS (and tiDAS beside it)
on one GB300, in Mpixels/s, with roofline fractions and the FP64 CPU oracle
timed on the host cores in the same run.

Workload: 128-element linear array, 11 plane waves (-10..+10 deg), 4096
samples per channel, 512 x 1024 pixel grid, cubic interpolation, F# 1.5;
64 frames of FP16 channel data synthesised from 100k complex-Gaussian speckle
scatterers plus 10 bright targets per frame.  One step = das_forward over the
64-frame batch (inputs resident in HBM; the 738 MB batch exceeds the 129 MB
L2, so every step streams it from HBM).  tiDAS is timed on 256 frames of
1024 x 512 sparse reflectivity with 63-tap kernels fitted from the same
geometry.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
python bench.py --profile-case CASE [--frames F] [--dtype f16|f32] [--variant V]
                [--kz KZ] [--kernels N] [--iters I] [--density P]

--profile-case runs one kernel case a few times on seeded random inputs of
the benchmark's shapes and prints nothing but "ok": the command that the
profiler summaries run under ncu.  Nothing is timed or checked there.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixels/s exact DAS vs tiDAS on 1 GB300 at stated NRMSE vs FP64 oracle; % HBM/tensor peak"
GEOM = "pw128_compound"
BATCH = 64
TIDAS_FRAMES = 256
TAPS = 63
KZ = 16  # rows of the 2D band kernels


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tidas", action="store_true")
    ap.add_argument("--no-fista", action="store_true")
    ap.add_argument("--no-line", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-config1", action="store_true")
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--fista-iters", type=int, default=200)
    ap.add_argument("--profile-case", default=None,
                    choices=["das", "das_adjoint", "tidas", "tidas_adjoint", "tidas2d",
                             "tidas2d_adjoint", "varying", "line", "mlp", "synth",
                             "synth_adjoint"])
    ap.add_argument("--frames", type=int, default=8)
    ap.add_argument("--dtype", default="f16", choices=["f16", "f32"])
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--kz", type=int, default=16)
    ap.add_argument("--geom", default=GEOM)
    ap.add_argument("--kernels", type=int, default=524288)
    ap.add_argument("--density", type=float, default=1.0,
                    help="synth: fraction of nonzero pixels of the reflectivity map")
    return ap.parse_args()


def run_profile_case(a):
    """One kernel case, a.iters times, on seeded random inputs (the kernels'
    cost does not depend on the values)."""
    import torch
    from paper_2507_15464_gb300 import ops
    from tidas_workloads import presets
    g = presets.geometry(a.geom)
    gen = torch.Generator(device="cuda").manual_seed(0)
    if a.profile_case == "mlp":
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
    elif a.profile_case == "line":
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
    elif a.profile_case in ("das", "das_adjoint"):
        dt = torch.float16 if (a.dtype == "f16" and a.profile_case == "das") else torch.float32
        P = ops.DasPlan(g, rf_dtype=dt)
        if a.profile_case == "das":
            x = torch.randn(P.rf_shape(a.frames), device="cuda", generator=gen).to(dt)
            fn = lambda: P.forward(x)
        else:
            x = torch.randn(P.img_shape(a.frames), device="cuda", generator=gen)
            fn = lambda: P.adjoint(x)
    elif a.profile_case in ("synth", "synth_adjoint"):
        # the deconvolution geometry (1024 x 1024 grid, 11 x 128 records), one
        # frame: a Bernoulli(density) x normal map, or random channel data
        from tidas_workloads import generators, presets
        gd = presets.geometry("pw128_deconv")
        P = ops.DasPlan(gd)
        if a.profile_case == "synth":
            x = torch.from_numpy(generators.bernoulli_normal(
                (1, gd["nz"], gd["nx"]), a.density, (3,))).cuda()
            fn = lambda: P.synthesize_grid(x)
        else:
            x = torch.randn(P.rf_shape(1), device="cuda", generator=gen)
            fn = lambda: P.synthesize_adjoint(x)
    elif a.profile_case == "varying":
        # per-pixel kernels at the generator's layout: kz rows of 64 columns
        # (63 taps) per pixel (row form at kz = 1, band form above)
        nz, nx = g["nz"], g["nx"]
        shape = (nz, nx, 64) if a.kz == 1 else (nz, nx, a.kz, 64)
        k = torch.randn(shape, device="cuda", generator=gen)
        x = torch.randn((a.frames, nz, nx), device="cuda", generator=gen)
        if a.variant == 1:
            x = x.to(torch.bfloat16)
        fn = lambda: ops.tidas_forward_varying(k, x, variant=a.variant, taps=TAPS)
    else:
        nz, nx = g["nz"], g["nx"]
        band = a.profile_case.startswith("tidas2d")
        k = torch.randn((nz, a.kz, TAPS) if band else (nz, TAPS), device="cuda", generator=gen)
        x = torch.randn((a.frames, nz, nx), device="cuda", generator=gen)
        if a.variant == 1:
            x = x.to(torch.bfloat16)
        if band:
            f = ops.tidas_forward_2d if a.profile_case == "tidas2d" else ops.tidas_adjoint_2d
        else:
            f = ops.tidas_forward if a.profile_case == "tidas" else ops.tidas_adjoint
        fn = lambda: f(k, x, variant=a.variant)
    for _ in range(a.iters):
        fn()
    torch.cuda.synchronize()
    print("ok")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- workload bits
def active_updates(g):
    """Exact count of (pixel, element) pairs inside the F# aperture, times angles."""
    from tidas_workloads.presets import angles_rad
    xs = g["x0"] + (np.arange(g["nx"]) + 0.5) * g["dx"]
    zs = g["z0"] + (np.arange(g["nz"]) + 0.5) * g["dz"]
    xn = (np.arange(g["n_elem"]) - 0.5 * (g["n_elem"] - 1)) * g["pitch"]
    cnt = 0
    for z in zs:
        r = np.abs(xs[:, None] - xn[None, :]) * g["fnum"] / z
        cnt += int(np.count_nonzero(r <= 0.5))
    return cnt * len(angles_rad(g))


# --------------------------------------------------------- multi-rank logic
# Frames are sharded across ranks with no data-path collective: every rank
# synthesises its own batch (its own scatterer seeds) and beamforms it; only
# the step time is reduced (max over ranks), and the value counts the frames of
# all ranks.
def rank_seed_base(rank):
    """Scatterer seed base of a rank's frames: frame f of rank r draws from
    seed (1 + 1000 r, f), so no two ranks image the same frame."""
    return 1 + 1000 * rank


def max_over_ranks(torch, values, world, device):
    """Element-wise max of a list of floats over the ranks (one all-reduce)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_mpix_s(frames_per_rank, pixels_per_frame, world, ms):
    """Weak scaling: every rank's frames, divided by the slowest rank's time."""
    return frames_per_rank * pixels_per_frame * world / (ms * 1e-3) / 1e6


def make_rf(plan, torch, nf, seed_base=1):
    """Synthesise nf frames of channel data on the GPU (speckle + targets)."""
    from tidas_workloads import generators
    rf = torch.empty(plan.rf_shape(nf), dtype=plan.rf_dtype, device="cuda")
    chunk = 8
    for f0 in range(0, nf, chunk):
        fs = list(range(f0, min(nf, f0 + chunk)))
        ps, am = zip(*[generators.compound_speckle_frame(f, seed=seed_base) for f in fs])
        pos = torch.from_numpy(np.stack(ps)).cuda()
        amp = torch.from_numpy(np.stack(am)).cuda()
        plan.synthesize(pos, amp, out=rf[f0:f0 + len(fs)])
    torch.cuda.synchronize()
    return rf


def time_steps(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / steps  # ms per step


# ------------------------------------------------------------ CPU oracle
def oracle_das_sample(g, rf_host_frame, seconds=10.0):
    """Time the FP64 oracle on sampled pixels of one frame; returns
    (Mpixels/s, pixels timed, threads)."""
    import oracle
    O = oracle.Oracle(g)
    rf64 = rf_host_frame.astype(np.float64)
    rng = np.random.default_rng(0)
    npx = 512
    t0 = time.perf_counter()
    O.das_pixels(rf64, rng.choice(g["nx"] * g["nz"], npx, replace=False))
    dt = time.perf_counter() - t0
    npx = int(min(g["nx"] * g["nz"], max(512, npx * seconds / max(dt, 1e-3))))
    pix = rng.choice(g["nx"] * g["nz"], npx, replace=False)
    t0 = time.perf_counter()
    O.das_pixels(rf64, pix)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return npx / dt / 1e6, npx, threads


# ------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2507_15464_gb300 import capi, ops
    from tidas_workloads import presets, generators

    hbm_peak, bf16_peak, peak_src = peaks()
    g = presets.geometry(GEOM)
    P16 = ops.DasPlan(g, rf_dtype=torch.float16)
    rf = make_rf(P16, torch, BATCH, seed_base=rank_seed_base(rank))
    img = torch.empty(P16.img_shape(BATCH), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    npx = g["nx"] * g["nz"]

    def step():
        P16.forward(rf, out=img)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = time_steps(torch, step, args.steps, args.warmup, stream)
    ms = max_over_ranks(torch, [ms], world, "cuda")[0]
    clocks = clk.summary()
    value = whole_job_mpix_s(BATCH, npx, world, ms)

    # ---- roofline of the step's dominant kernel, das_tc_kernel.  A step is two
    # launches inside one das_forward call: das_tc_pack_kernel (repacks the
    # batch, ~7 % of the step) and das_tc_kernel.  They cannot be timed apart
    # through the C ABI, so "achieved" divides by the whole step's event time
    # (a lower bound for the kernel itself).
    updates = active_updates(g) * BATCH
    flops = updates * 10.0  # cubic: 4 tap MACs + 1 apodization MAC per update
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    fp32_peak = sms * 128 * 2 * 2.070e9 / 1e12  # TFLOP/s at the maximum SM clock
    alg_bytes = rf.numel() * 2 + img.numel() * 4
    # DRAM bytes of one das_tc_kernel launch (64 frames), from a one-pass ncu
    # capture of the current kernel (dram__bytes_read + dram__bytes_write);
    # None whenever the kernel changes after that capture
    traffic = 688.8e6 if BATCH == 64 else None
    # DRAM bytes of the step's two launches from the same capture: the repack
    # reads the plan's read window of the batch and writes its staged copy (the
    # rest of the staging layout stays zero), the DAS kernel reads that copy
    # (L2 serves the re-reads of neighbouring tiles) and writes the image
    step_traffic = {"das_tc_pack_kernel": 1175.9e6, "das_tc_kernel": 688.8e6} \
        if BATCH == 64 else None
    roof = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": fp32_peak,
            "unit": "TFLOP/s", "traffic": traffic, "kernel": "das_tc_kernel",
            "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flop x 2070 MHz" % sms,
            "work": "%.4g updates x 10 flop (cubic taps + apodization)" % updates,
            "g_updates_s": updates / (ms * 1e-3) / 1e9,
            "timed": "whole step (das_tc_pack_kernel + das_tc_kernel)",
            "step_traffic": step_traffic,
            "step_traffic_over_algorithmic": (sum(step_traffic.values()) / alg_bytes
                                              if step_traffic else None),
            "hw_counters": {"issue_active": 0.675, "tensor_pipe_active": 0.068,
                            "warps_active": 0.373, "l2_hit_rate": 0.903,
                            "warp_instructions_per_pair": 697,
                            "source": "ncu, profiles/das_tc_kernel_pw128_compound_64frames_f16.md"},
            "note": "instruction-issue- and latency-bound: 69 % of issue slots busy, "
                    "mostly the weight-building warps; tensor pipe 6.8 % busy.  The frac above is "
                    "the algorithmic flops (10 per update) over a derived CUDA-core FP32 "
                    "peak; the hardware counters are the bound"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    hbm = {"achieved_gbs": alg_bytes / (ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
           "peak_source": peak_src, "bytes_per_launch": alg_bytes}
    hbm["frac"] = hbm["achieved_gbs"] / hbm_peak

    # ---- accuracy of this batch vs the FP64 oracle (same channel data)
    extra = {}
    if rank == 0:
        import oracle
        O = oracle.Oracle(g)
        rng = np.random.default_rng(1)
        errs = []
        for f in (0, BATCH - 1):
            pix = rng.choice(npx, 400, replace=False)
            ref = O.das_pixels(rf[f].float().cpu().numpy().astype(np.float64), pix)
            got = img[f].flatten()[torch.from_numpy(pix).cuda()].double().cpu().numpy()
            errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        extra["nrmse_vs_oracle"] = float(max(errs))

    # ---- other DAS cases (not the headline)
    sub = {}
    for nf, dt in ((1, torch.float16), (8, torch.float16), (1, torch.float32), (8, torch.float32),
                   (64, torch.float32)):
        P = P16 if dt == torch.float16 else ops.DasPlan(g, rf_dtype=torch.float32)
        x = rf[:nf].float().contiguous() if dt == torch.float32 else rf[:nf].contiguous()
        y = torch.empty(P.img_shape(nf), device="cuda")
        m = time_steps(torch, lambda: P.forward(x, out=y), max(3, args.steps), 2, stream)
        sub["B%d_%s" % (nf, "f16" if dt == torch.float16 else "f32")] = {
            "ms": m, "mpix_s": nf * npx / (m * 1e-3) / 1e6}
    extra["das_cases"] = sub
    del P, x, y

    # ---- end to end through the public API with host buffers
    rf_host = torch.empty(rf.shape, dtype=rf.dtype, pin_memory=True)
    rf_host.copy_(rf)
    img_host = torch.empty(img.shape, dtype=torch.float32, pin_memory=True)
    rf_dev = torch.empty_like(rf)

    def e2e_step():
        rf_dev.copy_(rf_host, non_blocking=True)
        P16.forward(rf_dev, out=img)
        img_host.copy_(img, non_blocking=True)

    serial_ms = time_steps(torch, e2e_step, max(3, args.steps // 2), 2, stream)
    del rf_dev

    # serving form: uploads and read-backs of neighbouring batches overlap the
    # beamforming (ops.DasStreamer); every step still copies its 738 MB in and
    # its image out inside the timed region
    from paper_2507_15464_gb300.ops import DasStreamer
    streamer = DasStreamer(P16, BATCH)
    host_in = [rf_host, torch.empty_like(rf_host, pin_memory=True)]
    host_in[1].copy_(rf_host)
    host_out = [img_host, torch.empty_like(img_host, pin_memory=True)]
    for k in range(max(3, args.warmup)):
        streamer.submit(host_in[k & 1], host_out[k & 1])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # A stream's first upload and last read-back overlap nothing (about 3.5 ms
    # together); over at least 64 steps they weigh what they would in a
    # continuing stream at most 0.06 ms per step
    n_e2e = max(64, args.steps)
    # a plan freed by the garbage collector inside the loop would synchronise
    # the device (cudaFree) and drain the pipeline: collect first, then hold it
    import gc
    # The host -> device link is shared with the other GPUs of the machine, so
    # a window of steps can run slower than the next; three windows, median
    # reported, all listed
    windows = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gc.collect()
        gc.disable()
        e0.record(streamer.up)
        for k in range(n_e2e):
            streamer.submit(host_in[k & 1], host_out[k & 1])
        streamer.down.wait_stream(streamer.comp)
        e1.record(streamer.down)
        torch.cuda.synchronize()
        gc.enable()
        windows.append(e0.elapsed_time(e1) / n_e2e)
    e2e_ms = sorted(windows)[1]
    ok_e2e = torch.equal(host_out[(n_e2e - 1) & 1], img.cpu())
    e2e_ms, serial_ms = max_over_ranks(torch, [e2e_ms, serial_ms], world, "cuda")
    first, count = P16.read_window()
    e2e = {"value": whole_job_mpix_s(BATCH, npx, world, e2e_ms), "unit": "Mpixels/s",
           "h2d_bytes_per_step": streamer.h2d_bytes, "d2h_bytes_per_step": img.numel() * 4,
           "ms_per_step": e2e_ms, "steps": n_e2e,
           "windows_ms_per_step": windows,
           "form": "ops.DasStreamer: copies of neighbouring steps overlap the beamforming; "
                   "the stream's first upload and last read-back are inside each timed window; "
                   "median of three windows",
           "upload": "the plan's read window of every record, samples %d..%d of %d "
                     "(das_upload_window; the samples DAS weights)"
                     % (first, first + count - 1, g["n_samples"]),
           "image_matches_device_step": bool(ok_e2e),
           "serial": {"value": whole_job_mpix_s(BATCH, npx, world, serial_ms),
                      "ms_per_step": serial_ms, "h2d_bytes_per_step": rf.numel() * 2,
                      "form": "whole-record upload, beamforming and read-back on one stream"}}

    # ---- the 64-element single-angle case (DAS, 31-tap fit and apply)
    if rank == 0 and not args.no_config1:
        extra["config1"] = bench_config1(torch, ops, capi, generators, stream, args,
                                         cpu=not args.no_cpu_baseline)

    # ---- tiDAS variants on the 256-frame reflectivity batch
    if not args.no_tidas:
        extra["tidas"] = bench_tidas(torch, ops, capi, generators, g, P16, args, stream, hbm_peak,
                                     bf16_peak, ms / BATCH)

    # ---- learned kernel generator (training, inference, varying tiDAS)
    if not args.no_learned and rank == 0:
        refl16 = torch.from_numpy(np.stack([
            generators.bernoulli_normal((g["nz"], g["nx"]), 0.02, (2, f)) for f in range(16)
        ])).cuda()
        extra["learned"] = bench_learned(torch, capi, generators, refl16, args.epochs)
        del refl16
        extra["learned_band"] = bench_learned_band(torch, capi, generators, args.epochs)

    # ---- FISTA deconvolution, exact vs tiDAS operator
    if not args.no_fista and rank == 0:
        extra["fista"] = bench_fista(torch, capi, generators, args.fista_iters,
                                     cpu=not args.no_cpu_baseline)

    # ---- single-line experiment of Section 3 (600 x 600 sweep)
    if not args.no_line and rank == 0:
        extra["line_sweep"] = bench_line(torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n, thr = oracle_das_sample(g, rf[0].cpu().numpy())
        cpu = {"value": v, "unit": "Mpixels/s", "cores": thr, "kind": "oracle",
               "sample": "%d random pixels of frame 0 (FP64 oracle DAS, 11 angles x 128 "
                         "elements, cubic)" % n}

    line = {
        "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic",
        "config": {"workload": "compounded plane-wave DAS: 128 el, 11 angles -10..10 deg, "
                               "4096 samples, 512x1024 px, cubic, F#1.5, FP16 channel data, "
                               "FP32 accumulate",
                   "global_batch": BATCH * world, "frames_per_gpu": BATCH,
                   "parallelism": "frames sharded across ranks, no collective",
                   "l2": "inputs larger than L2 (738 MB per step)"},
        "roofline": roof, "hbm": hbm, "clocks": clocks, "e2e": e2e,
        "gpu_launches": 2 * args.steps, "cpu_baseline": cpu,
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def bench_tidas(torch, ops, capi, generators, g, P16, args, stream, hbm_peak, bf16_peak,
                das_ms_per_frame):
    from paper_2507_15464_gb300.ops import DasPlan
    P32 = DasPlan(g, rf_dtype=torch.float32)
    kern, _ = P32.fit_kernels(TAPS)
    nz, nx = g["nz"], g["nx"]
    refl = torch.empty((TIDAS_FRAMES, nz, nx), dtype=torch.float32, device="cuda")
    for f in range(TIDAS_FRAMES):
        refl[f] = torch.from_numpy(generators.bernoulli_normal((nz, nx), 0.02, (2, f))).cuda()
    refl_bf = refl.to(torch.bfloat16)
    out = torch.empty_like(refl)
    npx = TIDAS_FRAMES * nz * nx
    res = {"frames": TIDAS_FRAMES, "taps": TAPS}
    for variant, x, name in ((capi.VARIANT_DIRECT, refl, "direct_f32"),
                             (capi.VARIANT_GEMM_BF16, refl_bf, "gemm_bf16"),
                             (capi.VARIANT_GEMM_RESID, refl, "gemm_bf16_resid")):
        try:
            ops.tidas_forward(kern, x, variant=variant, out=out)
        except capi.TidasError as e:
            res[name] = {"unavailable": str(e)}
            continue
        m = time_steps(torch, lambda: ops.tidas_forward(kern, x, variant=variant, out=out),
                       max(3, args.steps), 2, stream)
        in_bytes = x.numel() * x.element_size()
        gbs = (in_bytes + out.numel() * 4) / (m * 1e-3) / 1e9
        r = {"ms": m, "mpix_s": npx / (m * 1e-3) / 1e6,
             "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak},
             "speedup_vs_das_per_frame": das_ms_per_frame / (m / TIDAS_FRAMES)}
        # accuracy vs the FP64 oracle on sampled rows (same input values)
        import oracle
        rows = np.array([0, 333, 1023])
        frames = np.array([0, TIDAS_FRAMES - 1])
        xin = x[frames][:, rows].double().cpu().numpy()
        ref = oracle.tidas_conv(kern[rows].cpu().numpy(), xin)
        got = out[frames][:, rows].double().cpu().numpy()
        r["nrmse_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        res[name] = r
    # tiDAS vs exact DAS on the same reflectivity (first frame): DAS of the
    # channel data that the reflectivity map produces
    rf = P32.synthesize_grid(refl[:1].contiguous())
    das_img = P32.forward(rf)
    ops.tidas_forward(kern, refl[:1].contiguous(), variant=capi.VARIANT_DIRECT, out=out[:1])
    d = das_img[0].double()
    res["nrmse_vs_exact_das"] = float((out[0].double() - d).norm() / d.norm())
    res["band_2d"] = bench_tidas2d(torch, ops, capi, P32, refl, refl_bf, out, d, args, stream,
                                   bf16_peak, das_ms_per_frame)
    res["frontier"] = bench_kz_frontier(torch, ops, capi, P32, refl, refl_bf, out, d, args,
                                        stream, das_ms_per_frame)
    if not args.no_cpu_baseline:
        # the FP64 oracle's Eq. (2.13) on 8 of the frames, all rows, host cores
        import oracle
        nfr = 8
        kh = kern.double().cpu().numpy()
        xs = refl[:nfr].double().cpu().numpy()
        t0 = time.perf_counter()
        oracle.tidas_conv(kh, xs)
        dt = time.perf_counter() - t0
        res["oracle_cpu"] = {"kind": "oracle", "frames": nfr, "seconds": dt,
                             "mpix_s": nfr * nz * nx / dt / 1e6,
                             "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
                             "sample": "%d of the %d frames, every row, FP64" % (nfr, TIDAS_FRAMES)}
    return res


def bench_kz_frontier(torch, ops, capi, P32, refl, refl_bf, out, das0, args, stream,
                      das_ms_per_frame, kzs=(1, 4, 8, 16, 32)):
    """Accuracy against speed of tiDAS over the band depth kz (63 taps) on the
    same 256-frame batch: for each kz the kernels are fitted from the exact
    PSFs, the tcgen05 band GEMM is timed, and its image is compared with the
    FP64 oracle (sampled rows) and with exact DAS of the same reflectivity
    (frame 0, FP32 direct form); the speed-up is per frame over the
    tensor-core DAS of the headline step.  kz = 1 is the row-wise model."""
    nf, nz, nx = refl.shape
    rows = [0, 333, nz - 1]
    frames = np.array([0, nf - 1])
    xin = refl_bf[frames].double().cpu().numpy()
    front = []
    for kz in kzs:
        kk = P32.fit_kernels_2d(kz, TAPS)
        ws = ops.band_workspace(nz, nx, nf, capi.VARIANT_GEMM_BF16)
        fn = lambda: ops.tidas_forward_2d(kk, refl_bf, variant=capi.VARIANT_GEMM_BF16,  # noqa: E731
                                          out=out, workspace=ws)
        m = time_steps(torch, fn, max(3, args.steps), 2, stream)
        ref = _band_rows_oracle(kk.cpu().numpy(), xin, rows)
        got = out[frames][:, rows].double().cpu().numpy()
        e_orc = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        ops.tidas_forward_2d(kk, refl[:1].contiguous(), variant=capi.VARIANT_DIRECT, out=out[:1])
        e_das = float((out[0].double() - das0).norm() / das0.norm())
        front.append({"kz": kz, "taps": TAPS, "gemm_ms": m,
                      "mpix_s": nf * nz * nx / (m * 1e-3) / 1e6,
                      "speedup_vs_das_per_frame": das_ms_per_frame / (m / nf),
                      "nrmse_vs_exact_das": e_das, "nrmse_vs_oracle": e_orc})
        del kk, ws
    return front


def _band_rows_oracle(kern, x, rows):
    """FP64 oracle of output rows `rows` of the 2D band forward map, each from
    the slab of input rows its band reaches."""
    import oracle
    nz, kz, _ = kern.shape
    cz = kz // 2
    out = []
    for i in rows:
        lo, hi = max(0, i - (kz - 1) + cz), min(nz - 1, i + cz)
        out.append(oracle.tidas_conv2d(kern[lo:hi + 1], x[:, lo:hi + 1])[:, i - lo])
    return np.stack(out, axis=1)


def bench_tidas2d(torch, ops, capi, P32, refl, refl_bf, out, das0, args, stream, bf16_peak,
                  das_ms_per_frame):
    """2D band kernels (KZ x TAPS per depth row) on the same 256-frame batch:
    kernel fit, direct FP32 and tcgen05 Toeplitz GEMM forward maps, accuracy
    against the oracle and against the exact DAS image."""
    nf, nz, nx = refl.shape
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    k2 = P32.fit_kernels_2d(KZ, TAPS)
    t1.record(stream)
    torch.cuda.synchronize()
    res = {"kz": KZ, "taps": TAPS, "fit_ms": t0.elapsed_time(t1)}
    cz = KZ // 2
    # valid band slices summed over the output rows (rows near the edges have fewer)
    nu = sum(min(KZ - 1, z + cz) - max(0, z + cz - (nz - 1)) + 1 for z in range(nz))
    useful = 2.0 * nf * nu * nx * TAPS
    # MMA work as issued: per (output row, 128 frames, 2 column tiles, slice)
    # every tile takes 3 chunks of 64 input columns
    ntiles = -(-nx // 128)
    mma = 2.0 * 128 * 128 * 192 * ntiles * (-(-nf // 128)) * nu
    kh = k2.cpu().numpy()
    for variant, x, name in ((capi.VARIANT_DIRECT, refl, "direct_f32"),
                             (capi.VARIANT_GEMM_BF16, refl_bf, "gemm_bf16")):
        ws = ops.band_workspace(nz, nx, nf, variant)
        fn = lambda: ops.tidas_forward_2d(k2, x, variant=variant, out=out,  # noqa: E731
                                          workspace=ws)
        try:
            fn()
        except capi.TidasError as e:
            res[name] = {"unavailable": str(e)}
            continue
        m = time_steps(torch, fn, max(3, args.steps), 2, stream)
        r = {"ms": m, "mpix_s": nf * nz * nx / (m * 1e-3) / 1e6,
             "useful_tflops": useful / (m * 1e-3) / 1e12,
             "speedup_vs_das_per_frame": das_ms_per_frame / (m / nf)}
        if variant == capi.VARIANT_GEMM_BF16:
            a = mma / (m * 1e-3) / 1e12
            u = useful / (m * 1e-3) / 1e12
            # the call is the operand repack plus the GEMM; both are in `ms`.
            # frac counts the method's own work (2 kz taps flop per output
            # pixel); the executed MMA work also multiplies the zero band
            # padding (K = 192 columns per 128-column tile for 63 taps)
            r["tensor"] = {"useful_tflops": u, "peak_tflops": bf16_peak, "frac": u / bf16_peak,
                           "useful_flops_per_call": useful,
                           "mma_tflops": a, "mma_frac": a / bf16_peak,
                           "mma_flops_per_call": mma, "timed": "repack + GEMM"}
        rows = [0, 333, nz - 1]
        frames = np.array([0, nf - 1])
        xin = x[frames].double().cpu().numpy()
        ref = _band_rows_oracle(kh, xin, rows)
        got = out[frames][:, rows].double().cpu().numpy()
        r["nrmse_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        res[name] = r
    ops.tidas_forward_2d(k2, refl[:1].contiguous(), variant=capi.VARIANT_DIRECT, out=out[:1])
    res["nrmse_vs_exact_das"] = float((out[0].double() - das0).norm() / das0.norm())
    return res


def bench_line(torch, stream):
    """The experiment of Section 3.3 / Table 3.2 row 2: a unit scatterer on
    each of 600 line points (2 to 42 mm), reconstructed with every one of the
    600 fixed delay curves: theta (Eq. (2.12)) and the local / global errors
    for all 360 000 pairs, plus the channel data and DAS lines they need."""
    import time

    from paper_2507_15464_gb300.ops import LineExperiment
    from tidas_workloads.line_scenarios import paper_line
    res = {}
    for f0, zf in ((5e6, 25e-3), (7e6, 25e-3), (5e6, 15e-3), (5e6, 35e-3)):
        p = paper_line(f0=f0, z_focus=zf)
        E = LineExperiment(p)
        eps = E.window()
        rf = E.synthesize()
        g = E.das_lines(rf)
        E.sweep(rf, g, eps)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        E.synthesize(out=rf)
        ev[1].record(stream)
        E.das_lines(rf, out=g)
        ev[2].record(stream)
        th, el, eg = E.sweep(rf, g, eps)
        ev[3].record(stream)
        torch.cuda.synchronize()
        ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]
        th_h, el_h, eg_h = th.cpu().numpy(), el.cpu().numpy(), eg.cpu().numpy()
        key = "f0_%gMHz_focus_%gmm" % (f0 / 1e6, zf * 1e3)
        r = {"synth_ms": ms[0], "das_lines_ms": ms[1], "sweep_ms": ms[2],
             "total_ms": sum(ms), "pairs": int(th_h.size),
             "pairs_per_s": th_h.size / (ms[2] * 1e-3),
             "frac_local_below_5pct": float((el_h < 0.05).mean()),
             "frac_global_below_5pct": float((eg_h < 0.05).mean()),
             "theta_p5_p95": [float(np.percentile(th_h, 5)), float(np.percentile(th_h, 95))]}
        r["fig_3_1"] = line_peaks_and_fwhm(torch, E, rf, g, eps, zf)
        # curves that keep the local error below 5 % for the most scatterers
        good = (el_h < 0.05).sum(axis=1)
        r["best_curve_depth_mm"] = float(E.depth(int(np.argmax(good))) * 1e3)
        r["best_curve_scatterers_below_5pct"] = int(good.max())
        if f0 == 5e6 and zf == 25e-3:
            # sampled pairs against the FP64 oracle on the same channel data,
            # and the oracle's own rate on a bounded sample (about 10 s)
            import oracle.line as oline
            O = oline.LineOracle(p)
            rf_h, g_h = rf.cpu().numpy(), g.cpu().numpy()
            errs = []
            t0 = time.perf_counter()
            n_or = 0
            for rr in (100, 344, 500):
                S, gl = rf_h[rr].astype(np.float64), g_h[rr].astype(np.float64)
                for s in (rr - 20, rr, rr + 20, 344):
                    t_, l_, e_ = O.sweep_pair(S, gl, rr, s, eps)
                    errs.append(abs(l_ - el_h[s, rr]))
                    errs.append(abs(e_ - eg_h[s, rr]))
                    errs.append(abs(t_ - th_h[s, rr]) / max(abs(t_), 1e-12))
                    n_or += 1
            dt = time.perf_counter() - t0
            r["max_dev_vs_oracle"] = float(max(errs))
            r["oracle_pairs_per_s"] = n_or / dt
            r["paper_table_3_2"] = {"das_min": 28.35, "tidas_min": 21.11,
                                    "note": "Python on unstated hardware; context only"}
            r["line_reconstruction"] = bench_line_reconstruction(torch, stream, E, rf, th, eps)
        res[key] = r
        del rf, g
    return res


def _fwhm_rows(env, spacing):
    """Full width at half maximum of each row's main peak, linear
    interpolation between line points (reporting only)."""
    out = np.empty(env.shape[0])
    for k, e in enumerate(env):
        i = int(np.argmax(e))
        half = 0.5 * e[i]
        lo = i
        while lo > 0 and e[lo - 1] > half:
            lo -= 1
        hi = i
        while hi < e.size - 1 and e[hi + 1] > half:
            hi += 1
        left = lo - (e[lo] - half) / (e[lo] - e[lo - 1]) if lo > 0 else float(lo)
        right = hi + (e[hi] - half) / (e[hi] - e[hi + 1]) if hi < e.size - 1 else float(hi)
        out[k] = (right - left) * spacing
    return out


def line_peaks_and_fwhm(torch, E, rf, das_lines, eps, z_focus):
    """Fig. 3.1 / 3.2: for every scatterer, the peak and the FWHM of the DAS
    line and of its tiDAS reconstruction under the focal point's delay curve
    (envelopes on the GPU), summarised over depth."""
    from paper_2507_15464_gb300.ops import envelope
    D = E.D
    z = np.array([E.depth(i) for i in range(D)])
    s_f = int(np.argmin(np.abs(z - z_focus)))
    ti = E.fixed_lines(rf, s_f, eps)
    env_d = envelope(das_lines).cpu().numpy().astype(np.float64)
    env_t = envelope(ti).cpu().numpy().astype(np.float64)
    dz = (z[-1] - z[0]) / (D - 1)
    pk_d, pk_t = env_d.max(axis=1), env_t.max(axis=1)
    fw_d, fw_t = _fwhm_rows(env_d, dz), _fwhm_rows(env_t, dz)
    near = np.abs(z - z[s_f]) <= 2e-3
    ratio = pk_t / pk_d
    dfw = np.abs(fw_t - fw_d)
    c = E.p["c"]
    return {"focal_curve_depth_mm": float(z[s_f] * 1e3),
            "peak_das_over_focal": [float(np.min(pk_d / pk_d[s_f])), float(np.max(pk_d / pk_d[s_f]))],
            "peak_ratio_tidas_over_das": {"at_focus": float(ratio[s_f]),
                                          "median_within_2mm": float(np.median(ratio[near])),
                                          "median_all": float(np.median(ratio))},
            "fwhm_abs_diff_us": {"at_focus": float(dfw[s_f] * 2 / c * 1e6),
                                 "median_within_2mm": float(np.median(dfw[near]) * 2 / c * 1e6),
                                 "median_all": float(np.median(dfw) * 2 / c * 1e6)},
            "fwhm_das_at_focus_us": float(fw_d[s_f] * 2 / c * 1e6),
            "note": "FWHM in two-way time of the line's envelope; peaks of the envelopes"}


def bench_line_reconstruction(torch, stream, E, rf, theta, eps):
    """Section 3.4 / Table 3.1: lines of 5 and 100 scatterers reconstructed by
    DAS and by the line model of Eq. (2.13) with the delay curves of the 25
    and 35 mm points (theta: that curve's row of the sweep); envelopes on the
    GPU, mean side-lobe levels outside the main lobes (-20 dB pulse width)."""
    from paper_2507_15464_gb300.ops import envelope
    from tidas_workloads.line_scenarios import scenarios
    D = E.D
    z = np.array([E.depth(i) for i in range(D)])
    # main-lobe half-width in depth: the pulse envelope 20 dB down, two-way
    alpha = np.log(2.0) / eps ** 2
    half = E.p["c"] * np.sqrt(np.log(10.0) / alpha) / 2.0

    def sl_db(env, pts):
        side = np.ones(D, bool)
        for j in pts:
            side &= np.abs(z - z[j]) > half
        return float(20.0 * np.log10(env[side].mean() / env.max()))

    def timed(fn, reps=20):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    for name, amps in scenarios(D).items():
        pts = np.nonzero(amps)[0]
        S = E.combine(rf, torch.from_numpy(amps.astype(np.float32)).cuda())
        S1 = S.reshape(1, *S.shape)
        das = E.das_lines(S1)[0]
        env_das = envelope(das).cpu().numpy()
        out = {"scatterers": int(pts.size), "das_line_ms": timed(lambda: E.das_lines(S1))}
        for zs in (25e-3, 35e-3):
            s = int(np.argmin(np.abs(z - zs)))
            th = theta[s].contiguous()
            ti = E.model(S, s, th, eps)
            env_ti = envelope(ti).cpu().numpy()
            sd, st_ = sl_db(env_das, pts), sl_db(env_ti, pts)
            out["curve_%gmm" % (zs * 1e3)] = {
                "tidas_line_ms": timed(lambda: E.model(S, s, th, eps)),
                "mean_sl_das_db": sd, "mean_sl_tidas_db": st_,
                "relative_sl_error": abs(st_ - sd) / abs(sd),
                "peak_ratio_tidas_over_das": float(env_ti[pts].mean() / env_das[pts].mean())}
        res[name] = out
    res["paper_table_3_1"] = "parity unpinned: the paper's SL definition and line geometry are not given"
    return res


def bench_fista(torch, capi, generators, iters, cpu=True):
    """Deconvolution workload: 1024 x 1024 reflectivity grid, 128-element array,
    11 angles; b = exact DAS of the grid's channel data + 30 dB Gaussian noise;
    `iters` FISTA iterations with the L1 prior, timed end to end, with the
    exact operator and with tiDAS (63-tap kernels fitted from the geometry)."""
    from paper_2507_15464_gb300 import deconv
    from paper_2507_15464_gb300.ops import DasPlan
    from tidas_workloads import presets
    g = presets.geometry("pw128_deconv")
    P = DasPlan(g)
    shape = (1, g["nz"], g["nx"])
    x_true = torch.from_numpy(generators.bernoulli_normal(shape, 0.02, (3,))).cuda()
    exact = deconv.ExactOperator(P)
    clean = exact.forward(x_true, None)
    rms = (float(deconv.dot(clean, clean)) / clean.numel()) ** 0.5
    noise = torch.from_numpy(generators.standard_normal(shape, (3, 1))).cuda()
    b = torch.empty_like(clean)
    deconv.axpby(1.0, clean, rms * 10 ** (-30 / 20), noise, b)
    v0 = torch.from_numpy(generators.standard_normal(shape, (3, 2))).cuda()
    kern, _ = P.fit_kernels(TAPS)
    kern2 = P.fit_kernels_2d(KZ, TAPS)
    res = {"grid": "1024x1024", "iters": iters}
    for name, op in (("exact", exact),
                     ("tidas_direct", deconv.TidasOperator(kern, capi.VARIANT_DIRECT)),
                     ("tidas_gemm_resid", deconv.TidasOperator(kern, capi.VARIANT_GEMM_RESID)),
                     ("tidas_band_direct", deconv.TidasBandOperator(kern2))):
        L, _ = deconv.power_iteration(op, v0, 30)
        htb = op.adjoint(b, torch.empty_like(b))
        lam = 0.01 * float(np.abs(htb.cpu().numpy()).max())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = deconv.fista(op, b, lam, 1.01 * L, iters)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        err = float(deconv.dot(x, x))
        tmp = torch.empty_like(x)
        deconv.axpby(1.0, x, -1.0, x_true, tmp)
        rel = (float(deconv.dot(tmp, tmp)) / float(deconv.dot(x_true, x_true))) ** 0.5
        # convergence: data residual and objective against the start x = 0
        r = op.forward(x, None)
        deconv.axpby(1.0, r, -1.0, b, r)
        resid = (float(deconv.dot(r, r)) / float(deconv.dot(b, b))) ** 0.5
        f0 = 0.5 * float(deconv.dot(b, b))
        f = deconv.objective(op, x, b, lam)
        # the solution against the true model: ||H_exact x - b|| / ||b||
        re_ = exact.forward(x, None)
        deconv.axpby(1.0, re_, -1.0, b, re_)
        resid_exact = (float(deconv.dot(re_, re_)) / float(deconv.dot(b, b))) ** 0.5
        res[name] = {"seconds": dt, "ms_per_iter": dt / iters * 1e3, "L": L, "lambda": lam,
                     "data_residual": resid, "data_residual_exact_operator": resid_exact,
                     "objective_ratio": f / f0,
                     "rel_err_vs_truth": rel, "x_norm2": err,
                     "note": "the band-limited PSF makes the sparse map unrecoverable in "
                             "200 iterations (rel_err_vs_truth near 1 for any operator); "
                             "data_residual and objective_ratio show the solve"}
    res["speedup_tidas_gemm_resid_vs_exact"] = res["exact"]["seconds"] / res["tidas_gemm_resid"]["seconds"]
    if cpu:
        # the FP64 oracle's FISTA with the row-kernel tiDAS operator (Eq. (2.13)
        # and its transpose) on the same data, 3 iterations on the host cores; the
        # exact operator's FP64 synthesis of a 1024 x 1024 grid takes minutes
        import oracle
        from oracle import fista as ofista
        kh = kern.double().cpu().numpy()
        bh = b[0].double().cpu().numpy()
        lam = res["tidas_direct"]["lambda"]
        L = 1.01 * res["tidas_direct"]["L"]
        n_it = 3
        t0 = time.perf_counter()
        ofista.fista(lambda v: oracle.tidas_conv(kh, v), lambda v: oracle.tidas_conv_adjoint(kh, v),
                     bh, lam, L, n_it)
        dt = time.perf_counter() - t0
        res["oracle_cpu_tidas"] = {"kind": "oracle", "iters": n_it, "ms_per_iter": dt / n_it * 1e3,
                                   "cores": int(os.environ.get("OMP_NUM_THREADS",
                                                               os.cpu_count() or 1))}
        res["oracle_cpu_exact"] = oracle_exact_iteration_estimate(g, x_true[0].cpu().numpy())
    return res


def oracle_exact_iteration_estimate(g, x_true, frac=64):
    """One FISTA iteration with the exact operator costs a synthesis of the
    whole grid, a DAS of the whole grid and their transposes (the same loops
    as the forward maps).  The FP64 oracle's cost is linear in the pixels it
    synthesises and beamforms, so it is timed on 1/frac of them (pixels with
    a stride of frac through the grid, every one synthesised with its own
    reflectivity, and the DAS of as many pixels) and scaled to the grid:
    iteration ~ 2 (synthesis + DAS)."""
    import oracle
    O = oracle.Oracle(g)
    npx = g["nx"] * g["nz"]
    sel = np.arange(0, npx, frac)
    pos = O.grid_positions()[sel]
    amp = np.zeros((sel.size, 2))
    amp[:, 0] = x_true.ravel()[sel]
    amp[amp[:, 0] == 0, 0] = 1.0  # every sampled pixel costs a full synthesis
    t0 = time.perf_counter()
    rf = O.synthesize(pos, amp)
    t1 = time.perf_counter()
    O.das_pixels(rf, sel)
    t2 = time.perf_counter()
    synth_s, das_s = (t1 - t0) * frac, (t2 - t1) * frac
    return {"kind": "oracle", "ms_per_iter": 2.0 * (synth_s + das_s) * 1e3,
            "synthesis_s": synth_s, "das_s": das_s,
            "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "sample": "synthesis and DAS of 1/%d of the 1024 x 1024 pixels, scaled to the "
                      "grid; an iteration counts each map and its transpose" % frac}


def bench_config1(torch, ops, capi, generators, stream, args, cpu=True):
    """The 64-element case: one 0 degree plane wave, 2048 x 64 FP32 channel
    data from 200 N(0,1) scatterers in a 19 x 30 mm box (seed 0), a 128 x 256
    image with linear interpolation and F# 1.5 Hann apodization; 31-tap row
    kernels fitted from exact single-scatterer PSFs and applied to the same
    scatterers placed on their nearest pixels."""
    import oracle
    from tidas_workloads import presets
    g = presets.geometry("pw64_single")
    P = ops.DasPlan(g)
    pos, amp = generators.single_frame_speckle(0, n=200)
    posd = torch.from_numpy(np.ascontiguousarray(pos[None])).cuda()
    ampd = torch.from_numpy(np.ascontiguousarray(amp[None]).astype(np.float32)).cuda()
    rf = P.synthesize(posd, ampd)
    img = torch.empty(P.img_shape(1), device="cuda")
    npx = g["nx"] * g["nz"]
    res = {"workload": "64 el, 0 deg, 2048 samples, 128 x 256 px, linear, F# 1.5, FP32",
           "scatterers": 200}
    ms_syn = time_steps(torch, lambda: P.synthesize(posd, ampd, out=rf), max(3, args.steps), 2,
                        stream)
    ms = time_steps(torch, lambda: P.forward(rf, out=img), max(3, args.steps), 2, stream)
    O = oracle.Oracle(g)
    rf_h = rf[0].double().cpu().numpy()
    t0 = time.perf_counter()
    ref = O.das(rf_h)
    t_orc = time.perf_counter() - t0
    got = img[0].double().cpu().numpy()
    res["das"] = {"ms": ms, "mpix_s": npx / (ms * 1e-3) / 1e6, "synthesis_ms": ms_syn,
                  "nrmse_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
    # tiDAS: 31-tap kernels, the scatterers on their nearest pixels
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    k31, _ = P.fit_kernels(31)
    t1e.record(stream)
    torch.cuda.synchronize()
    refl = np.zeros((1, g["nz"], g["nx"]), np.float32)
    ix = np.clip(np.floor((pos[:, 0] - g["x0"]) / g["dx"]).astype(int), 0, g["nx"] - 1)
    iz = np.clip(np.floor((pos[:, 1] - g["z0"]) / g["dz"]).astype(int), 0, g["nz"] - 1)
    np.add.at(refl[0], (iz, ix), amp[:, 0].astype(np.float32))
    refl_d = torch.from_numpy(refl).cuda()
    exact = P.forward(P.synthesize_grid(refl_d))
    kh = k31.double().cpu().numpy()
    tref = oracle.tidas_conv(kh, refl.astype(np.float64))
    res["tidas"] = {"taps": 31, "fit_ms": t0e.elapsed_time(t1e)}
    for variant, name in ((capi.VARIANT_DIRECT, "direct_f32"), (capi.VARIANT_GEMM_BF16, "gemm_bf16"),
                          (capi.VARIANT_GEMM_RESID, "gemm_resid")):
        x = refl_d.to(torch.bfloat16) if variant == capi.VARIANT_GEMM_BF16 else refl_d
        out = torch.empty_like(refl_d)
        m = time_steps(torch, lambda: ops.tidas_forward(k31, x, variant=variant, out=out),
                       max(3, args.steps), 2, stream)
        y = out[0].double()
        res["tidas"][name] = {
            "ms": m, "mpix_s": npx / (m * 1e-3) / 1e6,
            "nrmse_vs_oracle": float(np.linalg.norm(y.cpu().numpy() - tref) / np.linalg.norm(tref)),
            "nrmse_vs_exact_das": float((y - exact[0].double()).norm() / exact[0].double().norm()),
            "speedup_vs_das": ms / m}
    if cpu:
        t0 = time.perf_counter()
        kf, _ = O.fit_kernels(31)
        t_fit = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.tidas_conv(kf, refl.astype(np.float64))
        t_conv = time.perf_counter() - t0
        res["oracle_cpu"] = {"kind": "oracle",
                             "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
                             "das_mpix_s": npx / t_orc / 1e6, "das_ms": t_orc * 1e3,
                             "tidas_fit_ms": t_fit * 1e3, "tidas_conv_ms": t_conv * 1e3,
                             "tidas_mpix_s": npx / t_conv / 1e6}
    P.close()
    return res


def bench_learned(torch, capi, generators, refl, epochs):
    """Learned kernel generator: train on 20k exact PSFs (x, z, F# 1-3,
    angle +-15 deg; seeds 4-5), then generate per-pixel kernels for the
    512 x 1024 grid under an unseen geometry (F# 1.7, 7.5 deg), with exact
    kernels as fallback above 2 % NRMSE, and drive spatially varying tiDAS."""
    import math
    from paper_2507_15464_gb300 import generator as gen
    from paper_2507_15464_gb300.ops import DasPlan, _ptr, _stream, tidas_forward
    from tidas_workloads import presets
    geom = presets.geometry(GEOM)
    P = DasPlan(geom)
    res = {"train_samples": 20000, "epochs": epochs, "batch": 256}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s, tgt = gen.training_set(P, n=20000, seed=4)
    torch.cuda.synchronize()
    res["training_set_seconds"] = time.perf_counter() - t0
    net = gen.KernelMLP(batch=256)
    x16 = torch.empty((20000, 64), dtype=torch.bfloat16, device="cuda")
    net.encode(s, x16)
    rng = np.random.default_rng([5])
    perms = torch.from_numpy(np.stack([rng.permutation(20000) for _ in range(epochs)])
                             .astype(np.int32)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.fit(x16, tgt, epochs, perms, lr0=1e-3, log_every=max(1, epochs // 4))
    torch.cuda.synchronize()
    res["training_seconds"] = time.perf_counter() - t0
    res["loss_curve"] = losses
    fnum, ang = 1.7, 7.5 * math.pi / 180.0
    smp = gen.grid_samples(geom, fnum, ang)
    npix = smp.shape[0]
    stream = torch.cuda.current_stream()
    learned = net.infer(P, smp)
    exact = gen.exact_kernels(P, smp)
    ms_inf = time_steps(torch, lambda: net.infer(P, smp), 3, 1, stream)
    ms_exact = time_steps(torch, lambda: gen.exact_kernels(P, smp), 2, 1, stream)
    flops = 2.0 * npix * (4 * 256 + 2 * 256 * 256 + 256 * 63)
    res["inference"] = {"kernels": npix, "ms": ms_inf, "kernels_per_s": npix / (ms_inf * 1e-3),
                        "tensor": {"achieved_tflops": flops / (ms_inf * 1e-3) / 1e12,
                                   "peak_tflops": peaks()[1],
                                   "frac": flops / (ms_inf * 1e-3) / 1e12 / peaks()[1]},
                        "exact_psf_ms": ms_exact, "speedup_vs_exact_fit": ms_exact / ms_inf}
    mixed = torch.empty_like(learned)
    err = torch.empty((npix,), device="cuda")
    capi.call("tidas_kernel_fallback", _ptr(learned), 64, _ptr(exact), 64, npix, 63, 0.02,
              _ptr(mixed), 64, _ptr(err), _stream())
    e = err.cpu().numpy()
    ex = exact.cpu().numpy()[:, :63].reshape(geom["nz"], geom["nx"], 63)
    si = np.broadcast_to(ex[:, geom["nx"] // 2:geom["nx"] // 2 + 1, :], ex.shape)
    e_si = (np.linalg.norm(si - ex, axis=2) / np.linalg.norm(ex, axis=2)).ravel()
    res["kernel_nrmse"] = {"learned_mean": float(e.mean()), "learned_median": float(np.median(e)),
                           "fallback_fraction": float((e > 0.02).mean()),
                           "shift_invariant_mean": float(e_si.mean())}
    # images: spatially varying tiDAS with the mixed kernels vs exact single-angle DAS
    g1 = dict(geom, angles_deg=[7.5], fnum=fnum)
    P1 = DasPlan(g1)
    nf = refl.shape[0]
    out = torch.empty_like(refl)
    capi.call("tidas_forward_varying", _ptr(mixed), 64, 63, geom["nz"], geom["nx"], _ptr(refl),
              _ptr(out), nf, _stream())
    ms_var = time_steps(torch, lambda: capi.call("tidas_forward_varying", _ptr(mixed), 64, 63,
                                                  geom["nz"], geom["nx"], _ptr(refl), _ptr(out),
                                                  nf, _stream()), 3, 1, stream)
    res["varying_tidas"] = {"frames": nf, "ms": ms_var,
                            "mpix_s": nf * npix / (ms_var * 1e-3) / 1e6}
    das = P1.forward(P1.synthesize_grid(refl[:1].contiguous()))
    k_row, _ = P1.fit_kernels(63)
    y_si = tidas_forward(k_row, refl[:1].contiguous())
    d = das[0].double()
    res["image_nrmse_vs_exact_das"] = {
        "learned_varying": float((out[0].double() - d).norm() / d.norm()),
        "shift_invariant_rows": float((y_si[0].double() - d).norm() / d.norm())}
    return res


def bench_learned_band(torch, capi, generators, epochs, kz=8, frames=256):
    """Learned band kernels: the generator trained on 20k exact kz x 63 band
    PSFs (seeds 4-5) emits a kernel per pixel of the 512 x 1024 grid under the
    unseen geometry (F# 1.7, 7.5 deg), exact kernels replace those more than
    2 % off, and the tcgen05 varying band GEMM applies them.  Images are
    compared with exact single-angle DAS of the same reflectivity, beside the
    fixed band kernels of plain tiDAS (fitted at the centre column), the exact
    per-pixel band kernels (the best kz x 63 kernels can do) and the row
    kernels."""
    import math
    from paper_2507_15464_gb300 import generator as gen, ops
    from paper_2507_15464_gb300.ops import DasPlan, _ptr, _stream
    from tidas_workloads import presets
    geom = presets.geometry(GEOM)
    P = DasPlan(geom)
    nz, nx = geom["nz"], geom["nx"]
    res = {"kz": kz, "taps": TAPS, "train_samples": 20000, "epochs": epochs}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s, tgt = gen.training_set(P, n=20000, seed=4, kz=kz)
    torch.cuda.synchronize()
    res["training_set_seconds"] = time.perf_counter() - t0
    net = gen.KernelMLP(batch=256, kz=kz)
    x16 = torch.empty((20000, 64), dtype=torch.bfloat16, device="cuda")
    net.encode(s, x16)
    rng = np.random.default_rng([5])
    perms = torch.from_numpy(np.stack([rng.permutation(20000) for _ in range(epochs)])
                             .astype(np.int32)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.fit(x16, tgt, epochs, perms, lr0=1e-3, log_every=max(1, epochs // 4))
    torch.cuda.synchronize()
    res["training_seconds"] = time.perf_counter() - t0
    res["loss_curve"] = losses
    del s, tgt, x16, perms
    fnum, ang = 1.7, 7.5 * math.pi / 180.0
    smp = gen.grid_samples(geom, fnum, ang)
    npix = smp.shape[0]
    stream = torch.cuda.current_stream()
    learned = net.infer(P, smp)
    ms_inf = time_steps(torch, lambda: net.infer(P, smp), 3, 1, stream)
    flops = 2.0 * npix * (4 * 256 + 2 * 256 * 256 + 256 * net.out)
    res["inference"] = {"kernels": npix, "ms": ms_inf,
                        "tflops": flops / (ms_inf * 1e-3) / 1e12}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    exact = gen.exact_kernels(P, smp, kz=kz)
    torch.cuda.synchronize()
    res["exact_psf_seconds"] = time.perf_counter() - t0
    mixed = torch.empty_like(learned)
    err = torch.empty((npix,), device="cuda")
    capi.call("tidas_kernel_fallback", _ptr(learned), net.out, _ptr(exact), net.out, npix,
              net.out, 0.02, _ptr(mixed), net.out, _ptr(err), _stream())
    e = err.cpu().numpy()
    res["kernel_nrmse"] = {"learned_mean": float(e.mean()), "learned_median": float(np.median(e)),
                           "fallback_fraction": float((e > 0.02).mean())}
    del learned
    # images of frame 0 against exact single-angle DAS
    g1 = dict(geom, angles_deg=[7.5], fnum=fnum)
    P1 = DasPlan(g1)
    refl = torch.from_numpy(np.stack([
        generators.bernoulli_normal((nz, nx), 0.02, (2, f)) for f in range(frames)])).cuda()
    refl_bf = refl.to(torch.bfloat16)
    das = P1.forward(P1.synthesize_grid(refl[:1].contiguous()))[0].double()
    km = mixed.view(nz, nx, kz, gen.SLOT)
    ke = exact.view(nz, nx, kz, gen.SLOT)
    out = torch.empty((frames, nz, nx), device="cuda")
    fn = lambda: ops.tidas_forward_varying(km, refl_bf, variant=capi.VARIANT_GEMM_BF16,  # noqa
                                           out=out, taps=TAPS)
    fn()
    ms32 = time_steps(torch, fn, 5, 2, stream)
    y32 = out.clone()
    # the same kernels stored in BF16 once (they depend on the geometry, not on
    # the frames): half the dominant stream, bit-identical images
    km16 = km.to(torch.bfloat16)
    fn = lambda: ops.tidas_forward_varying(km16, refl_bf, variant=capi.VARIANT_GEMM_BF16,  # noqa
                                           out=out, taps=TAPS)
    fn()
    ms = time_steps(torch, fn, 5, 2, stream)
    same16 = bool(torch.equal(out, y32))
    del km16, y32
    cz = kz // 2
    nu = sum(min(kz - 1, z + cz) - max(0, z + cz - (nz - 1)) + 1 for z in range(nz))
    useful = 2.0 * frames * nu * nx * TAPS
    _, bf16_peak, _ = peaks()
    res["varying_gemm"] = {"frames": frames, "ms": ms, "mpix_s": frames * npix / (ms * 1e-3) / 1e6,
                           "tensor": {"useful_tflops": useful / (ms * 1e-3) / 1e12,
                                      "peak_tflops": bf16_peak,
                                      "frac": useful / (ms * 1e-3) / 1e12 / bf16_peak},
                           "fp32_kernels_ms": ms32, "bf16_kernels_image_identical": same16,
                           "note": "per-pixel B tiles built per (row, slice, chunk); kernels "
                                   "read in BF16 (%.2f GB per call; FP32 %.2f GB: fp32_kernels_ms)"
                                   % (nz * nx * kz * gen.SLOT * 2 / 1e9,
                                      nz * nx * kz * gen.SLOT * 4 / 1e9)}

    def nr(y):
        return float((y.double() - das).norm() / das.norm())

    y_l = out[0].clone()
    y_e = ops.tidas_forward_varying(ke, refl[:1].contiguous(), taps=TAPS)[0]
    k2 = P1.fit_kernels_2d(kz, TAPS)
    y_b = ops.tidas_forward_2d(k2, refl[:1].contiguous())[0]
    k1, _ = P1.fit_kernels(TAPS)
    y_r = ops.tidas_forward(k1, refl[:1].contiguous())[0]
    res["image_nrmse_vs_exact_das"] = {"learned_band_varying": nr(y_l),
                                       "exact_band_varying": nr(y_e),
                                       "fixed_band": nr(y_b), "fixed_rows": nr(y_r)}
    del mixed, exact, km, ke, out
    res["compound"] = learned_band_compound(torch, capi, gen, ops, net, P, geom, refl, kz)
    return res


def learned_band_compound(torch, capi, gen, ops, net, P, geom, refl, kz, z_row=400, rows=128):
    """The compounded workload itself (11 plane waves, F# 1.5) on a slab of
    rows: DAS is linear in the transmit events, so a pixel's compound kernel
    is the sum of its single-angle kernels.  Learned kernels (as inferred,
    and with exact ones where more than 2 % off), exact ones, the fixed band
    kernels of plain tiDAS and row kernels, against exact compound DAS."""
    import math
    from paper_2507_15464_gb300.ops import DasPlan, _ptr, _stream
    sub = dict(geom, nz=rows, z0=geom["z0"] + z_row * geom["dz"])
    Ps = DasPlan(sub)
    npix = rows * sub["nx"]
    kl = torch.zeros((npix, net.out), device="cuda")
    km = torch.zeros_like(kl)
    kx = torch.zeros_like(kl)
    ma = torch.empty_like(kl)
    stream = torch.cuda.current_stream()
    t_inf = 0.0
    for deg in geom["angles_deg"]:
        smp = gen.grid_samples(sub, geom["fnum"], math.radians(deg))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        la = net.infer(P, smp)
        e1.record(stream)
        ea = gen.exact_kernels(P, smp, kz=kz)
        capi.call("tidas_kernel_fallback", _ptr(la), net.out, _ptr(ea), net.out, npix, net.out,
                  0.02, _ptr(ma), net.out, None, _stream())
        torch.cuda.synchronize()
        t_inf += e0.elapsed_time(e1)
        kl += la
        km += ma
        kx += ea
    r = refl[:1, z_row:z_row + rows].contiguous()
    das = Ps.forward(Ps.synthesize_grid(r))[0].double()

    def nr(y):
        return float((y[0].double() - das).norm() / das.norm())

    shape = (rows, sub["nx"], kz, gen.SLOT)
    rb = r.to(torch.bfloat16)
    return {"slab": "rows %d..%d (z %.1f-%.1f mm), 512 columns, 11 angles, F# 1.5"
                    % (z_row, z_row + rows - 1, 1e3 * sub["z0"], 1e3 * (sub["z0"] + rows * sub["dz"])),
            "inference_ms_per_angle_per_slab": t_inf / len(geom["angles_deg"]),
            "image_nrmse_vs_exact_das": {
                "learned_band_varying": nr(ops.tidas_forward_varying(
                    kl.view(shape), rb, variant=capi.VARIANT_GEMM_BF16, taps=TAPS)),
                "learned_band_varying_with_fallback": nr(ops.tidas_forward_varying(
                    km.view(shape), rb, variant=capi.VARIANT_GEMM_BF16, taps=TAPS)),
                "exact_band_varying": nr(ops.tidas_forward_varying(kx.view(shape), r, taps=TAPS)),
                "fixed_band": nr(ops.tidas_forward_2d(Ps.fit_kernels_2d(kz, TAPS), r)),
                "fixed_rows": nr(ops.tidas_forward(Ps.fit_kernels(TAPS)[0], r))}}


# ------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    from tidas_workloads import presets, generators
    g = presets.geometry(GEOM)
    O = oracle.Oracle(g)
    # a bounded sample of the workload: channel data of frame 0's brightest
    # scatterers (the oracle cannot synthesise 100k scatterers per step in
    # seconds), then FP64 DAS of a fixed set of random pixels per step
    pos, amp = generators.compound_speckle_frame(0)
    rf = O.synthesize(pos[-200:], amp[-200:])
    rng = np.random.default_rng(0)
    npx = 32768
    pix = rng.choice(g["nx"] * g["nz"], npx, replace=False)
    for _ in range(args.warmup):
        O.das_pixels(rf, pix[:32])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.das_pixels(rf, pix)
    dt = (time.perf_counter() - t0) / args.steps
    value = npx / dt / 1e6
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixels/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "compounded plane-wave DAS: 128 el, 11 angles -10..10 deg, "
                               "4096 samples, 512x1024 px, cubic, F#1.5 (FP64 CPU oracle)",
                   "global_batch": 1, "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": "Mpixels/s", "cores": threads, "kind": "oracle",
                         "sample": "%d random pixels of one frame per step" % npx},
        "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.profile_case:
        run_profile_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
