#!/usr/bin/env python
"""Throughput of the P2S per-frame synthesis path on GB300.

Workload (one step): 64 RGB frames of 512 x 512, K = 100 basis PSFs of 33 x 33
taps (dictionary of 50,000 PSFs), network 33-128-128-100, D/r0 ~ U[1, 5],
Philox seed 10^6 + i per frame, synthetic blob images.  A step is one
p2s_simulate call over the batch: fields, warp, network and blur.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp16|fp32]
                  [--form scatter|gather] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(test infrastructure) on the host cores on a bounded sample of the same
workload, the only other place this script runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P2S frames/s & Mpix/s at 512² RGB K=100 vs roofline; p50/p99 frame latency"
N_FRAMES, HW, CH, K, TAPS, N_DICT = 64, 512, 3, 100, 33, 50_000
DIMS = [33, 128, 128, 100]
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes per 512x512 RGB frame of a kernel (dram__bytes_read.sum + dram__bytes_write.sum of one
# 8-frame launch under ncu, divided by 8: the traffic is proportional to the frames, 16-bit beta and
# x_w exceeding L2 already at 8 frames).  Each figure holds for the kernel source it was measured
# on (sha1 prefix of the file); a changed source reports traffic null until it is measured again.
TRAFFIC = {
    "blur_tc_gather16": {"bytes_per_frame": (496030976 + 20580352) / 8, "source": "k_gather.cu", "sha1": "52a4511d7d65"},
    "blur_tc_gather_h2": {"bytes_per_frame": (501780992 + 20037120) / 8, "source": "k_gather_h2.cu", "sha1": "02bbbc949cb0"},
    "net_tc": {"bytes_per_frame": (5723648 + 405348096) / 8, "source": "k_net.cu", "sha1": "dfdcffe784cd"},
    "blur_tc_scatter": {"bytes_per_frame": (505978624 + 20813312) / 8, "source": "k_scatter.cu", "sha1": "93a62d87a421"},
}
# the blur kernels: tensor flops 2 K T per pixel (the contraction; the fused kernel adds the
# network's), tap accumulation 2 C T FP32 flops per pixel on the FMA pipe
BLUR_KERNELS = ("blur_tc_gather16", "blur_tc_gather_h2", "blur_tc_gather8", "blur_tc_gather16f", "blur_tc_gather_x32",
                "fused_tc_gather", "blur_tc_scatter")


def source_sha1(name: str) -> str:
    import hashlib

    path = os.path.join(ROOT, "paper_2107_11627_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def roofline(kstats, peaks, peak_src, clk, px_per_launch, C, taps):
    """Roofline of the dominant kernel (by time in the timed region) and of every kernel.

    The tensor peak is the burst figure when the clocks sampled in the timed region sat at
    the maximum SM clock (a short region at full clock), the sustained one otherwise.  For a
    blur kernel the three-roof bound max(tensor, FP32-pipe tap accumulation, HBM) is added;
    the FP32 peak is 152 SMs x 128 FMA lanes x 2 flop x the sampled SM clock."""
    if not kstats:
        return None, []
    mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    at_max = bool(clk) and clk["sm_mhz"] >= 0.97 * clk["sm_max_mhz"]
    tc_key = "bf16_tflops" if at_max else "bf16_tflops_sustained"
    tc_peak = peaks[tc_key]
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    hbm = peaks["hbm_gbs"]
    per_kernel = []
    for s_ in kstats:
        avg_s = s_["total_ms"] / 1e3 / s_["launches"]
        e = {"kernel": s_["name"], "ms_per_launch": avg_s * 1e3}
        if s_["bytes"] > 0:
            gbs = s_["bytes"] / s_["launches"] / avg_s / 1e9
            e["achieved_gbs"], e["hbm_frac"] = gbs, gbs / hbm
        if s_["flops"] > 0 and "fp32" not in s_["name"] and s_["name"] != "fields_colour":
            tf = s_["flops"] / s_["launches"] / avg_s / 1e12
            e["achieved_tflops"], e["tensor_frac"] = tf, tf / tc_peak
        per_kernel.append(e)
    dom = max(kstats, key=lambda s_: s_["total_ms"])
    avg_s = dom["total_ms"] / 1e3 / dom["launches"]
    name = dom["name"]
    if "fp32" in name:
        achieved = dom["flops"] / dom["launches"] / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None, "kernel": name,
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz (sampled)"}
        return roof, per_kernel
    if dom["flops"] <= 0:
        achieved = dom["bytes"] / dom["launches"] / avg_s / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": name, "peak_source": f"{peak_src} hbm_gbs"}, per_kernel
    achieved = dom["flops"] / dom["launches"] / avg_s / 1e12
    t = TRAFFIC.get(name)
    traffic, note = None, "no ncu DRAM figure for this kernel"
    if t is not None and px_per_launch == N_FRAMES * 512 * 512:
        if source_sha1(t["source"]) == t["sha1"]:
            traffic, note = t["bytes_per_frame"] * N_FRAMES, "ncu, 8-frame launch scaled to the launch's frames"
        else:
            note = f"{t['source']} changed since its DRAM bytes were measured"
    roof = {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
            "frac": achieved / tc_peak, "traffic": traffic, "traffic_unit": "bytes per launch", "traffic_note": note,
            "kernel": name, "peak_source": f"{peak_src} {tc_key} ({'clocks at max' if at_max else 'below max clock'})"}
    if name in BLUR_KERNELS:
        T = taps * taps
        t_tc = dom["flops"] / dom["launches"] / (tc_peak * 1e12)
        t_fp32 = 2.0 * C * T * px_per_launch / (fp32_peak * 1e12)
        t_hbm = dom["bytes"] / dom["launches"] / (hbm * 1e9)
        roofs = {"tensor": t_tc, "fp32_taps": t_fp32, "hbm": t_hbm}
        bound = max(roofs, key=roofs.get)
        roof["three_roof"] = {"tensor_ms": t_tc * 1e3, "fp32_taps_ms": t_fp32 * 1e3, "hbm_ms": t_hbm * 1e3,
                              "bound": bound, "roof_ms": roofs[bound] * 1e3, "measured_ms": avg_s * 1e3,
                              "frac": roofs[bound] / avg_s, "fp32_peak_tflops": fp32_peak}
    return roof, per_kernel


def workload_name(precision: str, form: str) -> str:
    return (f"{N_FRAMES} RGB frames {HW}x{HW}, K={K}, {TAPS}x{TAPS} taps, MLP 33-128-128-100, "
            f"{precision} {form} blur, D/r0~U[1,5]")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as td

        torch.cuda.set_device(local)
        td.init_process_group("nccl")
        return td, rank, world, local
    return None, rank, world, local


def replica_inputs(rank: int, n_frames: int):
    """Rank r's share of a weak-scaling run: its own frames (image seeds, Philox seeds and
    D/r0 draws disjoint from every other rank's); no data crosses ranks."""
    from paper_2107_11627_gb300 import inputs

    first = rank * n_frames
    return {"image_seed": 1000 + first, "philox_seeds": inputs.frame_seeds(n_frames, 10**6 + first),
            "d_over_r0": inputs.frame_strengths(n_frames, 1.0, 5.0, 7 + rank)}


def max_over_ranks(td, value: float, device=None) -> float:
    """The job's time is the slowest rank's (the only collective of the run)."""
    if td is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def oracle_frame(H, layers, x, dr, seed, rows=None, form="scatter"):
    """(seconds, output) of the FP64 oracle for frame x (or its first `rows` rows)."""
    import oracle

    if rows is not None:
        x = x[:rows]
    t0 = time.perf_counter()
    y = oracle.frame.simulate(x.astype(np.float64), seed, dr, H, layers, oracle.fields.CorrParams(8, (16.0,)),
                              (TAPS, TAPS), form=form).y
    return time.perf_counter() - t0, y


def oracle_frame_time(H, layers, x, dr, seed, rows=None, form="scatter"):
    return oracle_frame(H, layers, x, dr, seed, rows, form)[0]


def run_reference(args):
    """The oracle as it stands, on the host cores, bounded sample per step."""
    _, rank, world, _ = (None, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0)
    if rank != 0:
        return 0
    from paper_2107_11627_gb300 import basis, inputs

    H = basis.build_basis(K, TAPS, N_DICT)
    layers = inputs.mlp_weights(DIMS, 42)
    dr = inputs.frame_strengths(N_FRAMES, 1.0, 5.0, 7)
    rows = args.ref_rows
    xs = [inputs.blob_image(HW, HW, CH, 1000 + i) for i in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        oracle_frame_time(H, layers, xs[i], float(dr[i % N_FRAMES]), 10**6 + i, rows)
    ts = [oracle_frame_time(H, layers, xs[args.warmup + i], float(dr[(args.warmup + i) % N_FRAMES]),
                            10**6 + args.warmup + i, rows) for i in range(args.steps)]
    frac = rows / HW
    fps = args.steps * frac / sum(ts)
    cores = os.cpu_count()
    sample = f"rows 0..{rows - 1} of one {HW}x{HW}x3 frame per step (full path, FP64 NumPy), scaled to frames"
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.precision, args.form)},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


SERVE_SIZES = [(256, 256), (512, 512), (576, 1024), (720, 1280), (1080, 1920), (1152, 2048)]


def run_batching(args, Hb, layers, precision, form, frames=96, steps=5):
    """96 RGB frames of uneven size (long side in {128..1024}, aspect 1..16:9), D/r0 ~ U[0.5, 6]:
    autotuned kernel and tile shape, captured as a CUDA graph (the gather kernels take the
    whole uneven batch in one persistent launch; the scatter kernel one launch per size)."""
    import torch

    from paper_2107_11627_gb300 import inputs, p2s

    sizes = inputs.uneven_sizes(frames, seed=96)
    xs = [torch.from_numpy(inputs.blob_image(h, w, CH, 5000 + i)).cuda() for i, (h, w) in enumerate(sizes)]
    ys = [torch.empty_like(x) for x in xs]
    dr = inputs.frame_strengths(frames, 0.5, 6.0, 9)
    seeds = inputs.frame_seeds(frames, 2 * 10**6)
    sim = p2s.Simulator(Hb, (TAPS, TAPS), layers, anchor_spacing=8, corr_len_px=(16.0,), precision=precision,
                        form=form)
    tune = sim.autotune(xs, dr, seeds, out=ys, reps=1)
    tune = {**tune, "candidates": {str(k): v for k, v in tune["candidates"].items()}, "best": str(tune["best"])}
    sim.set_option("graphs", 1)
    for _ in range(2):
        sim.simulate(xs, dr, seeds, out=ys)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream = torch.cuda.current_stream()
    ev[0].record(stream)
    for _ in range(steps):
        sim.simulate(xs, dr, seeds, out=ys)
    ev[1].record(stream)
    torch.cuda.synchronize()
    sim.check()
    ms = ev[0].elapsed_time(ev[1]) / steps
    mpx = sum(h * w for h, w in sizes) / 1e6
    out = {"workload": f"{frames} RGB frames of uneven size (long side 128..1024, aspect 1..16:9), "
                       f"{precision} {form}, autotuned, CUDA graph", "precision": precision, "form": form,
           "frames_per_s": frames / (ms / 1e3), "mpix_per_s": mpx / (ms / 1e3), "ms_per_call": ms,
           "mpix_per_call": mpx, "autotune": tune, "graph_instantiations": sim.get_option("graph_instantiations"),
           "graph_updates": sim.get_option("graph_updates")}
    sim.close()
    return out


def run_serving(args, Hb, layers, precision, form, rate=200.0, seconds=30.0, saturate=256):
    """Poisson arrivals of single RGB frames (sizes 256^2 .. 2048x1152, D/r0 ~ U[0.5, 6], own seed each)
    into the request loop; p50/p99 latency from submission to result in host memory."""
    import torch

    from paper_2107_11627_gb300 import inputs, p2s

    rng = np.random.default_rng(200)
    pin_in = {hw: torch.from_numpy(inputs.blob_image(hw[0], hw[1], CH, 6000 + i)).pin_memory().numpy()
              for i, hw in enumerate(SERVE_SIZES)}
    ring = 6
    pin_out = {hw: [torch.empty(hw + (CH,), dtype=torch.float32).pin_memory().numpy() for _ in range(ring)]
               for hw in SERVE_SIZES}
    sim = p2s.Simulator(Hb, (TAPS, TAPS), layers, anchor_spacing=8, corr_len_px=(16.0,), precision=precision,
                        form=form)
    srv = p2s.Server(sim, hbm_budget_bytes=8 << 30, max_inflight=4, max_batch=16)

    def drive(arrivals):
        t0 = time.perf_counter()
        tickets = []
        for k, t_arr in enumerate(arrivals):
            hw = SERVE_SIZES[rng.integers(len(SERVE_SIZES))]
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            tickets.append(srv.submit(pin_in[hw], float(rng.uniform(0.5, 6.0)), 10**7 + k, pin_out[hw][k % ring]))
        lat = [srv.wait(t, 120.0) for t in tickets]
        return lat, time.perf_counter() - t0

    drive(np.zeros(8))  # warm-up: kernels, pools
    n = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    lat, el = drive(arrivals)
    lat_sat, el_sat = drive(np.zeros(saturate))
    st = srv.stats()
    srv.close()
    sim.close()
    mean_px = float(np.mean([h * w for h, w in SERVE_SIZES]))
    return {"workload": f"Poisson {rate:.0f} req/s for {seconds:.0f} s, RGB frames of "
                        f"{'/'.join(f'{w}x{h}' for h, w in SERVE_SIZES)}, {precision} {form}",
            "precision": precision, "form": form,
            "requests": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "frames_per_s": n / el, "saturation": {"requests": saturate, "frames_per_s": saturate / el_sat,
                                                  "mpix_per_s": saturate * mean_px / 1e6 / el_sat,
                                                  "p50_ms": float(np.percentile(lat_sat, 50))},
            "mean_batch": st["mean_batch"], "peak_hbm_bytes": st["peak_bytes"],
            "latency_includes": "host->device copy, path, device->host copy"}


def run_bf16_line(args, Hb, layers, xs, ys, xs_host, dr, seeds, local):
    """The contract's BF16 path on the same workload: BF16 operands for the network and the
    contraction, scatter form (the form whose BF16 error stays inside 2e-3 of the FP64
    oracle; the gather form's per-output-pixel coefficients put BF16 above it), timed like
    the headline with its own roofline and clocks, frame 0 checked against the oracle."""
    import torch

    from paper_2107_11627_gb300 import p2s

    sim = p2s.Simulator(Hb, (TAPS, TAPS), layers, anchor_spacing=8, corr_len_px=(16.0,), precision="bf16",
                        form="scatter")
    for _ in range(args.warmup):
        sim.simulate(xs, dr, seeds, out=ys)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    sim.profile(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks.start()
    ev[0].record(stream)
    for _ in range(args.steps):
        sim.simulate(xs, dr, seeds, out=ys)
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sim.profile(False)
    sim.check()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    kstats = sim.profile_read()
    peaks, peak_src = load_peaks()
    roof, kroofs = roofline(kstats, peaks, peak_src, clk, N_FRAMES * HW * HW, CH, TAPS)
    out = {"precision": "bf16", "form": "scatter", "value": N_FRAMES / (ms / 1e3), "unit": "frames/s",
           "mpix_per_s": N_FRAMES * HW * HW / 1e6 / (ms / 1e3), "ms_per_step": ms, "steps": args.steps,
           "roofline": roof, "kernel_roofs": kroofs, "clocks": clk,
           "gpu_launches": sum(k["launches"] for k in kstats)}
    if not args.no_cpu_baseline:
        _, y_ref = oracle_frame(Hb, layers, xs_host[0], float(dr[0]), int(seeds[0]), form="scatter")
        err = ys[0].cpu().numpy().astype(np.float64) - y_ref
        out["accuracy"] = {"frame": 0, "vs": "FP64 oracle", "rel_l2": float(np.linalg.norm(err) / np.linalg.norm(y_ref)),
                           "max_abs": float(np.abs(err).max()), "tol_rel_l2": 2e-3}
    sim.close()
    return out


def run_spectral(args, layers, xs, ys, dr, seeds, n_dict=8000):
    """Wavelength-dependent RGB (three PSF sets at 570, 540, 450 nm) on the headline workload
    and precision: three single-channel passes.  The channel bases come from an n_dict-draw
    dictionary each (throughput does not depend on the basis values)."""
    import torch

    from paper_2107_11627_gb300 import basis, p2s

    bases = basis.build_basis_spectral(K, TAPS, n_dict)
    sim = p2s.SpectralSimulator(bases, (TAPS, TAPS), layers, anchor_spacing=8, corr_len_px=(16.0,),
                                precision=args.precision, form=args.form)
    for _ in range(args.warmup):
        sim.simulate(xs, dr, seeds, out=ys)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(args.steps):
        sim.simulate(xs, dr, seeds, out=ys)
    ev[1].record(stream)
    torch.cuda.synchronize()
    sim.check()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    sim.close()
    return {"workload": f"{N_FRAMES} RGB frames {HW}x{HW}, three wavelength bases (570/540/450 nm), "
                        f"{args.precision} {args.form}", "frames_per_s": N_FRAMES / (ms / 1e3), "ms_per_step": ms,
            "bases_from_dictionary_of": n_dict}


def fp32_batched_fps(Hb, layers, frames=8):
    """The plain FP32 batched path at 512^2 RGB (scatter form), for comparison with serving."""
    import torch

    from paper_2107_11627_gb300 import inputs, p2s

    sim = p2s.Simulator(Hb, (TAPS, TAPS), layers, anchor_spacing=8, corr_len_px=(16.0,), precision="fp32",
                        form="scatter")
    xs = [torch.from_numpy(x).cuda() for x in inputs.blob_batch(frames, HW, HW, CH, 1000)]
    dr = inputs.frame_strengths(frames, 1.0, 5.0, 7)
    seeds = inputs.frame_seeds(frames)
    sim.simulate(xs, dr, seeds)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.simulate(xs, dr, seeds)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    sim.close()
    return frames / el


def main():
    global N_FRAMES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="fp16", choices=["bf16", "fp16", "fp32", "fp8"])
    ap.add_argument("--form", default="gather", choices=["scatter", "gather", "fft"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=128, help="rows per step of the reference arm's sample")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--frames", type=int, default=64, help="frames per step (profiling runs only)")
    ap.add_argument("--no-batching", action="store_true", help="skip the uneven-size batching workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload")
    ap.add_argument("--no-bf16-line", action="store_true", help="skip the BF16 (scatter) line of an FP16 run")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="Poisson arrival window of the serving run")
    ap.add_argument("--spectral", action="store_true",
                    help="also time wavelength-dependent RGB (three bases, 570/540/450 nm) on the workload")
    ap.add_argument("--gather-split", type=int, default=None,
                    help="tensor-core gather kernel: 0 fused, 1 or 2 blur-only (default: the library's)")
    args = ap.parse_args()
    N_FRAMES = args.frames
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2107_11627_gb300 import basis, inputs, p2s

    td, rank, world, local = dist()
    torch.cuda.set_device(local)
    Hb = basis.build_basis(K, TAPS, N_DICT)
    layers = inputs.mlp_weights(DIMS, 42)
    sim = p2s.Simulator(Hb, (TAPS, TAPS), layers, anchor_spacing=8, corr_len_px=(16.0,),
                        precision=args.precision, form=args.form)
    if args.gather_split is not None:
        sim.set_option("gather_split", args.gather_split)
    share = replica_inputs(rank, N_FRAMES)
    xs_host = inputs.blob_batch(N_FRAMES, HW, HW, CH, share["image_seed"])
    dr = share["d_over_r0"]
    seeds = share["philox_seeds"]
    xs = [torch.from_numpy(x).cuda() for x in xs_host]
    ys = [torch.empty_like(x) for x in xs]
    stream = torch.cuda.current_stream()

    def step():
        sim.simulate(xs, dr, seeds, out=ys)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if td is not None:
            td.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    sim.profile(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    clocks.start()
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    sim.profile(False)
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    kstats = sim.profile_read()
    total_ms = max_over_ranks(td, total_ms, "cuda")
    frames_total = N_FRAMES * args.steps * world
    fps = frames_total / (total_ms / 1e3)
    mpix = fps * HW * HW / 1e6

    # roofline of the dominant kernel, from its own launches in the timed region
    peaks, peak_src = load_peaks()
    roof, kernel_roofs = roofline(kstats, peaks, peak_src, clk, N_FRAMES * HW * HW, CH, TAPS)
    launches = sum(s["launches"] for s in kstats)

    # end to end through the host-buffer entry point: H2D + path + D2H inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        pin_in = [torch.from_numpy(x).pin_memory() for x in xs_host]
        pin_out = [torch.empty_like(p).pin_memory() for p in pin_in]
        hin = [p.numpy() for p in pin_in]
        hout = [p.numpy() for p in pin_out]
        sim.simulate_host(hin, dr, seeds, out=hout)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sim.simulate_host(hin, dr, seeds, out=hout)
        el = time.perf_counter() - t0
        el = max_over_ranks(td, el, "cuda")
        bytes_step = N_FRAMES * HW * HW * CH * 4
        e2e = {"value": N_FRAMES * args.e2e_steps * world / el, "unit": "frames/s",
               "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": bytes_step}

    cpu, acc = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        form = args.form if args.form in ("scatter", "gather") else "scatter"
        t, y_ref = oracle_frame(Hb, layers, xs_host[0], float(dr[0]), int(seeds[0]), form=form)
        cpu = {"value": 1.0 / t, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"frame 0 of the batch ({HW}x{HW}x3), full path, FP64 NumPy, one run"}
        y_gpu = ys[0].cpu().numpy().astype(np.float64)
        err = y_gpu - y_ref
        acc = {"frame": 0, "vs": "FP64 oracle", "rel_l2": float(np.linalg.norm(err) / np.linalg.norm(y_ref)),
               "max_abs": float(np.abs(err).max())}

    bf16_line = None
    if rank == 0 and world == 1 and args.precision == "fp16" and not args.no_bf16_line:
        bf16_line = run_bf16_line(args, Hb, layers, xs, ys, xs_host, dr, seeds, local)

    batching = serving = spectral = None
    tc_path = args.precision in ("fp16", "bf16")
    # the a9 workloads on the headline path and on the contract's BF16 (scatter) path
    paths = [(args.precision, args.form)] + ([("bf16", "scatter")] if args.precision == "fp16" else [])
    if rank == 0 and world == 1 and tc_path and not args.no_batching:
        batching = [run_batching(args, Hb, layers, pr, fm) for pr, fm in paths]
    if rank == 0 and world == 1 and tc_path and not args.no_serving:
        fp32_fps = fp32_batched_fps(Hb, layers)
        serving = [run_serving(args, Hb, layers, pr, fm, seconds=args.serve_seconds) for pr, fm in paths]
        for sv in serving:
            sv["fp32_batched_512_frames_per_s"] = fp32_fps
    if rank == 0 and world == 1 and args.spectral:
        spectral = run_spectral(args, layers, xs, ys, dr, seeds)

    if rank == 0:
        dtype = {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3"}[args.precision]
        line = {"metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": workload_name(args.precision, args.form), "frames": N_FRAMES, "H": HW,
                           "W": HW, "C": CH, "K": K, "taps": f"{TAPS}x{TAPS}", "precision": args.precision,
                           "form": args.form, "anchor_spacing": 8, "parallelism": f"replicas x{world}",
                           "l2": f"inputs larger than L2 ({N_FRAMES * HW * HW * CH * 4 / 1e6:.0f} MB per step)"},
                "mpix_per_s": mpix,
                "latency_ms": {"step_p50": float(np.percentile(step_ms, 50)),
                               "step_p99": float(np.percentile(step_ms, 99)),
                               "frame_p50": float(np.percentile(step_ms, 50)) / N_FRAMES},
                "roofline": roof, "kernel_roofs": kernel_roofs, "bf16": bf16_line, "cpu_baseline": cpu, "accuracy": acc, "batching": batching, "serving": serving, "spectral": spectral, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
                "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()} for s in kstats]}
        print(json.dumps(line), flush=True)
    sim.close()
    if td is not None:
        td.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
