"""Benchmark of the FoE Poisson denoiser's iPiano solve on GB300.

Workload (one "step"): the 512x512 set of the paper's noise levels -- peaks {1, 2, 4, 8, 30} x
{direct model, Anscombe quadratic model} = 10 seeded synthetic 512x512 images, 300 iterations each,
denoised as one batch through the C ABI (foe_denoise_batch, each image with its own data term).  Metric: MPix.iter/s, i.e.
pixels x iterations per second (whole job, inputs already in HBM; L2 flushed between steps).

Printed as one JSON line on rank 0.  Extra keys:
  - the TF32 and plain-FP32 paths on the same workload, and the single-image latency;
  - the roofline of the fused step kernel;
  - the FP64 oracle on the host cores;
  - an end-to-end figure through the public API with host buffers;
  - 64 uneven images in one CUDA graph, the training step (unrolled and implicit-differentiation gradients),
    the continuous-batching server, the binning variant and backtracking step control;
  - the SM clocks seen meanwhile.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec bf16|tf32|fp32]
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 512
ITERS = 300
PEAKS = (1.0, 2.0, 4.0, 8.0, 30.0)
FLOP_PER_PIXEL_ITER = 2 * 2 * 48 * 49   # forward + adjoint 7x7 convolutions of 48 filters, FMA = 2 flop
METRIC = "MPix·iter/s at 512² (TC BF16 vs FP32 plain, PSNR Δ≤0.02dB vs FP64); serve p99"
CONFIG_NAME = "512x512 x peaks{1,2,4,8,30} x models{direct,anscombe-L2}, 300 iters, 48 7x7 filters"


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the timing rule: the job is as slow as its slowest rank)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput in units per second: every rank processes its own equal share (weak scaling)."""
    return world * units_per_rank / seconds


def rank_seed(base: int, rank: int) -> int:
    """Seeds of rank r's synthetic inputs: distinct per rank so replicas never denoise the same images."""
    return base + 100 * rank


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = {"foe_pair_step": ("foe_pair.cu", "foe_ptx.cuh", "foe_common.cuh"),
                  "foe_tc_step": ("foe_tc.cu", "foe_ptx.cuh", "foe_common.cuh"),
                  "foe_f32_step": ("foe_f32.cu", "foe_common.cuh")}


def code_only(text: str) -> str:
    """CUDA/C++ source without its // comments, trailing blanks and blank lines (the sources here put no // inside
    string literals), so that a comment edit does not count as a code change."""
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_source_sha(kernel_key: str) -> str:
    """Hash of the code of one kernel's sources: an ncu figure is only used while that code is unchanged."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel_key]:
        with open(os.path.join(ROOT, "paper_1609_05722_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if it matches the source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get(kernel_key)
    if not e or e.get("source_sha") != kernel_source_sha(kernel_key):
        return None
    return e.get("bytes_per_launch")


# ----------------------------------------------------------------------------- accuracy vs the stored oracle set

def load_golden():
    """FP64 oracle results of the 512x512 set (written by tests/golden/make_oracle_512.py from the oracle alone):
    per (model, peak) its PSNR against the clean image and its output at sampled pixels."""
    with open(os.path.join(ROOT, "tests", "golden", "oracle_512.json")) as f:
        return json.load(f)


def psnr(x, clean, peak) -> float:
    """10 log10(peak^2 / mean (x - clean)^2), the PSNR of the paper's tables on the [0, peak] scale."""
    e = np.asarray(x, dtype=np.float64) - np.asarray(clean, dtype=np.float64)
    return float(10.0 * np.log10(peak * peak / np.mean(e * e)))


def accuracy_rows(golden, outputs):
    """outputs: {(model, peak): H x W output}.  Per case: the oracle's PSNR, this output's PSNR and the difference,
    and the max |x - x_oracle| over the stored sample of pixels on the [0, 255] scale (255 / peak)."""
    from paper_1609_05722_gb300 import synth
    idx = np.array(golden["sample_index"])
    rows = []
    for c in golden["cases"]:
        key = (c["model"], c["peak"])
        if key not in outputs:
            continue
        x = outputs[key]
        pi = PEAKS.index(c["peak"])
        clean = synth.clean_image(H, W, 1000 + 10 * pi) * c["peak"]
        p = psnr(x, clean, c["peak"])
        rows.append({"model": c["name"], "peak": c["peak"], "psnr_oracle": round(c["psnr_oracle"], 4),
                     "psnr": round(p, 4), "dpsnr_db": round(p - c["psnr_oracle"], 4),
                     "max_abs_255": float(np.abs(x.ravel()[idx] - np.array(c["x_sample"])).max() * 255.0 / c["peak"])})
    return rows


# ----------------------------------------------------------------------------- oracle (CPU) timing

def oracle_sample(target_s: float = 12.0, nthreads=None):
    """The FP64 oracle as it stands on the host cores: one 512x512 image, iterations run until ~target_s
    (nthreads None: every host core, as the oracle defaults to)."""
    import oracle as O
    from paper_1609_05722_gb300 import synth
    k, a = synth.filter_bank()
    y = synth.poisson_observation(synth.clean_image(H, W, 1000), 4.0, 5000)
    d = O.anscombe(y)
    pr = O.Problem(k, a, H, W, model=O.MODEL_ANS_L2, lam=1.0, tau=1e-3, gamma=0.8, nthreads=nthreads)
    u, up = d.copy(), d.copy()
    t0 = time.perf_counter()
    n = 0
    while True:
        un = pr.step(d, u, up)
        up, u = u, un
        n += 1
        if time.perf_counter() - t0 >= target_s:
            break
    dt = time.perf_counter() - t0
    threads = nthreads or O.default_threads()
    return {"value": H * W * n / dt / 1e6, "unit": "MPix·iter/s", "cores": threads,
            "kind": "oracle",
            "sample": f"FP64 oracle, one 512x512 image (Anscombe quadratic model), {n} iPiano iterations, "
                      f"{threads} threads, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        oracle_sample(2.0)
    t_steps = []
    for _ in range(args.steps):
        s = oracle_sample(10.0)
        vals.append(s["value"])
        t_steps.append(H * W / (s["value"] * 1e6))
    cb = oracle_sample(0.0)
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MPix·iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(t_steps)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CONFIG_NAME + " (oracle: bounded per-iteration sample of one image)",
                       "step": "~10 s of FP64 oracle iterations on one 512x512 image"},
            "cpu_baseline": {"value": v, "unit": "MPix·iter/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": "each step: FP64 oracle iterations on one 512x512 image for ~10 s"},
            "e2e": {"value": v, "unit": "MPix·iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- serving leg

def serving_pool(rank: int):
    """Page-locked pool of noisy images that requests are cropped from (generating 2000 fresh images would
    dominate the run): 2048^2 natural-image stand-ins at 4 peaks and one 4096^2 microscopy-like tile."""
    import torch
    from paper_1609_05722_gb300 import synth
    pool = {}
    for j, peak in enumerate((1.5, 3.0, 8.0, 20.0)):
        c = synth.clean_image(2048, 2048, 7000 + j + 100 * rank)
        pool[peak] = torch.from_numpy(synth.poisson_observation(c, peak, 7100 + j + 100 * rank).astype(np.float32)).pin_memory()
    c = synth.microscopy_tile(4096, 4096, 7200 + rank)
    pool["micro"] = torch.from_numpy(synth.poisson_observation(c, 1.5, 7201 + rank).astype(np.float32)).pin_memory()
    return pool


def run_serving(F, ctx, pool, n_req: int, rate: float, prec: int, budget: int, per_tick: int, graphs: bool,
                per_request: bool = False):
    """Replays a Poisson arrival stream in real time.  Latency = completion time - scheduled arrival time."""
    import torch
    from paper_1609_05722_gb300 import synth
    arrivals = synth.serving_arrivals(n_req, rate, 42)
    reqs = []
    rng = np.random.default_rng(4242)
    for t, spec in arrivals:
        if spec.microscopy:
            key, side_h, side_w = "micro", 4096, 4096
        else:
            key = min((1.5, 3.0, 8.0, 20.0), key=lambda p: abs(np.log(p / spec.peak)))
            side_h, side_w = 2048, 2048
        base = pool[key]
        H, W = min(spec.H, side_h), min(spec.W, side_w)
        r0 = int(rng.integers(0, side_h - H + 1))
        c0 = int(rng.integers(0, side_w - W + 1))
        ptr = base.data_ptr() + 4 * (r0 * side_w + c0)
        peak = 1.5 if key == "micro" else key
        view = base.view(side_h, side_w)[r0:r0 + H, c0:c0 + W]
        reqs.append((t, H, W, ptr, side_w, peak, 150 if peak < 5 else 100, view))
    out = torch.empty(4096 * 4096, dtype=torch.float32).pin_memory()
    lat, pix, pix_it = [], 0, 0
    t0 = time.perf_counter()
    if per_request:
        # plain per-request path: one foe_denoise at a time, host copies in and out
        stream = torch.cuda.current_stream()
        for (ta, H, W, ptr, pitch, peak, iters, view) in reqs:
            now = time.perf_counter() - t0
            if now < ta:
                time.sleep(ta - now)
            ld = (W + 3) // 4 * 4
            yd = torch.empty((H, ld), dtype=torch.float32, device="cuda")
            yd[:, :W].copy_(view, non_blocking=True)
            xd = torch.empty_like(yd)
            F.foe_denoise(ctx, yd, xd, H, W, ld, peak, F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=prec, iters=iters),
                          stream=stream)
            out[:H * W].view(H, W).copy_(xd[:, :W], non_blocking=True)
            stream.synchronize()
            lat.append(time.perf_counter() - t0 - ta)
            pix += H * W
            pix_it += H * W * iters
        makespan = time.perf_counter() - t0
        return {"requests": len(reqs), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mpix_per_s": pix / makespan / 1e6,
                "mpix_iter_per_s": pix_it / makespan / 1e6, "makespan_s": makespan}
    srv = F.foe_server_create(ctx, budget, 64, per_tick, graphs, F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=prec))
    arrival_of, size_of = {}, {}
    i, done = 0, 0
    try:
        while done < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i][0] <= now:
                ta, H, W, ptr, pitch, peak, iters, _ = reqs[i]
                rid = F.foe_server_submit(srv, ptr, out.data_ptr(), H, W, peak, iters, y_pitch=pitch, x_pitch=W,
                                          ctx=ctx)
                arrival_of[rid] = ta
                size_of[rid] = (H * W, iters)
                i += 1
            st = F.foe_server_get_stats(srv)
            if st["queued"] == 0 and st["active"] == 0 and st["finishing"] == 0:
                if i < len(reqs):
                    time.sleep(max(0.0, reqs[i][0] - (time.perf_counter() - t0)))
                continue
            F.foe_server_tick(srv, ctx)
            tdone = time.perf_counter() - t0
            for rid in F.foe_server_poll(srv):
                lat.append(tdone - arrival_of[rid])
                pix += size_of[rid][0]
                pix_it += size_of[rid][0] * size_of[rid][1]
                done += 1
        st = F.foe_server_get_stats(srv)
    finally:
        F.foe_server_destroy(srv)
    makespan = time.perf_counter() - t0
    return {"requests": len(reqs), "rate_hz": rate, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mpix_per_s": pix / makespan / 1e6,
            "mpix_iter_per_s": pix_it / makespan / 1e6, "makespan_s": makespan, "ticks": st["ticks"],
            "launches": st["launches"], "hbm_budget_gb": budget / 2**30, "peak_state_gb": st["bytes_peak"] / 2**30,
            "max_active": 64, "iters_per_tick": per_tick, "graphs": graphs}


# ----------------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "tf32", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--no-train", dest="train", action="store_false",
                    help="skip the prior-training leg (128 x 180^2, 50 unrolled iterations)")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the leg with 64 uneven images in one CUDA graph")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests in the serving leg (Poisson arrivals, 200/s); 0 skips it")
    ap.add_argument("--serve-baseline-requests", type=int, default=60,
                    help="prefix of the same stream run through the plain per-request path")
    ap.add_argument("--main-only", action="store_true",
                    help="time the main path only (no FP32 comparison, single-image or end-to-end legs); "
                         "used for profiler captures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.main_only:
        args.fp32_steps = 0
        args.no_cpu_baseline = True

    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__ as G
    from paper_1609_05722_gb300 import build as B
    B.build()
    from paper_1609_05722_gb300 import foe as F
    from paper_1609_05722_gb300 import synth

    # cpu baseline first (rank 0, before any GPU work would compete for host cores)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(12.0)
        cpu["single_thread"] = oracle_sample(8.0, nthreads=1)

    k, a = synth.filter_bank()
    ctx = F.foe_create(k, a)
    stream = torch.cuda.current_stream()
    ld = W
    # 10 images: peaks x models; rank-dependent seeds (weak scaling: every rank its own images)
    ys_host, ys, xs = [], [], []
    for mi, model in enumerate((F.FOE_MODEL_DIRECT, F.FOE_MODEL_ANS_L2)):
        for pi, peak in enumerate(PEAKS):
            seed = rank_seed(1000 + 10 * pi, rank)
            y = synth.poisson_observation(synth.clean_image(H, W, seed), peak, seed + 5000).astype(np.float32)
            yh = torch.from_numpy(y).pin_memory()
            ys_host.append(yh)
            ys.append(yh.to(dev))
            xs.append(torch.empty((H, ld), dtype=torch.float32, device=dev))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2 (129 MB)

    def descs(xbufs, ybufs, lo, hi, iters=ITERS):
        # images 0-4 take the direct model, 5-9 the Anscombe quadratic model (one batch, per-image data terms)
        return [{"y": ybufs[j], "x": xbufs[j], "H": H, "W": W, "ld": ld, "peak": PEAKS[j % 5], "iters": iters,
                 "model": F.FOE_MODEL_DIRECT if j < 5 else F.FOE_MODEL_ANS_L2} for j in range(lo, hi)]

    def one_step(prec, xbufs=xs, ybufs=ys):
        # the ten images in one batched solve: one step launch per iteration over the tiles of all of them
        F.foe_denoise_batch(ctx, descs(xbufs, ybufs, 0, 10), F.SolveOpts(prec=prec), stream=stream)

    golden = load_golden() if rank == 0 else None

    def snapshot():
        """The outputs of the last step, keyed (model, peak), on the host."""
        torch.cuda.synchronize()
        return {(int(mi), PEAKS[pi]): xs[5 * mi + pi][:, :W].double().cpu().numpy()
                for mi in (0, 1) for pi in range(5)}

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            one_step(prec)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        total = 0.0
        F.foe_profile(ctx, True)
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(prec)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        F.foe_profile(ctx, False)
        loop_ms, launches, pix = F.foe_profile_read(ctx)
        torch.cuda.synchronize()
        if world > 1:
            total = max_over_ranks(total, dist, dev)
            dist.barrier()
        return total, loop_ms, launches, pix

    prec_main = {"bf16": F.FOE_PREC_BF16, "tf32": F.FOE_PREC_TF32, "fp32": F.FOE_PREC_FP32}[args.prec]
    try:
        F.foe_denoise_batch(ctx, descs(xs, ys, 0, 1, 1), F.SolveOpts(prec=prec_main), stream=stream)  # a probe
    except F.FoeError as e:
        if e.status == F.FOE_EUNSUPPORTED and prec_main != F.FOE_PREC_FP32:
            prec_main = F.FOE_PREC_FP32  # tensor-core path not built into this library
        else:
            raise
    dtype = {F.FOE_PREC_BF16: "bf16", F.FOE_PREC_TF32: "tf32", F.FOE_PREC_FP32: "f32"}[prec_main]

    sampler = ClockSampler(local if world > 1 else 0)
    sampler.start()
    total_ms, loop_ms, launches, pix = timed(prec_main, args.steps, args.warmup)
    clocks = sampler.stop()
    accuracy = {dtype: accuracy_rows(golden, snapshot())} if golden else None
    pix_iters_step = 10 * H * W * ITERS
    value = job_value(pix_iters_step * args.steps, total_ms / 1e3, world) / 1e6
    ms_per_step = total_ms / args.steps

    # roofline of the fused step kernel (average launch = step-loop device time / launches)
    peaks, peak_src = measured_peaks()
    avg_launch_s = (loop_ms / 1e3) / max(launches, 1)
    pix_per_launch = pix / max(launches, 1)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # the step kernel is timed inside a ~31 ms step of back-to-back launches, not a seconds-long loop: the burst
    # figure is its denominator
    if prec_main != F.FOE_PREC_FP32:
        peak = peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained"))
        if prec_main == F.FOE_PREC_TF32:
            peak *= 1.1 / 2.25  # nominal dense TF32 : BF16 rate
        bound, unit = "tensor", "TFLOP/s"
        key = "foe_pair_step" if prec_main == F.FOE_PREC_BF16 else "foe_tc_step"
    else:
        peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, unit, key = "alu", "TFLOP/s", "foe_f32_step"
    achieved = pix_per_launch * FLOP_PER_PIXEL_ITER / avg_launch_s / 1e12
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": ncu_traffic(key), "peak_source": f"{peak_src}"
                + ((" bf16_tflops (burst)" + (" x 1.1/2.25 (nominal tf32:bf16)" if dtype == "tf32" else ""))
                   if bound == "tensor" else f" {sms} SMs x 128 FFMA/clk x 2 x sm_max_mhz"),
                "kernel": key, "avg_launch_us": avg_launch_s * 1e6, "pixels_per_launch": pix_per_launch}

    # plain FP32 path on the same workload (the comparison the metric names)
    fp32 = None
    if prec_main == F.FOE_PREC_BF16 and args.fp32_steps > 0:
        t32, l32, n32, p32 = timed(F.FOE_PREC_FP32, args.fp32_steps, 1)
        fp32 = {"value": world * pix_iters_step * args.fp32_steps / (t32 / 1e3) / 1e6, "unit": "MPix·iter/s",
                "ms_per_step": t32 / args.fp32_steps,
                "avg_launch_us": (l32 / 1e3) / max(n32, 1) * 1e6}
        if golden:
            accuracy["f32"] = accuracy_rows(golden, snapshot())

    if args.main_only:
        F.foe_destroy(ctx)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "MPix·iter/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                              "dtype": dtype, "roofline": roofline, "clocks": clocks, "main_only": True}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0

    # TF32 tensor-core convolutions on the same workload (the third precision of the comparison)
    tf32 = None
    if prec_main == F.FOE_PREC_BF16 and args.fp32_steps > 0:
        t3, l3, n3, p3 = timed(F.FOE_PREC_TF32, args.fp32_steps, 1)
        tf32 = {"value": job_value(pix_iters_step * args.fp32_steps, t3 / 1e3, world) / 1e6, "unit": "MPix·iter/s",
                "ms_per_step": t3 / args.fp32_steps, "avg_launch_us": (l3 / 1e3) / max(n3, 1) * 1e6}
        if golden:
            accuracy["tf32"] = accuracy_rows(golden, snapshot())

    # the I-divergence model (the paper's low-count data term) on the same five images: an accuracy row per
    # precision, outside the timed workload
    if golden and not args.main_only:
        for name, prec in (("bf16", F.FOE_PREC_BF16), ("tf32", F.FOE_PREC_TF32), ("f32", F.FOE_PREC_FP32)):
            if name not in accuracy:
                continue
            F.foe_denoise_batch(ctx, [dict(dd, model=F.FOE_MODEL_ANS_IDIV) for dd in descs(xs, ys, 5, 10)],
                                F.SolveOpts(prec=prec), stream=stream)
            torch.cuda.synchronize()
            outs = {(2, PEAKS[pi]): xs[5 + pi][:, :W].double().cpu().numpy() for pi in range(5)}
            accuracy[name] += accuracy_rows(golden, outs)

    # the stopping rule (relative change <= 1e-4, checked every 10 steps) on the timed workload: iterations taken
    # per image and the step time, against the fixed 300-iteration budget
    stopping = None
    if not args.main_only:
        tol, every = 1e-4, 10

        def tol_step():
            F.foe_denoise_batch(ctx, descs(xs, ys, 0, 10), F.SolveOpts(prec=prec_main, tol=tol, tol_every=every),
                                stream=stream)
            return F.foe_iters_done(ctx, 10, stream=stream)
        for _ in range(3):
            tol_step()
        tts = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            done = tol_step()
            e1.record(stream)
            e1.synchronize()
            tts.append(e0.elapsed_time(e1))
        acc_tol = accuracy_rows(golden, snapshot()) if golden else None
        stopping = {"tol": tol, "tol_every": every, "budget": ITERS,
                    "iters_done": {f"{m}@{p:g}": n for (m, p), n in
                                   zip([(m, p) for m in ("direct", "anscombe_l2") for p in PEAKS], done)},
                    "ms_per_step": float(np.median(tts)), "ms_per_step_fixed_budget": ms_per_step,
                    "images_per_s": 10 / (float(np.median(tts)) / 1e3),
                    "accuracy_vs_oracle_300": acc_tol}

    # step control by Lipschitz backtracking (FP32, one 512x512 image, 100 iterations, A2 model at peak 8): the
    # host decides every trial, so this leg reports its wall time and the trial counts, not a throughput target
    backtrack = None
    if not args.main_only and rank == 0:
        xb = torch.empty((H, ld), dtype=torch.float32, device=dev)
        ob = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_FP32, step=F.FOE_STEP_BACKTRACK, iters=100)
        F.foe_denoise(ctx, ys[8], xb, H, W, ld, 8.0, ob, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = F.foe_denoise(ctx, ys[8], xb, H, W, ld, 8.0, ob, stream=stream, report=True)
        wall = time.perf_counter() - t0
        tb, ab = F.foe_step_log(ctx)
        backtrack = {"H": H, "W": W, "iters": 100, "prec": "fp32", "wall_ms": wall * 1e3, "trials": int(len(tb)),
                     "rejected": int((~ab).sum()), "lipschitz_final": rb["lipschitz_final"],
                     "mpix_iter_per_s": H * W * 100 / wall / 1e6}

    # single-image latency (one 512x512 image, 300 iterations, A2 model at peak 8)
    xs1 = torch.empty((H, ld), dtype=torch.float32, device=dev)
    for _ in range(2):
        F.foe_denoise(ctx, ys[8], xs1, H, W, ld, 8.0, F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=prec_main,
                                                                    iters=ITERS), stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    for _ in range(3):
        flush.zero_()
        e0.record(stream)
        F.foe_denoise(ctx, ys[8], xs1, H, W, ld, 8.0, F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=prec_main,
                                                                    iters=ITERS), stream=stream)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))

    # binning variant (3x3 bins, solve at 9x peak, bilinear upscaling) on one 512x512 image at peak 0.5, the regime
    # the paper bins in: 300 iterations on the 171x171 bin image, against the same image solved at full size
    binned = None
    if not args.main_only and rank == 0:
        pk = 0.5
        yb_img = torch.from_numpy(synth.poisson_observation(synth.clean_image(H, W, 1200), pk, 6200)
                                  .astype(np.float32)).to(dev)
        yb_full = torch.zeros((H, ld), dtype=torch.float32, device=dev)
        yb_full[:, :W] = yb_img
        xb = torch.empty((H, ld), dtype=torch.float32, device=dev)
        ob = F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=prec_main, iters=ITERS)
        tb = {}
        for name, fn in (("binned", F.foe_denoise_binned), ("full", F.foe_denoise)):
            for _ in range(3):
                fn(ctx, yb_full, xb, H, W, ld, pk, ob, stream=stream)
            ts = []
            for _ in range(5):
                flush.zero_()
                e0.record(stream)
                fn(ctx, yb_full, xb, H, W, ld, pk, ob, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            tb[name] = float(np.median(ts))
        binned = {"H": H, "W": W, "peak": pk, "iters": ITERS, "bin_image": [(H + 2) // 3, (W + 2) // 3],
                  "binned_ms": tb["binned"], "full_ms": tb["full"]}

    # end to end through the public API: pinned host -> device, solve, device -> pinned host, each step
    xs_host = [torch.empty((H, ld), dtype=torch.float32).pin_memory() for _ in range(10)]
    ybuf = [torch.empty((H, ld), dtype=torch.float32, device=dev) for _ in range(10)]

    def e2e_step():
        for j in range(10):
            ybuf[j].copy_(ys_host[j], non_blocking=True)
        one_step(prec_main, xbufs=xs, ybufs=ybuf)
        for j in range(10):
            xs_host[j].copy_(xs[j], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    t_e2e = time.perf_counter() - t0
    if world > 1:
        t_e2e = max_over_ranks(t_e2e, dist, dev)
    e2e = {"value": job_value(pix_iters_step * args.steps, t_e2e, world) / 1e6, "unit": "MPix·iter/s",
           "h2d_bytes_per_step": 10 * H * W * 4, "d2h_bytes_per_step": 10 * H * ld * 4}

    # batched uneven instances in one graph: 64 images, sides {128..1024}, peaks log-U[1, 30], 100-300 iters
    batched = None
    if args.batched:
        specs = synth.batched_uneven_specs(64, seed=3 + 100 * rank)
        bys, bxs, bdescs = [], [], []
        for sp in specs:
            _, yb = synth.make_problem(sp)
            ldb = (sp.W + 3) // 4 * 4
            yd = torch.zeros((sp.H, ldb), dtype=torch.float32, device=dev)
            yd[:, :sp.W] = torch.from_numpy(yb.astype(np.float32)).to(dev)
            bys.append(yd)
            bxs.append(torch.zeros_like(yd))
            bdescs.append({"y": yd, "x": bxs[-1], "H": sp.H, "W": sp.W, "ld": ldb, "peak": sp.peak, "iters": sp.iters})
        gstream = torch.cuda.Stream(device=dev)
        bopts = F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=prec_main, use_graph=True)
        with torch.cuda.stream(gstream):
            for _ in range(2):
                F.foe_denoise_batch(ctx, bdescs, bopts, stream=gstream)
            gstream.synchronize()
            times = []
            for _ in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(gstream)
                F.foe_denoise_batch(ctx, bdescs, bopts, stream=gstream)
                e1.record(gstream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        bpix = sum(sp.H * sp.W * sp.iters for sp in specs)
        batched = {"images": len(specs), "pixel_iters": bpix, "ms": float(np.median(times)),
                   "value": bpix / (float(np.median(times)) / 1e3) / 1e6, "unit": "MPix·iter/s",
                   "graph": True, "sides": "H, W independently from {128,256,384,512,768,1024}",
                   "iters": "U{100..300} per image", "peaks": "log-U[1, 30]"}
        del bys, bxs, bdescs

    # prior training: 128 pairs of 180x180 at peak 4, 50 checkpointed iterations, loss + gradient per step
    train = None
    if args.train:
        TB, TH, TW, TT = 128, 180, 180, 50
        tld = (TW + 3) // 4 * 4
        tk, ta = synth.filter_bank()
        cl = torch.zeros((TB, TH, tld), dtype=torch.float32, device=dev)
        nz = torch.zeros((TB, TH, tld), dtype=torch.float32, device=dev)
        for s_ in range(TB):
            c_ = synth.clean_image(TH, TW, 20000 + s_ + 1000 * rank)
            cl[s_, :, :TW] = torch.from_numpy((c_ * 4.0).astype(np.float32)).to(dev)
            nz[s_, :, :TW] = torch.from_numpy(synth.poisson_observation(c_, 4.0, 21000 + s_ + 1000 * rank)
                                              .astype(np.float32)).to(dev)
        dkg = torch.empty((48, 49), dtype=torch.float32, device=dev)
        dag = torch.empty((48,), dtype=torch.float32, device=dev)
        topts = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_FP32, iters=TT)
        F.foe_train_step(ctx, cl, nz, TB, TH, TW, tld, topts, dkg, dag, 0, stream=stream)  # warm-up
        torch.cuda.synchronize()
        tt = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tloss = F.foe_train_step(ctx, cl, nz, TB, TH, TW, tld, topts, dkg, dag, 0, stream=stream)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1))
        train = {"images": TB, "H": TH, "W": TW, "iters": TT, "checkpoint_every": 7, "ms_per_step": float(np.median(tt)),
                 "loss": tloss, "grad_norm": float(torch.linalg.vector_norm(dkg)),
                 "unrolled_mpix_iter_per_s": TB * TH * TW * TT / (float(np.median(tt)) / 1e3) / 1e6,
                 "precision": "fp32 forward, recompute and backward"}
        # the paper's own gradient (implicit differentiation at u^T, conjugate gradients to 1e-5) on the same batch
        dki = torch.zeros_like(dkg)
        dai = torch.zeros_like(dag)
        F.foe_train_grad_implicit(ctx, cl, nz, TB, TH, TW, tld, topts, dki, dai, 200, 1e-5, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iloss, irep = F.foe_train_grad_implicit(ctx, cl, nz, TB, TH, TW, tld, topts, dki, dai, 200, 1e-5, stream=stream)
        e1.record(stream)
        e1.synchronize()
        train["implicit"] = {"ms_per_step": e0.elapsed_time(e1), "cg_iters": irep["cg_iters"],
                             "cg_relres": irep["cg_relres"], "breakdowns": irep["breakdowns"],
                             "grad_norm": float(torch.linalg.vector_norm(dki))}
        # the same with the CG's Hessian-vector products on TF32 tensor cores
        dkt = torch.zeros_like(dkg)
        dat = torch.zeros_like(dag)
        topts_tc = F.SolveOpts(model=F.FOE_MODEL_ANS_L2, prec=F.FOE_PREC_TF32, iters=TT)
        F.foe_train_grad_implicit(ctx, cl, nz, TB, TH, TW, tld, topts_tc, dkt, dat, 200, 1e-5, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, trep = F.foe_train_grad_implicit(ctx, cl, nz, TB, TH, TW, tld, topts_tc, dkt, dat, 200, 1e-5, stream=stream)
        e1.record(stream)
        e1.synchronize()
        train["implicit_tf32_hvp"] = {
            "ms_per_step": e0.elapsed_time(e1), "cg_iters": trep["cg_iters"], "cg_relres": trep["cg_relres"],
            "grad_rel_diff_vs_fp32": float(torch.linalg.vector_norm(dkt - dki) / torch.linalg.vector_norm(dki))}
        del cl, nz

    # serving leg: continuous batching under a 40 GB budget vs the plain per-request paths
    serve = None
    if args.serve_requests > 0:
        pool = serving_pool(rank)
        serve = run_serving(F, ctx, pool, args.serve_requests, 200.0, prec_main, 40 << 30, 10, True)
        if args.serve_baseline_requests > 0:
            nb = args.serve_baseline_requests
            serve["per_request_fp32_prefix"] = run_serving(F, ctx, pool, nb, 200.0, F.FOE_PREC_FP32, 0, 0, False, True)
            serve["per_request_bf16_prefix"] = run_serving(F, ctx, pool, nb, 200.0, prec_main, 0, 0, False, True)
            serve["batched_prefix"] = run_serving(F, ctx, pool, nb, 200.0, prec_main, 40 << 30, 10, True)
        # the same request mix offered at half the rate (about half the server's capacity): latency without queueing
        serve["half_rate"] = run_serving(F, ctx, pool, args.serve_requests // 2, 100.0, prec_main, 40 << 30, 10, True)
        del pool

    F.foe_destroy(ctx)
    per_step_launches = 10 + ITERS + 10
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MPix·iter/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded images, DCT-7 filter bank)",
                "config": {"workload": CONFIG_NAME, "images_per_step": 10, "H": H, "W": W, "iters": ITERS,
                           "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
                "fp32_plain": fp32, "tf32_tensor_core": tf32, "single_image_ms": float(np.median(lat)),
                "backtrack": backtrack, "binned": binned, "accuracy": accuracy, "stopping_rule": stopping,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "batched_uneven_graph": batched, "train": train, "serve": serve,
                "gpu_launches": per_step_launches * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
