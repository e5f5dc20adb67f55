"""Benchmark of the fused B-mode chain on one B300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the 2D full pipeline -- 128-element linear array, 256 scanlines,
2048 int16 samples per channel, DAS -> IQ envelope -> 60 dB log compression ->
scan conversion to 512x512 -- on a batch of 64 seeded synthetic phantom frames
per step (one batched launch per stage).  A step reads 64 x 128 MiB of channel
data, far larger than L2, so no flush is needed between steps.  Steps go
round-robin to two CUDA streams with their own output buffers, as the request
loop spreads batches over its streams; the same steps on one stream are timed
beside them.

Metric: beamformed samples*channels per second (n_tx * n_el * n_samples per
frame, all frames of all ranks) with frames/s and the p50/p99 step latency
(frames of a batch complete together).  One JSON line on rank 0.

--impl reference times the FP64 CPU oracle of the same chain (the only
reference this repository has) on the host cores, one full frame per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "beamformed samples·channels/s and frames/s (2D and 3D); p50/p99 frame latency"
UNIT = "samples*channels/s"
BATCH = 64          # frames per step of the workload; --frames changes it for small profiling runs only
SEED0 = 1000


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over the ranks (the job's time is its slowest
    rank's); x itself with one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (replicas: each rank does the same work)."""
    return units_per_rank * world / seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """Samples SM clock and throttle reasons through NVML while active."""

    REASONS = {
        "gpu_idle": 0x1, "applications_clocks_setting": 0x2, "sw_power_cap": 0x4, "hw_slowdown": 0x8,
        "sync_boost": 0x10, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
        "hw_power_brake_slowdown": 0x80, "display_clock_setting": 0x100,
    }

    def __init__(self, device_index=0, period=0.005):
        self.period = period
        self.index = device_index
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self.ok = False
        try:
            import pynvml

            pynvml.nvmlInit()
            import torch

            handle = None
            try:
                props = torch.cuda.get_device_properties(device_index)
                bus = "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
                handle = pynvml.nvmlDeviceGetHandleByPciBusId(bus.encode())
            except Exception:
                handle = pynvml.nvmlDeviceGetHandleByIndex(device_index)
            self.nv = pynvml
            self.h = handle
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(handle, pynvml.NVML_CLOCK_SM)
            self.ok = True
        except Exception as e:  # no NVML: fall back to nvidia-smi
            self.err = repr(e)

    def _run(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nv.nvmlDeviceGetClockInfo(self.h, self.nv.NVML_CLOCK_SM))
                self.reasons |= int(self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h))
            except Exception:
                pass
            time.sleep(self.period)

    SMI_FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __enter__(self):
        self._stop = threading.Event()
        if self.ok:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        else:
            import subprocess

            # nvidia-smi needs ~0.1 s to start: wait for its first sample, then
            # keep only the samples taken while the timed region runs
            self._rows = []
            first = threading.Event()
            try:
                self._smi = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.SMI_FIELDS}",
                                              "--format=csv,noheader,nounits", "-lms", "50", "-i", str(self.index)],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
            except OSError as e:
                self._smi, self.err = None, repr(e)
                return self

            def reader():
                for row in self._smi.stdout:
                    self._rows.append((time.perf_counter(), row))
                    first.set()

            self._reader = threading.Thread(target=reader, daemon=True)
            self._reader.start()
            first.wait(10.0)
        self._t_start = time.perf_counter()
        return self

    def __exit__(self, *a):
        self._t_end = time.perf_counter()
        self._stop.set()
        if self.ok:
            self._t.join()
        elif getattr(self, "_smi", None) is not None:
            time.sleep(0.06)   # the sample that covers the end of the region
            self._smi.terminate()
            self._smi.wait()
            self._reader.join(2.0)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            seen = set()
            rows = [r for t, r in self._rows if self._t_start <= t <= self._t_end + 0.06]
            for row in rows:
                f = [x.strip() for x in row.split(",")]
                try:
                    self.samples.append(float(f[0]))
                    self.max_mhz = float(f[1])
                except (ValueError, IndexError):
                    continue
                for n, v in zip(names, f[2:]):
                    if v.lower() == "active":
                        seen.add(n)
            self.smi_reasons = sorted(seen)

    def summary(self):
        src = "nvml" if self.ok else "nvidia-smi"
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "source": src,
                    "note": getattr(self, "err", "")}
        extra = {} if self.ok else {"nvml_unavailable": getattr(self, "err", "")}
        if self.ok:
            names = [k for k, v in self.REASONS.items() if self.reasons & v and k != "gpu_idle"]
        else:
            names = getattr(self, "smi_reasons", [])
        return {"sm_mhz": float(statistics.median(self.samples)), "sm_max_mhz": self.max_mhz, "reasons": names,
                "samples": len(self.samples), "source": src, **extra}


def kernel_source_hash():
    """Hash of the beamforming kernel's source and the library's compiler flags."""
    from paper_1711_06127_b300 import build

    src = os.path.join(ROOT, "paper_1711_06127_b300", "csrc", "das_kernel.cuh")
    return hashlib.sha256(open(src, "rb").read() + " ".join(build.CFLAGS).encode()).hexdigest()[:16]


def kernel_traffic():
    """DRAM traffic per launch of the beamforming kernel from the committed ncu
    summary, only if it was taken on the current kernel source and flags."""
    path = os.path.join(ROOT, "profiles", "das_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    h = kernel_source_hash()
    if rec.get("source_sha256_16") != h:
        return None
    return rec.get("bytes_per_launch_full_workload")


def workload():
    import phantom

    s = phantom.config2()
    return s


def cpu_oracle_rate(s, chs_host, budget_s=12.0, max_frames=None):
    """Times the FP64 oracle's whole chain on whole frames until budget_s."""
    import oracle

    p = s.params()
    per_frame = s.n_tx * s.n_el * s.n_samples
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.bmode(p, chs_host[done % len(chs_host)])
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_frames and done >= max_frames):
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def das_rate(fn, budget):
        n, t1 = 0, time.perf_counter()
        while True:
            fn(p, chs_host[n % len(chs_host)])
            n += 1
            e = time.perf_counter() - t1
            if e >= budget:
                return per_frame * n / e, n, e

    # beside the chain: the beamforming node alone, the FP64 oracle loops and the same loops in FP32
    r64, n64, e64 = das_rate(oracle.das, budget_s / 4)
    r32, n32, e32 = das_rate(oracle.das_f32, budget_s / 4)
    return {"value": per_frame * done / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{done} whole frame(s) of the 128-element/256-line/2048-sample workload through the "
                      f"FP64 oracle chain (DAS in C/OpenMP, envelope/log/scan conversion in numpy), {el:.1f} s",
            "das_only": {"fp64": {"value": r64, "unit": UNIT, "frames": n64, "seconds": e64},
                         "fp32": {"value": r32, "unit": UNIT, "frames": n32, "seconds": e32},
                         "note": "receive delay-and-sum alone on whole frames, same C/OpenMP loops in FP64 "
                                 "(the oracle) and FP32 (a timing reference, not an oracle)"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import phantom
    import torch

    s = workload()
    chs = [phantom.synth_channels(s, phantom.default_phantom(s, SEED0), SEED0).numpy()]
    import oracle

    p = s.params()
    for _ in range(args.warmup):
        oracle.bmode(p, chs[0])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.bmode(p, chs[0])
        times.append(time.perf_counter() - t0)
    per_frame = s.n_tx * s.n_el * s.n_samples
    total = sum(times)
    value = per_frame * len(times) / total
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": s.name, "frames_per_step": 1, "note": "one whole frame per step on the host cores"},
        "frames_per_s": len(times) / total,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "one whole frame per step of the same workload through the FP64 oracle chain"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _percentiles(xs):
    srt = sorted(xs)
    if not srt:
        return None, None
    pick = lambda q: srt[min(len(srt) - 1, int(round(q * (len(srt) - 1))))]
    return pick(0.5), pick(0.99)


def bench_table1(args, dev, stream):
    """The 2D configurations of the run-time table (64 channels, "n_tx / lines
    per transmit" 64/1, 64/2, 128/1, 128/2; 45 mm; 0.0225 mm isotropic output):
    per-node device time of the unfused chain (one launch per node, as the
    paper times its nodes) and of the fused chain, single frames, each timed over
    calls queued back to back on the device."""
    import torch

    import paper_1711_06127_b300 as supra
    import phantom

    out = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps=20):
        # These kernels take microseconds, less than the host needs to issue one call: the
        # timed calls are queued behind a ~2 ms device-side wait (torch's sleep kernel, before
        # the first event), so that the events measure the device running them back to back
        # rather than the host's launch rate.
        for _ in range(3):
            fn()
        sleep = getattr(torch.cuda, "_sleep", None)   # (without it: host-paced timing)
        if sleep is not None:
            with torch.cuda.stream(stream):
                sleep(4_000_000)
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    for n_tx, k in ((64, 1), (64, 2), (128, 1), (128, 2)):
        st = phantom.table1_setup(n_tx, k)
        plan = supra.Plan(**st.params())
        ch = phantom.synth_channels(st, phantom.make_phantom(st, 7000 + n_tx + k, 3000, n_points=5), 7000 + n_tx + k,
                                    device=dev)
        rf = plan.beamform(ch, stream=stream)
        env = plan.envelope(rf, stream=stream)
        bm = plan.logcompress(env, stream=stream)
        img = plan.scanconvert(bm, stream=stream)
        ws = torch.empty(max(1, supra.workspace_size([plan])), dtype=torch.uint8, device=dev)

        def chains():
            # the workspace for the plan's tile shape in effect (depth-segment boundary records)
            ws = torch.empty(max(1, supra.workspace_size([plan])), dtype=torch.uint8, device=dev)
            nodes = {"beamformer": timed(lambda: plan.beamform(ch, rf, stream)),
                     "envelope": timed(lambda: plan.envelope(rf, env, stream)),
                     "log_compression": timed(lambda: plan.logcompress(env, bm, stream)),
                     "scan_conversion": timed(lambda: plan.scanconvert(bm, img, stream))}
            fused = timed(lambda: plan.bmode(ch, img, ws, stream))
            return {"node_ms": nodes, "unfused_total_ms": sum(nodes.values()), "fused_ms": fused,
                    "fused_frames_per_s": 1e3 / fused}

        # default tile shape, then the shape the autotuner picks for the fused chain (depth
        # segments and resident CTAs of one-frame launches), which the beamforming node uses too
        default = chains()
        shape, tuned = None, None
        if not args.no_tune:
            shape, _, _ = plan.autotune_shape([ch], [img], ws, reps=10, stream=stream)
            tuned = chains()
        out.append({"config": f"{n_tx}/{k}", "workload": st.name, "n_lines": st.n_lines, "n_samples": st.n_samples,
                    "grid": "x".join(str(v) for v in plan.out_shape[::-1]), **(tuned or default),
                    "tile_shape": shape, "default_shape": default})
    return out


def bench_planewave(args, dev, stream):
    """Plane-wave imaging with coherent compounding: 11 plane waves at -10..10
    degrees per frame, 128 elements, 256 lines, 2048 samples, 512 x 512 output;
    64 frames per fused batched call (370 MB of records, larger than L2)."""
    import numpy as np
    import torch

    import paper_1711_06127_b300 as supra
    import phantom

    st = phantom.planewave_setup(128, 0.3e-3, 256, 2048, angles_deg=tuple(np.linspace(-10, 10, 11)), fc=7e6,
                                 fs=40e6, grid_n=(512, 512), name="planewave-128el-11angles-256lines-2048s-sc512")
    plan = supra.Plan(**st.params())
    nb = 64
    batch = torch.empty((nb, *plan.ch_shape), dtype=torch.int16, device=dev)
    for k in range(nb):
        batch[k].copy_(phantom.synth_channels(st, phantom.make_phantom(st, 8000 + k, 4000, n_points=3), 8000 + k,
                                              device=dev))
    chs = list(batch)
    outs = [torch.empty(plan.out_shape, dtype=torch.uint8, device=dev) for _ in range(nb)]
    ws = torch.empty(max(1, supra.workspace_size([plan] * nb)), dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(3):
        supra.bmode_batched([plan] * nb, chs, outs, ws, stream)
    reps = 10
    ev[0].record(stream)
    for _ in range(reps):
        supra.bmode_batched([plan] * nb, chs, outs, ws, stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    info = plan.info
    alg = nb * (info["aperture_bytes"] + info["image_bytes"])
    return {"workload": st.name, "angles": st.n_tx, "frames_per_call": nb, "ms_per_call": ms,
            "frames_per_s": nb / (ms * 1e-3),
            "samples_channels_per_s": nb * info["n_tx"] * info["n_el"] * info["n_samples"] / (ms * 1e-3),
            "aperture_gb_per_s": alg / (ms * 1e-3) / 1e9,
            "note": "each line reads its aperture from all 11 transmits' records (L2-resident per frame); "
                    "aperture bytes count every (transmit, element, depth) sample"}


def bench_compounding(args, dev, stream, s, ch):
    """Frequency compounding (a bank of 3 IQ demodulators at fc, fc +- fc/4)
    on one frame of the main workload: the envelope node with 1 and 3 bands,
    and the whole chain per frame (fused for one band; beamform -> banked
    envelope -> log compression -> scan conversion for three)."""
    import dataclasses

    import torch

    import paper_1711_06127_b300 as supra

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    res = {}
    for K in (1, 3):
        st = dataclasses.replace(s, n_bands=K, band_step=s.fc / 4 if K > 1 else 0.0)
        plan = supra.Plan(**st.params())
        rf = plan.beamform(ch, stream=stream)
        env = plan.envelope(rf, stream=stream)
        img = torch.empty(plan.out_shape, dtype=torch.uint8, device=dev)
        ws = torch.empty(max(1, supra.workspace_size([plan])), dtype=torch.uint8, device=dev)
        res[f"bands_{K}"] = {"envelope_node_ms": timed(lambda: plan.envelope(rf, env, stream)),
                             "chain_ms_per_frame": timed(lambda: plan.bmode(ch, img, ws, stream)),
                             "chain": "fused" if K == 1 else "unfused (beamform, banked envelope, log, scan conversion)"}
    res["workload"] = s.name
    return res


def bench_apod(args, dev, stream):
    """Learned apodization on 128 elements x 256 lines x 2048 samples: train on
    seeded frames labelled by the exact MV beamformer, then report DAS, MV and
    the learned form side by side on held-out frames (frames/s, per-frame
    latency, PSNR of the B-mode lines against MV, cyst contrast and CNR)."""
    import torch

    import paper_1711_06127_b300 as supra
    from paper_1711_06127_b300 import apod, quality
    import phantom

    s = phantom.config2()
    p = dict(s.params(), grid=None)
    plan = supra.Plan(**p)
    L = 32
    n_train, n_eval = args.apod_train_frames, args.apod_eval_frames
    P = plan.n_lines * plan.n_depth
    feat = torch.empty((n_train * P, supra.APOD_INPUTS), dtype=torch.bfloat16, device=dev)
    mask = torch.empty((n_train * P, 4), dtype=torch.int32, device=dev)
    norm = torch.empty((n_train * P,), dtype=torch.float32, device=dev)
    label = torch.empty((n_train * P,), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    for f in range(n_train):
        ch, _ = phantom.apod_frame(s, 4000 + f, device=dev)
        sl = slice(f * P, (f + 1) * P)
        plan.apod_features(ch, feat[sl], mask[sl], norm[sl], stream)
        plan.mv(ch, L, rf=label[sl].view(plan.line_shape), stream=stream)
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    data = apod.Dataset(feat, mask, norm, label)
    tr = apod.Trainer(phantom.apod_init(7), lr=args.apod_lr)
    # minibatches of interleaved blocks of 128 consecutive rows (each gradient tile reads one contiguous
    # block), at most eight 128-pixel tiles per SM (0 = that size): the gradient kernel runs one
    # CTA per SM and pays a fixed cost per step (weight staging, tensor-memory allocation, partial
    # gradients, the reduction and Adam launch) of about two and a half tiles, so a minibatch is a
    # whole number of tile rounds and several of them long
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    batch_rows = args.apod_batch if args.apod_batch > 0 else 8 * 128 * sms
    n_batches = max(1, -(-data.n // batch_rows))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    losses = []
    e0.record(stream)
    for ep in range(args.apod_epochs):
        losses.append(tr.epoch(data, n_batches, seed=ep, stream=stream, chunk=128))
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    pix = data.n * args.apod_epochs
    flops_per_pixel = 2 * (128 * 64 + 64 * 64 + 64 * 128) + 2 * (128 * 64 + 64 * 64 + 128 * 64 + 64 * 64 + 64 * 128)
    del feat, mask, norm, label, data
    torch.cuda.empty_cache()

    # ---- held-out frames: the three beamformers, each followed by envelope + log compression
    def chain(kind, ch, out):
        if kind == "das":
            return plan.bmode(ch, out, None, stream)
        rf = plan.mv(ch, L, stream=stream) if kind == "mv" else plan.apod(ch, tr.params, stream=stream)
        return plan.logcompress(plan.envelope(rf, stream=stream), out, stream=stream)

    def rf_of(kind, ch):
        if kind == "das":
            return plan.beamform(ch, stream=stream)
        return plan.mv(ch, L, stream=stream) if kind == "mv" else plan.apod(ch, tr.params, stream=stream)

    kinds = ("das", "mv", "apod")
    lat = {k: [] for k in kinds}
    q = {k: {"psnr_vs_mv": [], "contrast_db": [], "cnr": [], "fwhm_lat_mm": [], "fwhm_ax_mm": []} for k in kinds}
    # the three point targets of each frame: on the central axis at 0.25, 0.575, 0.9 of the imaged depth
    import numpy as np

    xs = np.asarray(p["line_origin"])[:, 0]
    zmax = p["depth0"] + (p["n_depth"] - 1) * p["depth_step"]
    targets = [(int(np.argmin(np.abs(xs))), int(round((f * zmax - p["depth0"]) / p["depth_step"])))
               for f in np.linspace(0.25, 0.9, 3)]
    out = torch.empty(plan.line_shape, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for f in range(n_eval):
        ch, cysts = phantom.apod_frame(s, 5000 + f, device=dev)
        for k in kinds:
            chain(k, ch, out)   # warm
            ev[0].record(stream)
            chain(k, ch, out)
            ev[1].record(stream)
            torch.cuda.synchronize()
            lat[k].append(ev[0].elapsed_time(ev[1]))
        bms, envs = {}, {}
        for k in kinds:
            rf = rf_of(k, ch)
            env = plan.envelope(rf, stream=stream)
            envs[k] = env.cpu().numpy()
            bms[k] = plan.logcompress(env, stream=stream).cpu().numpy()
        for k in kinds:
            q[k]["psnr_vs_mv"].append(quality.psnr(bms[k], bms["mv"]))
            for cy in cysts:
                st = quality.cyst_stats(p, envs[k], bms[k], cy, float(p.get("dyn_range_db", 60.0)))
                q[k]["contrast_db"].append(st["contrast_db"])
                q[k]["cnr"].append(st["cnr"])
            for tl, ti in targets:
                w = quality.point_fwhm(p, envs[k], tl, ti)
                q[k]["fwhm_lat_mm"].append(1e3 * w["lateral_m"])
                q[k]["fwhm_ax_mm"].append(1e3 * w["axial_m"])
    res = {"workload": s.name + "-mv-labels", "subaperture": L, "loading": 0.01,
           "train": {"frames": n_train, "pixels": P * n_train, "epochs": args.apod_epochs,
                     "minibatch_pixels": P * n_train // n_batches, "lr": args.apod_lr, "loss_first_epoch": losses[0],
                     "loss_last_epoch": losses[-1], "ms": train_ms, "pixels_per_s": pix / (train_ms * 1e-3),
                     "tflops": pix * flops_per_pixel / (train_ms * 1e-3) / 1e12, "data_prep_s": prep_s},
           "eval_frames": n_eval}
    for k in kinds:
        p50, p99 = _percentiles(lat[k])
        mean_ms = sum(lat[k]) / len(lat[k])
        name = {"das": "das", "mv": "mv", "apod": "learned"}[k]
        psnr = [v for v in q[k]["psnr_vs_mv"] if v != float("inf")]
        res[name] = {"frames_per_s": 1e3 / mean_ms, "latency_ms": {"p50": p50, "p99": p99},
                     "psnr_vs_mv_db": (sum(psnr) / len(psnr)) if psnr else None,
                     "cyst_contrast_db": sum(q[k]["contrast_db"]) / len(q[k]["contrast_db"]),
                     "cyst_cnr": sum(q[k]["cnr"]) / len(q[k]["cnr"]),
                     "point_fwhm_mm": {"lateral": float(np.median(q[k]["fwhm_lat_mm"])),
                                       "axial": float(np.median(q[k]["fwhm_ax_mm"]))}}
    res["note"] = ("single-frame launches, B-mode lines out (beamformer + envelope + log compression); "
                   "PSNR of 8-bit B-mode lines against MV's; cysts of each held-out frame; -6 dB widths of the "
                   "three axial point targets (median over frames and targets)")
    return res, tr.params


def bench_serving(args, dev, apod_params=None):
    """The request loop under open-loop Poisson streams: 2D frames of varied
    shapes and 3D volumes, each tagged DAS, learned apodization or MV (3D
    volumes run DAS), admitted by free device memory; frames/s and latency
    from scheduled arrival to completion on the device.  First the offered
    rate of the workload (2000 requests/s, beyond what one GPU completes: its
    latencies are backlog), then the same mix and seed at 80 % of the rate
    that run completed (a load the GPU carries: its latencies are service
    times), with the admission wait and the time from admission to
    completion reported apart."""
    import numpy as np
    import torch

    import paper_1711_06127_b300 as supra
    from paper_1711_06127_b300.serving import Server
    import phantom

    shapes2d = [(e, l, n) for e in (64, 96, 128) for l in (128, 192, 256) for n in (1024, 1536, 2048)]
    plans2d, pool2d = [], []
    for k, (e, l, n) in enumerate(shapes2d):
        st = phantom.linear_setup(e, 0.3e-3, l, n, fc=7e6, fs=40e6, grid_n=(512, 512), name=f"2d-{e}-{l}-{n}")
        plans2d.append(supra.Plan(**st.params()))
        pool2d.append(phantom.synth_channels(st, phantom.make_phantom(st, 6100 + k, 4000), 6100 + k, device=dev))
    plans3d, pool3d = [], []
    if not args.skip_3d:
        for k, lines in enumerate((32, 64)):
            st = phantom.config3(lines)
            plans3d.append(supra.Plan(**st.params()))
            pool3d.append(phantom.synth_channels(st, phantom.default_phantom(st, 6200 + k), 6200 + k, device=dev))
    if apod_params is None:
        apod_params = torch.as_tensor(phantom.apod_init(7)).to(dev)

    def run(n, rate):
        rng = np.random.default_rng(6000)
        t_arr = np.cumsum(rng.exponential(1.0 / rate, n))
        reqs, meta = [], []
        for i in range(n):
            is3d = bool(plans3d) and rng.random() < 0.3
            tag = ("das", "apod", "mv")[int(rng.integers(0, 3))]
            if is3d:
                k = int(rng.integers(0, len(plans3d)))
                plan, ch, kind = plans3d[k], pool3d[k], "das"
            else:
                k = int(rng.integers(0, len(plans2d)))
                plan, ch, kind = plans2d[k], pool2d[k], tag
            kw = dict(ch=ch, tag=i)
            if kind == "apod":
                kw["apod_params"] = apod_params
            elif kind == "mv":
                kw.update(mv_subaperture=32, mv_loading=0.01)
            reqs.append((kind, plan, kw))
            meta.append(("3d" if is3d else "2d", kind))
        srv = Server(int(args.serve_memory_gb * (1 << 30)), n_streams=4, max_batch=16, use_graphs=True)
        torch.cuda.synchronize()
        srv.submit_trace(reqs, t_arr)
        done = []
        deadline = time.perf_counter() + args.serve_timeout
        while len(done) < n and time.perf_counter() < deadline:
            got = srv.poll()
            for c in got:
                if c["out"] is not None:
                    srv.release(c["ticket"])
            done += got
            if not got:
                time.sleep(0.0005)
        st = srv.stats()
        srv.close()
        ok = [c for c in done if c["status"] == 0]
        res = {"requests": n, "completed": len(ok), "errors": len(done) - len(ok), "offered_rate_per_s": rate,
               "memory_gb": args.serve_memory_gb, "streams": 4, "max_batch": 16, "graphs": True}
        if ok:
            span = max(c["t_done"] for c in ok) - min(c["t_submit"] for c in ok)
            lat = [1e3 * (c["t_done"] - c["t_submit"]) for c in ok]
            p50, p99 = _percentiles(lat)
            res.update({"span_s": span, "frames_per_s": len(ok) / span,
                        "frames_2d_per_s": sum(1 for c in ok if meta[c["tag"]][0] == "2d") / span,
                        "volumes_3d_per_s": sum(1 for c in ok if meta[c["tag"]][0] == "3d") / span,
                        "latency_ms": {"p50": p50, "p99": p99}})
            by = {}
            for c in ok:
                by.setdefault("-".join(meta[c["tag"]]), []).append(c)

            def pcts(cs, f):
                a, b = _percentiles([1e3 * f(c) for c in cs])
                return {"p50": a, "p99": b}

            res["latency_ms_by_class"] = {
                k: dict(pcts(v, lambda c: c["t_done"] - c["t_submit"]), n=len(v),
                        admission_wait=pcts(v, lambda c: c["t_admit"] - c["t_submit"]),
                        admitted_to_done=pcts(v, lambda c: c["t_done"] - c["t_admit"]))
                for k, v in sorted(by.items())}
            res["admission_wait_ms"] = pcts(ok, lambda c: c["t_admit"] - c["t_submit"])
            res["admitted_to_done_ms"] = pcts(ok, lambda c: c["t_done"] - c["t_admit"])
            res["mean_batch"] = sum(c["batch_size"] for c in ok) / len(ok)
        res["stats"] = {k: st[k] for k in ("batches", "graph_launches", "graph_instantiations", "graph_updates",
                                           "memory_peak")}
        return res

    res = run(args.serve_requests, args.serve_rate)
    res["mix"] = ("70% 2D (27 shapes: 64/96/128 el x 128/192/256 lines x 1024/1536/2048 samples, 512x512 out), "
                  "30% 3D (1024 el, 32x32 or 64x64 lines, 1536 samples, 256^3 out); tags DAS / learned / MV "
                  "uniform, 3D runs DAS")
    if res.get("frames_per_s") and args.serve_sustain_requests > 0:
        rate = 0.8 * res["frames_per_s"]
        sus = run(args.serve_sustain_requests, rate)
        sus["note"] = ("the same mix and seed offered at 80 % of the rate the run above completed: latency from "
                       "scheduled arrival to completion on the device, split into the wait for memory admission "
                       "and the time from admission to completion")
        res["sustainable"] = sus
    return res


def run_ours(args):
    import torch

    global BATCH
    BATCH = args.frames
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1711_06127_b300 import build

    build.build()
    import paper_1711_06127_b300 as supra
    import phantom

    s = workload()
    p = s.params()
    plan = supra.Plan(**p)
    p_lines = dict(p, grid=None)
    plan_lines = supra.Plan(**p_lines)          # same beamforming kernel, log-compressed lines out
    info = plan.info
    # synthetic frames: distinct seeds per rank
    seeds = [SEED0 + rank * BATCH + k for k in range(BATCH)]
    # one allocation for the batch: frames at a uniform stride, as an acquisition ring buffer holds them
    batch = torch.empty((BATCH, *plan.ch_shape), dtype=torch.int16, device=dev)
    for k, sd in enumerate(seeds):
        batch[k].copy_(phantom.synth_channels(s, phantom.default_phantom(s, sd), sd, device=dev))
    chs = list(batch)
    # Steps go round-robin to two streams, as the request loop spreads its batches over its
    # streams, each stream with its own output buffers and workspace: the last CTAs of one
    # batch's launch then share the GPU with the first CTAs of the next instead of leaving
    # SMs idle.
    n_str = 2
    streams = [torch.cuda.current_stream()] + [torch.cuda.Stream(dev) for _ in range(n_str - 1)]
    stream = streams[0]
    outs_s = [[torch.empty(plan.out_shape, dtype=torch.uint8, device=dev) for _ in range(BATCH)]
              for _ in range(n_str)]
    outs = outs_s[0]
    lines_s = [[torch.empty(plan.line_shape, dtype=torch.uint8, device=dev) for _ in range(BATCH)]
               for _ in range(n_str)]
    ws_s = [torch.empty(max(1, supra.workspace_size([plan] * BATCH)), dtype=torch.uint8, device=dev)
            for _ in range(n_str)]
    ws = ws_s[0]
    plans = [plan] * BATCH

    def step(k, ns):
        j = k % ns
        supra.bmode_batched(plans, chs, outs_s[j], ws_s[j], streams[j])

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    def timed(fn, n, ns, clocks=False, warm=0):
        """n calls fn(k, ns), call k on stream k % ns.  Returns the total ms, each call's ms
        (from the point its stream reached it to its end) and the clock sampler.  The clock
        sampler starts first (it takes a moment to start); `warm` untimed calls queued after it
        keep the GPU busy up to the timed region, which a barrier and a synchronize open."""
        es = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(dev.index) if clocks else None
        if clk:
            clk.__enter__()
        for k in range(warm):
            fn(k, ns)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for st in streams[1:ns]:
            st.wait_stream(stream)
        for k in range(n):
            es[k].record(streams[k % ns])
            fn(k, ns)
            ee[k].record(streams[k % ns])
        for st in streams[1:ns]:
            stream.wait_stream(st)
        e1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        barrier()
        return e0.elapsed_time(e1), [es[k].elapsed_time(ee[k]) for k in range(n)], clk

    # tile shape of the workload from the project's autotuner (frames per group, staging-ring
    # shape, depth segments, CTAs per SM), kept in both plans
    tune = None
    if not args.no_tune:
        shape, tuned_ms, start_ms = plan.autotune_shape(chs, outs_s[0], ws_s[0], reps=5, stream=stream)
        plan_lines.tile_shape = shape
        tune = {"shape": shape, "ms_per_call": tuned_ms, "default_shape_ms_per_call": start_ms,
                "gain": start_ms / tuned_ms, "reps": 5,
                "note": "supra_autotune_tile_shape on the step's 64 frames; the timed steps use the picked shape"}
    for k in range(max(3, args.warmup)):
        step(k, n_str)
    torch.cuda.synchronize()
    assert supra.device_status() == 0

    # ---- timed region: exactly K steps (the W warm-up steps again right before it, untimed, so
    # that the GPU does not sit idle while the clock sampler starts)
    total_ms, step_ms, clk = timed(step, args.steps, n_str, clocks=True, warm=max(3, args.warmup))
    total_ms = max_over_ranks(total_ms, world, dev)
    per_frame = s.n_tx * s.n_el * s.n_samples
    frames = BATCH * args.steps * world
    value = job_rate(per_frame * BATCH * args.steps, world, total_ms * 1e-3)
    # the same steps one at a time on one stream: a batch's latency without a neighbour (at least
    # 100 steps, so that the figure does not rest on a handful of launches)
    n_one = max(args.steps, 100)
    one_ms, one_step_ms, _ = timed(step, n_one, 1)
    one_ms *= args.steps / n_one

    # ---- the dominant kernel alone: beamforming + envelope + log compression, same launch
    # shape, launches alternating over the two streams as above (and, beside it, on one stream)
    def das(k, ns):
        j = k % ns
        supra.bmode_batched([plan_lines] * BATCH, chs, lines_s[j], None, streams[j])

    for k in range(3):
        das(k, n_str)

    def kernel_leg(ns, budget_s, block=100, min_blocks=5):
        """Blocks of `block` launches until budget_s of launches and min_blocks blocks have
        run, whatever --steps is; the median block's ms per launch and the clocks seen."""
        per, t_end = [], time.perf_counter() + budget_s
        clk = ClockSampler(dev.index)
        clk.__enter__()
        while len(per) < min_blocks or time.perf_counter() < t_end:
            per.append(timed(das, block, ns)[0] / block)
        clk.__exit__(None, None, None)
        return float(statistics.median(per)), len(per) * block, clk.summary()

    das_ms, das_launches, das_clocks = kernel_leg(n_str, args.kernel_budget)
    das_ms_one, das_launches_one, _ = kernel_leg(1, args.kernel_budget / 2)
    alg_bytes = BATCH * (info["aperture_bytes"] + info["bmode_bytes"])
    peaks, peak_src = measured_peaks()
    achieved = alg_bytes / (das_ms * 1e-3) / 1e9
    ms_step = total_ms / args.steps
    if das_ms > ms_step:   # the step (this kernel + scan conversion) cannot be shorter: measure again
        das_ms, das_launches, das_clocks = kernel_leg(n_str, 2 * args.kernel_budget)
        achieved = alg_bytes / (das_ms * 1e-3) / 1e9

    # ---- the 3D workload: one 64x64-line pyramid volume (12 GiB of records) per launch
    vol3d = None
    if not args.skip_3d:
        s3 = phantom.config3()
        plan3 = supra.Plan(**s3.params())
        ch3 = phantom.synth_channels(s3, phantom.default_phantom(s3, 3000), 3000, device=dev)
        out3 = torch.empty(plan3.out_shape, dtype=torch.uint8, device=dev)
        ws3 = torch.empty(max(1, supra.workspace_size([plan3])), dtype=torch.uint8, device=dev)
        for _ in range(2):
            plan3.bmode(ch3, out3, ws3, stream)
        e3 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        n3 = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        e3[0].record(stream)
        for _ in range(n3):
            plan3.bmode(ch3, out3, ws3, stream)
        e3[1].record(stream)
        torch.cuda.synchronize()
        ms3 = e3[0].elapsed_time(e3[1]) / n3
        i3 = plan3.info
        # headless rendering of the volume: oblique orthographic MIP and emission-absorption, 512 x 512
        import numpy as np

        g3 = s3.grid
        ext = np.asarray(g3["spacing"]) * (np.asarray(g3["n"]) - 1)
        ctr = np.asarray(g3["origin"]) + ext / 2
        d = np.array([0.5, 0.3, 1.0])
        d /= np.linalg.norm(d)
        half = float(np.linalg.norm(ext)) / 2
        rt = np.cross(d, [0.0, 1.0, 0.0])
        rt = rt / np.linalg.norm(rt) * (2 * half / 512)
        dn = np.cross(d, rt)
        dn = dn / np.linalg.norm(dn) * (2 * half / 512)
        dt = float(min(g3["spacing"]))
        cam = {"centre": ctr - half * d, "right": rt, "down": dn, "dir": d, "t0": 0.0, "dt": dt,
               "n_steps": int(2 * half / dt)}
        rend = {}
        img = torch.empty((512, 512), dtype=torch.float32, device=dev)
        for mode in ("mip", "ea"):
            kw = dict(lo=64.0, hi=255.0, alpha=0.05) if mode == "ea" else {}
            supra.render(out3, g3, cam, 512, 512, mode, image=img, stream=stream, **kw)
            e3[0].record(stream)
            for _ in range(5):
                supra.render(out3, g3, cam, 512, 512, mode, image=img, stream=stream, **kw)
            e3[1].record(stream)
            torch.cuda.synchronize()
            ms = e3[0].elapsed_time(e3[1]) / 5
            rend[mode] = {"ms": ms, "samples_per_s": 512 * 512 * cam["n_steps"] / (ms * 1e-3)}
        rend["image"] = "512x512"
        rend["n_steps"] = cam["n_steps"]
        # sixteen volumes of the plan in one batched call (one allocation at a uniform stride: the
        # tensor-map staging path; delays and weights shared by the sixteen volumes)
        nb3 = 16
        batch3 = torch.empty((nb3, *plan3.ch_shape), dtype=torch.int16, device=dev)
        for k in range(nb3):
            batch3[k].copy_(ch3)
        outs3 = [torch.empty(plan3.out_shape, dtype=torch.uint8, device=dev) for _ in range(nb3)]
        ws3b = torch.empty(max(1, supra.workspace_size([plan3] * nb3)), dtype=torch.uint8, device=dev)
        supra.bmode_batched([plan3] * nb3, list(batch3), outs3, ws3b, stream)
        e3[0].record(stream)
        for _ in range(3):
            supra.bmode_batched([plan3] * nb3, list(batch3), outs3, ws3b, stream)
        e3[1].record(stream)
        torch.cuda.synchronize()
        ms3b = e3[0].elapsed_time(e3[1]) / 3
        i3b = plan3.info
        batched3 = {"volumes_per_call": nb3, "ms_per_call": ms3b, "volumes_per_s": nb3 * 1e3 / ms3b,
                    "aperture_gb_per_s": nb3 * (i3b["aperture_bytes"] + i3b["image_bytes"]) / (ms3b * 1e-3) / 1e9,
                    "frac_of_hbm_peak": nb3 * (i3b["aperture_bytes"] + i3b["image_bytes"]) / (ms3b * 1e-3) / 1e9
                    / measured_peaks()[0]["hbm_gbs"],
                    "note": "192 GiB of records per call; the sixteen volumes share each tile's delays and weights"}
        del batch3, outs3, ws3b
        vol3d = {"workload": s3.name, "ms_per_volume": ms3, "volumes_per_s": 1e3 / ms3, "render": rend,
                 "batched": batched3,
                 "samples_channels_per_s": i3["n_tx"] * i3["n_el"] * i3["n_samples"] / (ms3 * 1e-3),
                 "aperture_gb_per_s": (i3["aperture_bytes"] + i3["image_bytes"]) / (ms3 * 1e-3) / 1e9,
                 "frac_of_hbm_peak": (i3["aperture_bytes"] + i3["image_bytes"]) / (ms3 * 1e-3) / 1e9 / measured_peaks()[0]["hbm_gbs"],
                 "note": "one volume per launch (no frame batching), records resident"}
        del ch3, out3, ws3, plan3
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI from pinned host memory
    e2e_steps = 0 if args.skip_e2e else max(1, min(args.steps, args.e2e_steps))
    if e2e_steps:
        host_batch = torch.empty(batch.shape, dtype=torch.int16).pin_memory()
        host_batch.copy_(batch)
        host_out = torch.empty((BATCH, *plan.out_shape), dtype=torch.uint8).pin_memory()
        dev_batch = torch.empty_like(batch)
        dev_in = list(dev_batch)

    def e2e_step():
        dev_batch.copy_(host_batch, non_blocking=True)
        supra.bmode_batched(plans, dev_in, outs, ws, stream)
        for k, o in enumerate(outs):
            host_out[k].copy_(o, non_blocking=True)

    if e2e_steps:
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max(time.perf_counter() - t0, 1e-9)
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_value = job_rate(per_frame * BATCH * e2e_steps, world, e2e_s) if e2e_steps else None
    h2d = sum(c.numel() * c.element_size() for c in chs)
    d2h = sum(o.numel() for o in outs)
    assert supra.device_status() == 0

    # ---- the run-time table's 2D shapes (multi-line); learned apodization beside MV and DAS; the request loop
    table1 = bench_table1(args, dev, stream) if rank == 0 and not args.skip_table1 else None
    compounding = bench_compounding(args, dev, stream, s, chs[0]) if rank == 0 and not args.skip_table1 else None
    planewave = bench_planewave(args, dev, stream) if rank == 0 and not args.skip_table1 else None
    apod_res = serve_res = None
    if rank == 0 and not args.skip_apod:
        apod_res, trained = bench_apod(args, dev, stream)
    else:
        trained = None
    if rank == 0 and not args.skip_serve:
        serve_res = bench_serving(args, dev, trained)
    assert supra.device_status() == 0

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_oracle_rate(s, [batch[0].cpu().numpy()], budget_s=args.cpu_budget)
        def pct(v):
            srt = sorted(v)
            return srt[len(srt) // 2], srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]

        p50, p99 = pct(step_ms)
        p50_one, p99_one = pct(one_step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i16-in/f32", "data": "synthetic",
            "config": {"workload": s.name, "frames_per_step": BATCH, "n_el": s.n_el, "n_lines": s.n_lines,
                       "n_samples": s.n_samples, "grid": "512x512", "parallelism": f"replicas x{world}",
                       "l2": "inputs 8 GiB per step > L2, no flush"},
            "frames_per_s": frames / (total_ms * 1e-3),
            "latency_ms": {"p50": p50, "p99": p99,
                           "note": f"per step, from the point its stream reached it to its end, steps round-robin "
                                   f"over {n_str} streams (a step shares the GPU with its neighbours); the "
                                   f"{BATCH} frames of a step complete together"},
            "one_stream": {"ms_per_step": one_ms / args.steps, "latency_ms": {"p50": p50_one, "p99": p99_one},
                           "note": f"the same steps one after another on one stream ({n_one} of them)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": kernel_traffic(),
                         "kernel": f"das_kernel<{plan_lines.tile_shape['frames_per_group']},1> (beamform + envelope "
                                   f"+ log, {plan_lines.tile_shape['frames_per_group']} frames per CTA)",
                         "kernel_ms": das_ms,
                         "tile_shape": plan_lines.tile_shape,
                         "timing": f"median over blocks of 100 launches alternating over {n_str} streams (own "
                                   f"outputs each), {das_launches} launches in >= {args.kernel_budget} s",
                         "kernel_ms_le_step_ms": das_ms <= ms_step,
                         "frac_of_whole_step": alg_bytes / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "clocks": das_clocks,
                         "one_stream": {"kernel_ms": das_ms_one, "launches": das_launches_one,
                                        "frac": alg_bytes / (das_ms_one * 1e-3) / 1e9 / peaks["hbm_gbs"]},
                         "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peak_src},
            "autotune": tune,
            "full_array_gbs": BATCH * info["channel_bytes"] / (das_ms * 1e-3) / 1e9,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "volume_3d": vol3d,
            "table1_2d": table1,
            "envelope_compounding": compounding,
            "planewave_compounding": planewave,
            "learned_apodization": apod_res,
            "serving": serve_res,
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--kernel-budget", type=float, default=0.6,
                    help="seconds of launches of the dominant kernel alone for the roofline figure")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--frames", type=int, default=BATCH, help="frames per step (64 = the workload)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tile shape (no autotuner run)")
    ap.add_argument("--skip-3d", action="store_true")
    ap.add_argument("--skip-apod", action="store_true")
    ap.add_argument("--skip-table1", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--apod-train-frames", type=int, default=200)
    ap.add_argument("--apod-eval-frames", type=int, default=20)
    ap.add_argument("--apod-epochs", type=int, default=8)
    ap.add_argument("--apod-batch", type=int, default=0,
                    help="pixels per minibatch at most (0: eight 128-pixel tiles per SM, 151 552 on 148 SMs)")
    ap.add_argument("--apod-lr", type=float, default=1e-3)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-memory-gb", type=float, default=64.0)
    ap.add_argument("--serve-timeout", type=float, default=300.0)
    ap.add_argument("--serve-sustain-requests", type=int, default=3000,
                    help="requests of the second serving run, offered at 80 % of the first run's completed rate")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
