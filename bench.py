"""Benchmark of the separable width-5 convolution on GB300.

One step = one pass of the product path over one synthetic image: the fused
single-pass kernel on a 3 x 8192 x 8192 FP32 image (k = five seeded uniform
values normalised to sum 1), input and output resident in HBM.  The image
(805 MB in, 804 MB out) is far larger than the 129 MB L2, so no flush is
needed between steps.  Beside it, in the same run: the two-pass kernel pair
on the same image, the end-to-end offload call with host buffers
(sepconv5_run_host), the empty-launch overhead probe, and the FP64 CPU
oracle timed on a bounded sample (rank 0, one GPU only).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --case dtype=bf16,out=bf16,tile=128x128x2 --steps 5 --warmup 3

The second form times one configuration on its own and prints its JSON line
(the command the ncu summaries under profiles/ were taken with).

Multi-GPU (launched by torchrun): every rank convolves its own image (no
collective on the data path; weak scaling); the time is the max over ranks.
With --split rows the ranks share one image instead: each convolves a band
of its output rows, reading the band's 2-row halos from the source image, so
there is still no exchange (strong scaling).  The end-to-end offload leg
stays one whole image per rank in both modes.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import re
import shutil
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P, H, W = 3, 8192, 8192
SEED = 2
WORKLOAD = "3x8192x8192 f32 fused single-pass, k = 5 seeded uniform(0,1) taps / sum"
METRIC = "3-plane Mpix/s (fused single-pass, 3x8192x8192 FP32)"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "fused_f32_3x8192x8192.md")
# the files that define the fused kernel's code (template, device helpers, FP32 shapes)
FUSED_SOURCES = ["sc5_fused_impl.cuh", "sc5_device.cuh", "sc5_fused_f32.cu"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="only the timed fused leg")
    ap.add_argument("--serve-requests", type=int, default=10000, help="requests per offered load")
    ap.add_argument("--legs", default="c1,c3,c4,paper,pyramid,c5", help="extra configs to run beside the headline")
    ap.add_argument("--split", default="images", choices=["images", "rows"],
                    help="N > 1: every rank convolves its own image (weak scaling), or a band of rows of one "
                         "image with its halo read from the source (strong scaling)")
    ap.add_argument("--case", default=None,
                    help="time one configuration instead of the contract run (the command the ncu captures use): "
                         "comma-separated key=value with keys dtype, out, algo (fused|two_pass|direct|reduce), "
                         "layout (planar|hwc), planes, H, W, tile (THxTWxSTAGES), ctas, taps (kernel width), opitch "
                         "(output pitch in elements; 0: rows rounded to 16 bytes), batch (N > 0: the first N images "
                         "of the 256-image batch as one graph-replayed launch); --steps timed launches after --warmup")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers


def rank_image_seed(rank: int) -> int:
    """Every rank convolves its own image (weak scaling, no data exchange)."""
    return SEED + rank


def row_band(Hv: int, world: int, rank: int) -> tuple[int, int]:
    """Output rows [r0, r1) of a rank's band when the VALID rows of one image
    are split across ranks as evenly as possible.  The band reads input rows
    [r0, r1 + 4): its 2-row halos come from the source image, so bands need
    no exchange."""
    base, extra = divmod(Hv, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a per-rank time over all ranks (a no-op on one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, pixels_per_rank: int, ms_per_step: float) -> float:
    """3-plane Mpix/s of the whole job: all ranks' pixels over the slowest rank's time."""
    return world * pixels_per_rank / (ms_per_step / 1e3) / 1e6


def algorithmic_bytes(h: int, w: int, planes: int = P, es_in: int = 4, es_out: int = 4) -> int:
    """One read of every input pixel and one write of every VALID output pixel."""
    return planes * h * w * es_in + planes * (h - 4) * (w - 4) * es_out


FMA_PER_OUTPUT = 10  # the separable body: 5 multiply-adds per pass


def fma_peak() -> float:
    """FP32 multiply-adds per second of the GPU from its unit counts: 152 SMs x
    128 FP32 FMA per clock x the measured maximum SM clock (2.07 GHz)."""
    peaks = measured_peaks() or {}
    return 152 * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6


def measured_peaks() -> dict | None:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return None


def fused_source_hash() -> str:
    h = hashlib.sha256()
    for name in FUSED_SOURCES:
        with open(os.path.join(ROOT, "paper_1711_09791_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic() -> int | None:
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != fused_source_hash():
        return None
    return int(m_tr.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, each stamped with
    the host time at which it arrived.  start() returns once the first sample
    is in (or after a few seconds without one), so that sampling already runs
    when the warm-up begins; stop() reports the samples of the window that
    mark() opened and closed, plus the first sample after it, because a timed
    region of a few milliseconds can fall between two samples."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 10

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.t = None
        self.first = threading.Event()
        self.window = [None, None]

    def start(self, wait_s: float = 5.0):
        cmd = ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
               "-lms", str(self.PERIOD_MS)]
        # nvidia-smi block-buffers a pipe: line buffering makes each sample arrive (and be
        # time-stamped) when it is taken
        if shutil.which("stdbuf"):
            cmd = ["stdbuf", "-oL"] + cmd
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        self.first.wait(wait_s)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))
            self.first.set()

    def mark(self, which: int):
        """0: the window opens (before the warm-up); 1: it closes (after the timed steps)."""
        self.window[which] = time.perf_counter()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(3 * self.PERIOD_MS / 1e3)  # let the first sample after the window arrive
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        t0 = self.window[0] if self.window[0] is not None else float("-inf")
        t1 = self.window[1] if self.window[1] is not None else float("inf")
        inside = [ln for ts, ln in self.lines if t0 <= ts <= t1]
        after = [ln for ts, ln in self.lines if ts > t1][:1]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside + after:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        # median over the warm-up and timed steps (and the first sample after them)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_window": len(inside), "period_ms": self.PERIOD_MS,
                "window": "warm-up and timed steps of the headline and 0.25 s of the same launches right "
                          "after them (untimed), plus the next sample"}


# ------------------------------------------------------------------ CPU oracle leg


def oracle_sample(A: np.ndarray, k: np.ndarray, target_s: float = 10.0) -> dict:
    """Time the FP64 oracle (single thread, as it stands) on the top band of
    the image, sized to about target_s seconds; returns 3-plane Mpix/s."""
    import oracle
    k64 = k.astype(np.float64)
    # calibrate on a small band
    t0 = time.perf_counter()
    oracle.direct(A[:, :36, :].astype(np.float64), k64)
    per_row = (time.perf_counter() - t0) / 32.0
    rows = int(max(32, min(H - 4, target_s / max(per_row, 1e-9))))
    band = A[:, :rows + 4, :]
    t0 = time.perf_counter()
    oracle.direct(band.astype(np.float64), k64)
    dt = time.perf_counter() - t0
    px = rows * (W - 4)
    return {"value": px / dt / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": f"top {rows + 4} input rows x {W} cols x {P} planes of the image ({rows} x {W - 4} "
                      f"output pixels), FP64 direct Eq. 1, one thread, {dt:.1f} s"}


def cpu_two_pass_sample(A: np.ndarray, k: np.ndarray) -> dict:
    """The FP32 two-pass form with OpenMP on every host core (Listing 1's loop
    structure, horizontal pass over all rows) on the whole image: median of 5
    calls after a warm-up; 3-plane Mpix/s."""
    import cpu_baseline
    dt = cpu_baseline.time_two_pass(A, k, reps=5)
    return {"value": round(H * W / dt / 1e6, 1), "unit": "Mpix/s", "ms_per_image": round(dt * 1e3, 2),
            "cores": cpu_baseline.threads(), "nproc": os.cpu_count(), "cpu": cpu_baseline.cpu_model(),
            "kind": "fp32 two-pass, OpenMP", "flags": " ".join(cpu_baseline.FLAGS),
            "sample": f"the whole {P}x{H}x{W} image, median of 5 calls"}


def copy_probe(A_host, out_host, A_dev, out_dev, dev) -> dict:
    """Copy-only times for the offload bytes: host->device alone,
    device->host alone, and both at once on two streams (each the median of
    7 repetitions)."""
    import torch
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def t(fn, reps=7):
        # median of separately timed repetitions: one that meets a pause of
        # the GPU (tens of milliseconds, about every 2 s) does not move it
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            ts.append((time.perf_counter() - t0) * 1e3)
        return sorted(ts)[reps // 2]

    def h2d():
        with torch.cuda.stream(s1):
            A_dev.copy_(A_host, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            out_host.copy_(out_dev, non_blocking=True)

    def both():
        h2d()
        d2h()

    s3, s4 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ai, ad = A_host.view(-1), A_dev.view(-1)
    oh, od = out_host.view(-1), out_dev.view(-1)
    hi, ho = ai.numel() // 2, oh.numel() // 2

    def both_split():
        # each direction as two contiguous halves on two streams at once
        with torch.cuda.stream(s1):
            ad[:hi].copy_(ai[:hi], non_blocking=True)
        with torch.cuda.stream(s3):
            ad[hi:].copy_(ai[hi:], non_blocking=True)
        with torch.cuda.stream(s2):
            oh[:ho].copy_(od[:ho], non_blocking=True)
        with torch.cuda.stream(s4):
            oh[ho:].copy_(od[ho:], non_blocking=True)

    th, td, tb, ts = t(h2d), t(d2h), t(both), t(both_split)
    nb_in, nb_out = A_host.numel() * 4, out_host.numel() * 4
    return {"h2d_ms": round(th, 4), "d2h_ms": round(td, 4), "both_ms": round(tb, 4),
            "both_2streams_ms": round(ts, 4),
            "h2d_gbs": round(nb_in / th / 1e6, 1), "d2h_gbs": round(nb_out / td / 1e6, 1),
            "both_gbs": round((nb_in + nb_out) / tb / 1e6, 1),
            "both_2streams_gbs": round((nb_in + nb_out) / ts / 1e6, 1)}


def device_pauses(seconds: float = 6.0, ahead: int = 2000) -> dict:
    """Back-to-back device work with `ahead` launches (about 80 ms of work)
    queued in front of the host, so that no host hiccup can empty the queue:
    an elementwise kernel over 120 MB on one stream and a 12 MB
    device-to-device copy on another, for a few seconds.  A gap of more than
    5 ms between consecutive completions on one stream is the GPU itself
    pausing; the lists give when (seconds from the start) and for how long."""
    import torch
    x = torch.rand(30 << 20, device="cuda")
    y = torch.empty_like(x)
    src = torch.empty(12 << 20, dtype=torch.uint8, device="cuda")
    dst = torch.empty_like(src)
    sk, sc = torch.cuda.Stream(), torch.cuda.Stream()
    base = torch.cuda.Event(enable_timing=True)
    base.record(sk)
    base.synchronize()
    evs = {"kernel": [], "d2d_copy": []}
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for _ in range(8):
            with torch.cuda.stream(sk):
                torch.mul(x, 1.0001, out=y)
                e = torch.cuda.Event(enable_timing=True)
                e.record(sk)
                evs["kernel"].append(e)
            with torch.cuda.stream(sc):
                dst.copy_(src, non_blocking=True)
                e = torch.cuda.Event(enable_timing=True)
                e.record(sc)
                evs["d2d_copy"].append(e)
        if len(evs["kernel"]) > ahead:
            evs["kernel"][-ahead].synchronize()
    torch.cuda.synchronize()
    out = {"seconds": seconds, "queued_ahead": ahead, "launches_per_stream": len(evs["kernel"])}
    for kind, lst in evs.items():
        ts = [base.elapsed_time(e) for e in lst]
        gaps = [b - a for a, b in zip(ts, ts[1:])]
        srt = sorted(gaps)
        out[kind] = {"median_gap_ms": round(srt[len(srt) // 2], 4), "max_gap_ms": round(srt[-1], 3),
                     "pauses_over_5ms": [[round(t / 1e3, 2), round(g, 1)] for t, g in zip(ts[1:], gaps) if g > 5.0][:12]}
    del x, y, src, dst
    return out


# ------------------------------------------------------------------ other configs


def cuda_time(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def leg_c1(sc5, synth, stream):
    """3 x 512 x 512 FP32, k = [1,4,6,4,1]/16: a latency config (L2-resident)."""
    import torch
    h = w = 512
    A = torch.from_numpy(synth.image(1, h, w)).cuda()
    out = torch.empty((P, h - 4, w - 4), dtype=torch.float32, device="cuda")
    k = synth.kernel_binomial()
    res = {"workload": "3x512x512 f32, k=[1,4,6,4,1]/16"}
    for algo in ("fused", "two_pass"):
        plan = sc5.Plan(P, h, w, w, w - 4, algo=algo)
        ms = cuda_time(lambda: plan.run(A, out, k, stream=stream), 200, 20, stream)
        res[f"{algo}_us"] = round(ms * 1e3, 2)
        plan.close()
    plan = sc5.Plan(P, h, w, w, w - 4)
    b = sc5.Batch(plan, [{"in": A, "out": out, "H": h, "W": w, "in_pitch": w, "out_pitch": w - 4, "k": k}])
    ms = cuda_time(lambda: b.launch(stream), 200, 20, stream)
    res["fused_graph_us"] = round(ms * 1e3, 2)
    b.close()
    plan.close()
    return res


# The paper's image sizes (3 planes of N x N) and its best two-pass time per
# image with SIMD, OpenMP on the Xeon Phi 5110P (Table 2), for context only.
PAPER_SIZES_MS = {1152: 0.8, 1728: 2.0, 2592: 4.1, 3888: 8.8, 5832: 19.6, 8748: 59.2}


def leg_paper_sizes(sc5, stream):
    """3 x N x N FP32 for the paper's six image sizes, fused and two-pass,
    k = [1,4,6,4,1]/16, inputs uniform in [0, 255) drawn on the device
    (seeded).  Below 3 x 2592^2 the image and its result fit in L2."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(4)
    k = [1 / 16, 4 / 16, 6 / 16, 4 / 16, 1 / 16]
    res = {"workload": "3xNxN f32, N in the paper's sizes, k=[1,4,6,4,1]/16",
           "paper_ms_source": "Table 2, two-pass with SIMD, OpenMP, Xeon Phi 5110P"}
    for n, paper_ms in PAPER_SIZES_MS.items():
        A = torch.rand((P, n, n), generator=g, device="cuda") * 255.0
        out = torch.empty((P, n - 4, n - 4), dtype=torch.float32, device="cuda")
        row = {"paper_openmp_two_pass_ms": paper_ms}
        for algo in ("fused", "two_pass"):
            plan = sc5.Plan(P, n, n, n, n - 4, algo=algo)
            ms = cuda_time(lambda: plan.run(A, out, k, stream=stream), 50, 5, stream)
            plan.close()
            row[f"{algo}_ms"] = round(ms, 5)
        row["fused_mpix_s"] = round(n * n / (row["fused_ms"] / 1e3) / 1e6, 1)
        res[str(n)] = row
        del A, out
    torch.cuda.empty_cache()
    return res


def leg_pyramid(sc5, synth, stream, A_dev, k):
    """A five-level pyramid of the 3 x 8192 x 8192 FP32 image through
    sepconv5_pyramid_run: five chained REDUCE steps (blur with k, keep every
    second row and column), each level the input of the next.  Whole-pyramid
    CUDA-event time, and per level its REDUCE plan's time alone; algorithmic
    bytes per level = its input read once plus its output written once."""
    import torch
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks else 6800.0
    pyr = sc5.Pyramid(P, H, W, W, "f32", levels=5)
    levels, bufs = [], []
    for lv in range(1, 6):
        (h, w, _), (ho, wo, op) = pyr.level(lv - 1), pyr.level(lv)
        bufs.append(torch.empty((P, ho, op), dtype=torch.float32, device=A_dev.device))
        levels.append({"in": [h, w], "out": [ho, wo], "bytes": P * h * w * 4 + P * ho * wo * 4})
    total_ms = cuda_time(lambda: pyr.run(A_dev, bufs, k, stream=stream), 50, 5, stream)
    pyr.capture(A_dev, bufs, k)
    graph_ms = cuda_time(lambda: pyr.replay(stream), 50, 5, stream)
    srcs = [A_dev] + bufs[:-1]
    for lv, src, dst in zip(levels, srcs, bufs):
        h, w = lv["in"]
        plan = sc5.Plan(P, h, w, src.shape[-1], dst.shape[-1], algo="reduce")
        ms = cuda_time(lambda: plan.run(src, dst, k, stream=stream), 50, 5, stream)
        plan.close()
        lv["ms"] = round(ms, 5)
        lv["frac_of_measured_hbm"] = round(lv["bytes"] / ms / 1e6 / peak, 4)
    pyr.close()
    if sc5.device_status(stream) != 0:
        raise RuntimeError("a kernel reported a device error in the pyramid leg")
    alg = sum(lv["bytes"] for lv in levels)
    return {"workload": "5-level pyramid of 3x8192x8192 f32 (REDUCE steps, sepconv5_pyramid_run), k as the headline",
            "total_ms": round(total_ms, 5), "graph_replay_ms": round(graph_ms, 5), "launches": len(levels),
            "achieved_gbs": round(alg / total_ms / 1e6, 1), "frac_of_measured_hbm": round(alg / total_ms / 1e6 / peak, 4),
            "levels": levels}


def _batch_images(sc5, synth, dtype, shapes, x_dev, scales):
    """Device images of the 256-image batch in a stored format (converted on
    the GPU from the FP32 originals: input preparation, not the method)."""
    import torch
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "fp8e4m3": torch.float8_e4m3fn}[dtype]
    es = sc5.DTYPE_BYTES[dtype]
    imgs, keep = [], []
    for i, ((h, w), x) in enumerate(zip(shapes, x_dev)):
        s = scales[i] if dtype == "fp8e4m3" else 1.0
        pitch = -(-w * es // 16) * 16 // es
        A = torch.zeros((P, h, pitch), dtype=tdt, device="cuda")
        A[:, :, :w] = (x * s if s != 1.0 else x).to(tdt)
        op = -(-(w - 4) // 4) * 4
        imgs.append({"in": A, "H": h, "W": w, "in_pitch": pitch, "out_pitch": op,
                     "k": synth.kernel_normalised(3000 + i), "in_scale": s, "out_scale": s})
        keep.append(A)
    return imgs, keep


def leg_batch(sc5, synth, stream, dtypes):
    """The 256-image batch (H, W log-uniform in [64, 4096]): one persistent
    launch over the tile work-list, replayed from a CUDA graph, tile shape and
    CTAs per SM timed on the batch itself when it is created (ctas_per_sm =
    -2: every compiled shape at every feasible CTA count); FP32 and the stored
    formats."""
    import torch
    shapes = synth.batch_shapes(3, 256)
    x_dev = [torch.from_numpy(synth.image(3000 + i, h, w)).cuda() for i, (h, w) in enumerate(shapes)]
    scales = [448.0 / float(x.abs().max()) for x in x_dev]
    px = sum(h * w for h, w in shapes)
    t0 = time.perf_counter()
    sc5.autotune(2, [(d, o) for d, o in dtypes])
    tune_s = time.perf_counter() - t0
    results = {"workload": f"256 images, H and W log-uniform in [64,4096] (seed 3), {px / 1e6:.1f} Mpix x 3 planes",
               "autotune_s": round(tune_s, 1)}
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks else 6800.0
    for dtype, out_dtype in dtypes:
        imgs, keep = _batch_images(sc5, synth, dtype, shapes, x_dev, scales)
        odt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "fp8e4m3": torch.float8_e4m3fn}[out_dtype]
        outs = []
        for im in imgs:
            o = torch.empty((P, im["H"] - 4, im["out_pitch"]), dtype=odt, device="cuda")
            im["out"] = o
            if out_dtype == "f32":
                im["out_scale"] = 1.0
            outs.append(o)
        plan = sc5.Plan(P, 64, 64, in_dtype=dtype, out_dtype=out_dtype, ctas_per_sm=-2)
        t0 = time.perf_counter()
        b = sc5.Batch(plan, imgs)
        create_ms = (time.perf_counter() - t0) * 1e3
        ms = cuda_time(lambda: b.launch(stream), 20, 3, stream)
        info = b.info()
        alg = sum(P * h * w * sc5.DTYPE_BYTES[dtype] + P * (h - 4) * (w - 4) * sc5.DTYPE_BYTES[out_dtype]
                  for h, w in shapes)
        # narrow-to-narrow formats move 2-4 bytes per output: the FP32 multiply-adds of the
        # separable body (10 per output) on the FMA pipe bound them before HBM does
        outputs = sum(P * (h - 4) * (w - 4) for h, w in shapes)
        bound = "fma" if out_dtype != "f32" and dtype != "f32" else "hbm"
        results[f"{dtype}->{out_dtype}"] = {
            "bound": bound,
            "ms": round(ms, 4), "mpix_s": round(px / (ms / 1e3) / 1e6, 1), "achieved_gbs": round(alg / ms / 1e6, 1),
            "frac_of_measured_hbm": round(alg / ms / 1e6 / peak, 4),
            "tera_fma_per_s": round(outputs * FMA_PER_OUTPUT / (ms / 1e3) / 1e12, 2),
            "frac_of_fma_peak": round(outputs * FMA_PER_OUTPUT / (ms / 1e3) / fma_peak(), 4),
            "tiles": info["tiles"], "ctas": info["ctas"],
            "tile": f"{info['tile_h']}x{info['tile_w']}", "create_ms": round(create_ms, 1)}
        b.close()
        plan.close()
        del imgs, keep, outs
        torch.cuda.empty_cache()
    return results


def leg_serve(sc5, synth, n_req, link=None):
    """Serving stream: Poisson arrivals, sizes uniform over 640x480,
    1920x1080 and 4096x4096, per-request normalised k.  BF16 storage with
    continuous batching against FP32 with one launch per request, at 0.5x,
    0.8x and 0.95x of the measured saturation request rate of the BF16
    server.  Latency = completion of the result's copy to the host minus the
    request's scheduled arrival.  Pinned buffers: 8 outputs per size class."""
    import torch
    sizes = synth.SERVE_SIZES
    out = {"workload": f"{n_req} requests per load, sizes {sizes} (H, W), Poisson arrivals",
           "budget_bytes": 16 << 30}

    def make_pool(dtype, n_buf):
        """Per size class: one pinned input image and n_buf pinned output buffers."""
        tdt = {"bf16": torch.int16, "f32": torch.float32}[dtype]
        pool = []
        for ci, (h, w) in enumerate(sizes):
            x = synth.image(700 + ci, h, w)
            src = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16) if dtype == "bf16" else torch.from_numpy(x)
            src = src.contiguous().pin_memory()
            bufs = [torch.empty((P, h - 4, w - 4), dtype=tdt).pin_memory() for _ in range(n_buf)]
            pool.append((src, bufs, h, w))
        return pool

    def run(dtype, merge, rate, n, pool, seed):
        """One thread submits every request at its scheduled arrival time and
        polls the tickets once all are submitted.  The requests (sc5_image
        structures) are built before the clock starts, so the loop does no
        marshalling; the outputs of a size class rotate over its pinned
        buffers without waiting (the benchmark does not read them), so a
        client-side buffer never holds a submission back.  The server's own
        clock gives each latency (submit to result on the host), to which the
        submission's lateness against its arrival time is added."""
        srv = sc5.Server(hbm_budget_bytes=16 << 30, dtype=dtype, max_inflight=64, n_streams=2, merge=merge,
                         max_merge=8 if merge else 0)
        stream_ = synth.serve_stream(seed, n, rate) if rate else [(0.0, c, s) for (_, c, s) in synth.serve_stream(seed, n, 1.0)]
        n_buf = len(pool[0][1])
        used = [0] * len(pool)
        reqs = []
        for (t_arr, ci, kseed) in stream_:
            src, bufs, h, w = pool[ci]
            reqs.append({"in": src, "out": bufs[used[ci] % n_buf], "H": h, "W": w, "in_pitch": w,
                         "out_pitch": w - 4, "k": synth.kernel_normalised(kseed)})
            used[ci] += 1
        arr = sc5.make_images(reqs)
        tickets, late = [], []
        gc.collect()
        gc.disable()  # no collector pause holds the submitting thread back
        t_start = time.perf_counter()
        for j, (t_arr, ci, _) in enumerate(stream_):
            target = t_start + t_arr
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 2e-4:
                    time.sleep(target - now - 1e-4)
            t_sub = time.perf_counter()
            tk = srv.submit_image(arr[j])
            while tk is None:
                time.sleep(1e-4)
                tk = srv.submit_image(arr[j])
            late.append(t_sub - target)
            tickets.append((tk, target, t_sub, ci))
        lat = [[] for _ in pool]
        for tk, target, t_sub, ci in tickets:
            lat[ci].append(t_sub + srv.poll(tk, -1) * 1e-6 - target)
        wall = time.perf_counter() - t_start
        gc.enable()
        st = srv.stats()
        srv.close()
        px = sum(pool[ci][2] * pool[ci][3] for (_, ci, _) in stream_)
        all_ms = np.concatenate([np.array(v) for v in lat]) * 1e3
        res = {"offered_req_s": round(rate, 1) if rate else None, "achieved_req_s": round(n / wall, 1),
               "mpix_s": round(px / wall / 1e6, 1), "p50_ms": round(float(np.percentile(all_ms, 50)), 3),
               "p99_ms": round(float(np.percentile(all_ms, 99)), 3), "launches": st["launches"],
               "merged_max": st["merged_max"], "resident_peak_bytes": st["resident_peak_bytes"],
               "submit_late_p99_ms": round(float(np.percentile(np.array(late) * 1e3, 99)), 3),
               "per_size": {f"{h}x{w}": {"p50_ms": round(float(np.percentile(np.array(v) * 1e3, 50)), 3),
                                         "p99_ms": round(float(np.percentile(np.array(v) * 1e3, 99)), 3)}
                            for (_, _, h, w), v in zip(pool, lat) if v},
               "phases_ms": {f"{ph}_p{q}": round(st[f"{ph}_us_p{q}"] / 1e3, 3)
                             for ph in ("queue", "stage", "run") for q in (50, 99)}}
        return res

    pool_bf = make_pool("bf16", 8)
    # saturation: a burst long enough (about 2 s) to include a pause of the
    # GPU, so that the offered loads below are fractions of a sustained rate
    sat = run("bf16", True, 0.0, min(n_req, 8000), pool_bf, 11)
    rate_sat = sat["achieved_req_s"]
    # the link ceiling of this mix: each request's input crosses host->device
    # and its output device->host, both directions at once
    es = sc5.DTYPE_BYTES["bf16"]
    bytes_per_req = sum(P * h * w * es + P * (h - 4) * (w - 4) * es for h, w in sizes) / len(sizes)
    sat["link_bytes_per_req"] = int(bytes_per_req)
    if link and link.get("both_gbs"):
        both = max(link["both_gbs"], link.get("both_2streams_gbs", 0.0))
        sat["link_ceiling_req_s"] = round(both * 1e9 / bytes_per_req, 1)
        sat["frac_of_link"] = round(rate_sat * bytes_per_req / (both * 1e9), 4)
    out["saturation_bf16_merged"] = sat
    out["device_pauses"] = device_pauses(6.0)
    pool_f32 = make_pool("f32", 8)
    for frac in (0.5, 0.8, 0.95):
        rate = frac * rate_sat
        out[f"load_{frac}"] = {"bf16_merged": run("bf16", True, rate, n_req, pool_bf, 20 + int(frac * 100)),
                               "f32_per_request": run("f32", False, rate, n_req, pool_f32, 20 + int(frac * 100))}
    del pool_bf, pool_f32
    return out


# ------------------------------------------------------------------ one configuration


def parse_case(spec: str) -> dict:
    """`--case` key=value list -> options (defaults: 3 x 8192 x 8192 FP32 fused, planar)."""
    c = {"dtype": "f32", "out": None, "algo": "fused", "layout": "planar", "planes": P, "H": H, "W": W,
         "tile": "", "ctas": 0, "batch": 0, "taps": 5, "opitch": 0}
    for item in filter(None, (x.strip() for x in spec.split(","))):
        key, _, val = item.partition("=")
        if key not in c:
            raise SystemExit(f"--case: unknown key {key!r} (keys: {', '.join(c)})")
        c[key] = int(val) if key in ("planes", "H", "W", "ctas", "batch", "taps", "opitch") else val
    c["out"] = c["out"] or c["dtype"]
    return c


def run_case(args):
    """One configuration on a synthetic image (pixels uniform in [0, 255) drawn
    on the device, seed 2; k as the headline; FP8 inputs scaled by 448/max):
    median CUDA-event time of --steps launches after --warmup, and the
    algorithmic GB/s (input read once, output written once)."""
    import torch

    from paper_1711_09791_gb300 import sepconv5 as sc5
    from paper_1711_09791_gb300 import synth
    c = parse_case(args.case)
    sc5.load()
    if c["batch"] > 0:
        return run_case_batch(args, c, sc5, synth)
    Pc, Hc, Wc, dt, odt = c["planes"], c["H"], c["W"], c["dtype"], c["out"]
    es, eo = sc5.DTYPE_BYTES[dt], sc5.DTYPE_BYTES[odt]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "fp8e4m3": torch.float8_e4m3fn}
    g = torch.Generator(device="cuda").manual_seed(2)
    x = torch.rand((Pc, Hc, Wc), generator=g, device="cuda") * 255.0
    scale = 448.0 / float(x.max()) if dt == "fp8e4m3" else 1.0
    th = tw = st = 0
    if c["tile"]:
        th, tw, st = (int(v) for v in c["tile"].split("x"))
    n = c["taps"]
    Ho, Wo = sc5.reduce_dims(Hc, Wc) if c["algo"] == "reduce" else (Hc - n + 1, Wc - n + 1)
    if c["layout"] == "hwc":
        pitch = -(-3 * Wc * es // 16) * 16 // es
        opitch = -(-3 * Wo // 4) * 4
        A = torch.zeros((Hc, pitch), dtype=tdt[dt], device="cuda")
        A[:, :3 * Wc] = (x * scale).permute(1, 2, 0).reshape(Hc, 3 * Wc).to(tdt[dt])
        out = torch.empty((Ho, opitch), dtype=tdt[odt], device="cuda")
    else:
        pitch = -(-Wc * es // 16) * 16 // es
        opitch = c["opitch"] or -(-Wo * eo // 16) * 16 // eo
        A = torch.zeros((Pc, Hc, pitch), dtype=tdt[dt], device="cuda")
        A[:, :, :Wc] = (x * scale).to(tdt[dt])
        out = torch.empty((Pc, Ho, opitch), dtype=tdt[odt], device="cuda")
    del x
    plan = sc5.Plan(Pc, Hc, Wc, pitch, opitch, dt, odt, "valid", c["algo"], th, tw, st, c["ctas"], layout=c["layout"],
                    taps=n)
    k = synth.kernel_normalised(SEED)
    if n != 5:
        kn = synth.rng(100 + n).uniform(0, 1, n)
        k = (kn / kn.sum()).astype(np.float32)
    out_scale = scale if odt == "fp8e4m3" else 1.0
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 0)):
        plan.run(A, out, k, scale, out_scale, stream=stream)
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(args.steps, 1)):
        e0.record(stream)
        plan.run(A, out, k, scale, out_scale, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    if sc5.device_status(stream) != 0:
        raise SystemExit("a kernel reported a device error")
    info = plan.info()
    plan.close()
    ms = statistics.median(times)
    alg = Pc * Hc * Wc * es + Pc * Ho * Wo * eo
    return {"case": c, "ms": round(ms, 5), "gbs": round(alg / ms / 1e6, 1), "mpix_s": round(Hc * Wc / ms / 1e3, 1),
            "algorithmic_bytes": alg, "plan": info, "launches": len(times)}


def run_case_batch(args, c, sc5, synth):
    """The first N images of the 256-image batch (as the batch leg builds
    them), one persistent launch replayed from a CUDA graph: tile shape from
    the override or the built-in default, CTAs per SM as given (0: the
    shape's default); median CUDA-event time of --steps replays."""
    import torch
    dt, odt = c["dtype"], c["out"]
    shapes = synth.batch_shapes(3, 256)[:c["batch"]]
    x_dev = [torch.from_numpy(synth.image(3000 + i, h, w)).cuda() for i, (h, w) in enumerate(shapes)]
    scales = [448.0 / float(x.abs().max()) for x in x_dev]
    imgs, keep = _batch_images(sc5, synth, dt, shapes, x_dev, scales)
    del x_dev
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "fp8e4m3": torch.float8_e4m3fn}
    for im in imgs:
        im["out"] = torch.empty((P, im["H"] - 4, im["out_pitch"]), dtype=tdt[odt], device="cuda")
        if odt == "f32":
            im["out_scale"] = 1.0
    th = tw = st = 0
    if c["tile"]:
        th, tw, st = (int(v) for v in c["tile"].split("x"))
    plan = sc5.Plan(P, 64, 64, in_dtype=dt, out_dtype=odt, tile_h=th, tile_w=tw, stages=st, ctas_per_sm=c["ctas"])
    b = sc5.Batch(plan, imgs)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 0)):
        b.launch(stream)
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(args.steps, 1)):
        e0.record(stream)
        b.launch(stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    if sc5.device_status(stream) != 0:
        raise SystemExit("a kernel reported a device error")
    info = b.info()
    b.close()
    plan.close()
    ms = statistics.median(times)
    es, eo = sc5.DTYPE_BYTES[dt], sc5.DTYPE_BYTES[odt]
    alg = sum(P * h * w * es + P * (h - 4) * (w - 4) * eo for h, w in shapes)
    px = sum(h * w for h, w in shapes)
    return {"case": c, "ms": round(ms, 5), "gbs": round(alg / ms / 1e6, 1), "mpix_s": round(px / ms / 1e3, 1),
            "algorithmic_bytes": alg, "batch": info, "launches": len(times)}


# ------------------------------------------------------------------ main legs


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_1711_09791_gb300 import sepconv5, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sepconv5.load()
    rows = args.split == "rows"
    A = synth.image(SEED if rows else rank_image_seed(rank), H, W)
    k = synth.kernel_normalised(SEED)
    A_dev = torch.from_numpy(A).to(dev)
    out = torch.empty((P, H - 4, W - 4), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = sepconv5.Plan(P, H, W, W, W - 4, algo="fused")
    # rows split: this rank's band of output rows, as views with the whole image's plane strides
    r0, r1 = row_band(H - 4, world, rank) if rows else (0, H - 4)
    band = sepconv5.Plan(P, r1 - r0 + 4, W, W, W - 4, in_plane_stride=H * W, out_plane_stride=(H - 4) * (W - 4))
    band_in, band_out = A_dev[:, r0:, :], out[:, r0:, :]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, world, dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        n0 = sepconv5.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        return max_over_ranks(ms), sepconv5.launch_count() - n0

    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    smi_index = vis[local_rank] if local_rank < len(vis) and vis[local_rank].isdigit() else str(local_rank)
    sampler = ClockSampler(smi_index)
    sampler.start()
    sampler.mark(0)
    step = (lambda: band.run(band_in, band_out, k, stream=stream)) if rows else \
        (lambda: plan.run(A_dev, out, k, stream=stream))
    ms, launches = timed(step, args.steps, max(args.warmup, 3))
    # A timed region of a few milliseconds falls between two clock samples:
    # the same launches keep running, untimed and uncounted, for a quarter of
    # a second after it so that the sampler sees the GPU under this load.
    t_soak = time.perf_counter() + 0.25
    while time.perf_counter() < t_soak:
        for _ in range(16):
            step()
        torch.cuda.synchronize(dev)
    band.close()
    sampler.mark(1)
    clocks = sampler.stop()
    if sepconv5.device_status(stream) != 0:
        raise RuntimeError("a kernel reported a device error during the timed region")

    # bytes of this rank's launch (its band when the rows are split)
    alg = algorithmic_bytes(H, W) if not rows else P * (r1 - r0 + 4) * W * 4 + P * (r1 - r0) * (W - 4) * 4
    pixels = H * W
    # rows split: the ranks share one image, so the whole job is that image
    value = whole_job_value(1 if rows else world, pixels, ms)
    peaks = measured_peaks()
    if peaks and peaks.get("hbm_gbs"):
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    achieved = alg / (ms / 1e3) / 1e9
    extras = {}
    if not args.no_extras:
        # two-pass pair on the same image, same algorithmic bytes
        plan2 = sepconv5.Plan(P, H, W, W, W - 4, algo="two_pass")
        k2 = max(20, args.steps // 4)
        ms2, l2 = timed(lambda: plan2.run(A_dev, out, k, stream=stream), k2, 5)
        plan2.close()
        # the paper's single-pass algorithm as written: 25 products per output
        plan3 = sepconv5.Plan(P, H, W, W, W - 4, algo="direct")
        ms3, _ = timed(lambda: plan3.run(A_dev, out, k, stream=stream), k2, 5)
        plan3.close()
        extras["direct_single_pass"] = {"ms_per_step": round(ms3, 5), "value": round(world * pixels / (ms3 / 1e3) / 1e6, 1),
                                        "unit": "Mpix/s", "achieved_gbs": round(alg / (ms3 / 1e3) / 1e9, 1),
                                        "frac_of_measured_hbm": round(alg / (ms3 / 1e3) / 1e9 / peak, 4),
                                        "vs_fused": round(ms3 / ms, 3)}
        # the 3R x C agglomerated layout of Sec. 6 (rows of the 3 planes side by side)
        X = A_dev.permute(1, 0, 2).contiguous()
        Y = torch.empty((H - 4, P, W - 4), dtype=torch.float32, device=dev)
        pl = sepconv5.Plan(P, H, W, P * W, P * (W - 4), in_plane_stride=W, out_plane_stride=W - 4)
        msl, _ = timed(lambda: pl.run(X, Y, k, stream=stream), k2, 3)
        pl.close()
        del X, Y
        extras["layout_3RxC"] = {"ms_per_step": round(msl, 5), "frac_of_measured_hbm": round(alg / (msl / 1e3) / 1e9 / peak, 4),
                                 "vs_stacked": round(msl / ms, 3)}
        # pixel-interleaved (HWC) images: the same pixels as RGB triples
        X = A_dev.permute(1, 2, 0).contiguous()
        Y = torch.empty((H - 4, W - 4, P), dtype=torch.float32, device=dev)
        pl = sepconv5.Plan(P, H, W, P * W, P * (W - 4), layout="hwc")
        msh, _ = timed(lambda: pl.run(X, Y, k, stream=stream), k2, 3)
        pl.close()
        del X, Y
        extras["layout_HWC"] = {"ms_per_step": round(msh, 5), "frac_of_measured_hbm": round(alg / (msh / 1e3) / 1e9 / peak, 4),
                                "vs_planar": round(msh / ms, 3)}
        # other odd kernel widths through the fused kernel
        widths = {}
        for n in (3, 7, 9):
            kn = synth.rng(100 + n).uniform(0, 1, n)
            kn = (kn / kn.sum()).astype(np.float32)
            # output rows padded to a multiple of 4 values (16 bytes): vector stores
            opn = -(-(W - n + 1) // 4) * 4
            outn = torch.empty((P, H - n + 1, opn), dtype=torch.float32, device=dev)
            pl = sepconv5.Plan(P, H, W, W, opn, taps=n)
            msn, _ = timed(lambda: pl.run(A_dev, outn, kn, stream=stream), k2, 3)
            pl.close()
            algn = P * H * W * 4 + P * (H - n + 1) * (W - n + 1) * 4
            widths[f"taps_{n}"] = {"ms_per_step": round(msn, 5),
                                   "frac_of_measured_hbm": round(algn / (msn / 1e3) / 1e9 / peak, 4)}
            del outn
        extras["widths"] = widths
        # in place: Listing 1's two-pass structure vs the single pass with copy-back
        A_ip = A_dev.clone()
        ip = {}
        for algo in ("two_pass", "fused"):
            pl = sepconv5.Plan(P, H, W, W, W, border="keep", algo=algo)
            msi, _ = timed(lambda: pl.run_inplace(A_ip, k, stream=stream), k2, 3)
            pl.close()
            ip[algo] = {"ms_per_step": round(msi, 5), "vs_out_of_place_fused": round(msi / ms, 3)}
        del A_ip
        extras["in_place"] = {"two_pass_listing1": ip["two_pass"], "single_pass_copy_back": ip["fused"]}
        extras["two_pass"] = {"ms_per_step": round(ms2, 5), "value": round(world * pixels / (ms2 / 1e3) / 1e6, 1),
                              "unit": "Mpix/s", "achieved_gbs": round(alg / (ms2 / 1e3) / 1e9, 1),
                              "frac_of_measured_hbm": round(alg / (ms2 / 1e3) / 1e9 / peak, 4),
                              "launches_per_step": l2 / k2, "fused_speedup": round(ms2 / ms, 3)}
        # empty-kernel launch overhead
        n_probe = 2000
        ms_probe, _ = timed(lambda: sepconv5.empty_launches(1, stream), n_probe, 50)
        extras["empty_launch_us"] = round(ms_probe * 1e3, 3)
    # end to end: host buffers through sepconv5_run_host
    A_host = torch.from_numpy(A).pin_memory()
    out_host = torch.empty((P, H - 4, W - 4), dtype=torch.float32).pin_memory()
    e2e_steps = max(10, min(args.steps // 50, 30))
    for _ in range(2):
        plan.run_host(A_host, out_host, k, stream=stream)
    barrier()
    n0 = sepconv5.launch_count()
    gc.disable()  # no collector pause inside the wall-clock region
    t0 = time.perf_counter()
    step_ms = []
    for _ in range(e2e_steps):
        ts = time.perf_counter()
        plan.run_host(A_host, out_host, k, stream=stream)  # returns when the result is on the host
        step_ms.append((time.perf_counter() - ts) * 1e3)
    torch.cuda.synchronize(dev)
    e2e_mean_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    gc.enable()
    # The value uses the median call: a host thread that the OS leaves unscheduled for
    # tens of milliseconds, now and then, would otherwise set it; the mean and the
    # slowest call are reported beside it.
    e2e_ms = max_over_ranks(statistics.median(step_ms))
    e2e_launches = (sepconv5.launch_count() - n0) / e2e_steps
    # spot check the e2e result against the device result of the same (fused) plan
    plan.run(A_dev, out, k, stream=stream)
    torch.cuda.synchronize(dev)
    if not torch.equal(out_host[:, ::1024, ::1024].to(dev), out[:, ::1024, ::1024]):
        raise RuntimeError("offload result differs from the device result")
    e2e = {"value": round(world * pixels / (e2e_ms / 1e3) / 1e6, 1), "unit": "Mpix/s",
           "h2d_bytes_per_step": P * H * W * 4, "d2h_bytes_per_step": P * (H - 4) * (W - 4) * 4,
           "ms_per_step": round(e2e_ms, 4), "value_from": f"median of {e2e_steps} calls",
           "ms_per_step_mean": round(e2e_mean_ms, 4), "ms_per_step_max": round(max(step_ms), 4),
           "launches_per_step": e2e_launches,
           "api": "sepconv5_run_host (pinned host buffers, band-pipelined copies)"}
    # the ceiling of the offload path: plain copies over the CPU-GPU link
    e2e["link"] = copy_probe(A_host, out_host, A_dev, out, dev)
    lb = e2e["link"]
    e2e["frac_of_link"] = round(min(lb["both_ms"], lb["both_2streams_ms"]) / e2e_ms, 4)
    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        cpu = oracle_sample(A, k)
        cpu["fp32_two_pass_openmp"] = cpu_two_pass_sample(A, k)
    plan.close()
    del A_host, out_host
    legs = [] if args.no_extras or rank != 0 else [x.strip() for x in args.legs.split(",") if x.strip()]
    if "pyramid" in legs:
        extras["pyramid"] = leg_pyramid(sepconv5, synth, stream, A_dev, k)
    if legs:
        del A_dev, out
        torch.cuda.empty_cache()
        if "c1" in legs:
            extras["small_c1"] = leg_c1(sepconv5, synth, stream)
        if "c3" in legs or "c4" in legs:
            pairs = [("f32", "f32")] if "c3" in legs else []
            if "c4" in legs:
                pairs += [("bf16", "bf16"), ("bf16", "f32"), ("f16", "f16"), ("f16", "f32"),
                          ("fp8e4m3", "fp8e4m3"), ("fp8e4m3", "f32")]
            extras["batch_c3_c4"] = leg_batch(sepconv5, synth, stream, pairs)
        if "paper" in legs:
            extras["paper_sizes"] = leg_paper_sizes(sepconv5, stream)
        if "c5" in legs:
            extras["serve_c5"] = leg_serve(sepconv5, synth, args.serve_requests, e2e.get("link"))
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 5), "higher_is_better": True,
        "scaling": "strong" if rows else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": run_config(world, args.split),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": profiled_traffic(),
                     "peak_source": peak_src, "kernel": "fused_kernel<float,float> (single image)",
                     "algorithmic_bytes_per_launch": alg},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(extras)
    return line


def run_config(world: int, split: str = "images") -> dict:
    """The workload both arms report (the reference arm times the oracle on it)."""
    return {"workload": WORKLOAD, "planes": P, "H": H, "W": W, "seed": SEED, "border": "valid",
            "l2": "inputs larger than L2 (805 MB in, 804 MB out per step); no flush",
            "parallelism": f"replicas x{world}" if split == "images" else f"row bands x{world}"}


def run_reference(args, rank: int, world: int):
    """The oracle, as it stands, on the host cores: each step a bounded sample
    (a band of rows) of the same image and kernel."""
    if rank != 0:
        return None
    from paper_1711_09791_gb300 import synth
    import oracle
    A = synth.image(SEED, H, W)
    k = synth.kernel_normalised(SEED).astype(np.float64)
    rows = 512  # output rows per step: a fraction of a second of single-threaded FP64 work
    band = A[:, :rows + 4, :].astype(np.float64)
    for _ in range(3):
        oracle.direct(band, k)
    steps = max(1, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.direct(band, k)
    dt = (time.perf_counter() - t0) / steps
    value = rows * (W - 4) / dt / 1e6
    sample = f"{rows + 4} input rows x {W} cols x {P} planes per step ({rows} x {W - 4} output pixels), FP64 direct Eq. 1, one thread"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mpix/s", "n_gpus": world,
            "steps": steps, "warmup": 3, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "strong" if getattr(args, "split", "images") == "rows" else "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": run_config(world, getattr(args, "split", "images")),
            "cpu_baseline": {"value": round(value, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.case is not None:
        print(json.dumps(run_case(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
