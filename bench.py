"""Benchmark: SWIH likelihood maps on a 1024 x 1024 synthetic tracking scene.

One step is one pass of the whole hot path over one frame:
  quantise (K1) + weighted integral histograms (K2) for two plans
    - Manhattan + Euclidean (terms 1, x, y, x^2, y^2; 32-bit ring)
    - Gaussian approximant (terms x^k y^l, k, l <= 4; 64-bit ring)
  + window gather / translate / normalise / Bhattacharyya (K3) for every
    valid centre of 3 kernels x 3 windows (21, 41, 81): 8,602,224 windows.
The two plans share only the frame, so a step runs them on two streams (the
Gaussian plan on the main one, the other forked from it and joined back).
The metric is windows per second (whole job). Inputs are resident in HBM
when the timed region starts; the integral histograms (7.1 GB per step) are
far larger than L2, so no explicit L2 flush is done between steps.

Also reported: an end-to-end figure through the C ABI from pinned host memory
(frame and targets up, all nine maps back, every step, on copy streams that
overlap the kernels of neighbouring steps), the gathers alone, the roofline of
the dominant kernel (CUDA events on the launching stream, in the timed region
and with the step on one stream), SM clocks sampled during the timed region,
the step periods, and the CPU oracle timed on the host cores on a bounded
sample of the same workload.

At N = 1 the line also carries measurements of other workloads: a 128x128
frame's latency, the step on an i.i.d. frame (nothing to skip), the
many-region paths "batched_regions" (64 search regions of a 4096x4096 u16
frame, one batch replayed as a CUDA graph against one plan per region) and
"serving" (a Poisson stream of tracking queries at 2000/s against 16 resident
frames: the server's continuous batching against one plan per query, with
p50/p99 latency), "large_frame" (an 8192x8192 u16 frame whose integral
histograms exceed device memory, streamed in bands), the exponential kernel,
feature channels and the Fig. 6 sweep; each with its error against the
oracle where it makes maps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl swih|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KERNELS = ("manhattan", "euclidean", "gaussian")
WINDOWS = (21, 41, 81)
METRIC = "SWIH windows/s & HBM-roofline %; served p50/p99 latency vs plain per-ROI path"
WORKLOAD = ("1024x1024 u8 synthetic tracking scene (fBm background + 8 textured ellipses), "
            "B=32, Manhattan/Euclidean/Gaussian(sigma=w/4) kernels x windows 21/41/81, "
            "full valid likelihood map per kernel and window")


def windows_per_step(H=1024, W=1024):
    return len(KERNELS) * sum((H - w + 1) * (W - w + 1) for w in WINDOWS)


# ----------------------------------------------------------------------------- helpers
def progress(msg: str) -> None:
    """One line of progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = threading.Event()

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))
            self.first.set()

    def wait_first(self, timeout=5.0):
        if self.proc:
            self.first.wait(timeout)

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between wall times t0 and t1. A region
        shorter than the sampling period may hold none: then the last sample
        before it and the first after it, which bracket it, are summarised
        (marked "bracketing")."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        if t1 is not None:  # let a sample after the region arrive (at most 0.5 s)
            deadline = time.time() + 0.5
            while time.time() < deadline and not any(ts > t1 for ts, _ in self.lines):
                time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        samples = []
        for ts, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) == 7:
                samples.append((ts, parts))
        rows = [r for ts, r in samples if t0 is None or t0 <= ts <= t1]
        bracketing = False
        if not rows and t0 is not None:
            before = [r for ts, r in samples if ts < t0][-1:]
            after = [r for ts, r in samples if ts > t1][:1]
            rows = before + after
            bracketing = bool(rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = max(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
               "reasons": reasons, "samples": len(rows)}
        if bracketing:
            out["bracketing"] = True  # the samples just before and after the region
        return out


def code_sha256(path: str) -> str:
    """sha256 of a C++/CUDA source with its comments removed and whitespace runs
    collapsed: edits to comments alone keep the hash, any change to the code
    changes it. String and character literals are kept as written."""
    text = open(path).read()
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return hashlib.sha256(" ".join("".join(out).split()).encode()).hexdigest()


def profile_traffic(kernel_name: str, source: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current code of the kernel (code_sha256 recorded in the summary), else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel_name}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"code_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not (m and t):
        return None
    src = os.path.join(ROOT, "paper_1705_03524_gb300", "csrc", source)
    return float(t.group(1)) if code_sha256(src) == m.group(1) else None


def reduce_max_over_ranks(values):
    """Element-wise max of per-rank floats over the process group (one
    all-reduce; CUDA tensors under NCCL, CPU tensors under gloo)."""
    import torch
    import torch.distributed as tdist
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank_step, steps, world, max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank_step * steps * world / (max_ms * 1e-3)


# ----------------------------------------------------------------------------- swih arm

class FrameStep:
    """One benchmark step over a frame: the Manhattan+Euclidean plan's and the
    Gaussian plan's integral histograms, then each kernel's windows in one
    multi-window launch (swih_likelihood_scales). Targets are the window of
    each kernel and size centred on (tx, ty), set up untimed.

    With two streams (the default) the two plans, which share only the frame,
    run side by side: the Gaussian plan's build and gather on `stream`, the
    Manhattan+Euclidean plan's build and gathers on a second stream forked from
    it and joined back at the end of the step."""

    def __init__(self, S, dev, img, B, kernels, tx, ty, stream, windows=WINDOWS, streams=2):
        import torch

        H, W = img.shape
        self.stream = stream
        self.kernels = kernels
        self.windows = windows
        self.d_img = torch.from_numpy(img).to(dev)
        me = tuple(k for k in kernels if k != "gaussian")
        mw = max(windows)
        self.plan_me = S.Plan(S.make_desc(H, W, bins=B, kernels=me, max_win=(mw, mw))) if me else None
        self.plan_g = (S.Plan(S.make_desc(H, W, bins=B, kernels=("gaussian",), max_win=(mw, mw)))
                       if "gaussian" in kernels else None)
        self.plans = [pl for pl in (self.plan_me, self.plan_g) if pl is not None]
        self.plan_of = {"manhattan": self.plan_me, "euclidean": self.plan_me, "gaussian": self.plan_g}
        self.info_me = self.plan_me.info() if self.plan_me else None
        self.info_g = self.plan_g.info() if self.plan_g else None
        self.jobs = [(k, w) for k in kernels for w in windows]
        self.job_of = {k: [j for j, (kk, _) in enumerate(self.jobs) if kk == k] for k in kernels}
        for pl in self.plans:
            pl.build_ih(self.d_img, stream)
        self.targets = torch.empty((len(self.jobs), B), dtype=torch.float32, device=dev)
        for j, (k, w) in enumerate(self.jobs):
            self.plan_of[k].local_hist(k, w, w, tx, ty, 1, 1, self.targets[j], stream)
        self.maps = [torch.empty((H - w + 1, W - w + 1), dtype=torch.float32, device=dev) for _, w in self.jobs]
        for pl in self.plans:
            pl.sync_status(stream)
        self.windows_per_step = sum(m.numel() for m in self.maps)
        # the Manhattan+Euclidean plan's stream (the main one with streams=1)
        self.side = torch.cuda.Stream(device=dev) if streams > 1 and self.plan_me and self.plan_g else stream
        self.fork = torch.cuda.Event()
        self.join = torch.cuda.Event()
        self.stages = ([s for s, pl in (("build_me", self.plan_me), ("build_g", self.plan_g)) if pl]
                       + [f"gather_{k}" for k in kernels])

    def new_events(self):
        """Begin and end events of every stage of one step."""
        import torch

        return {st: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for st in self.stages}

    def run_maps(self, d_img, targets, maps, s, side, ev=None):
        """Enqueue one step on d_img: builds and gathers of both plans, the
        Manhattan+Euclidean ones on `side` (forked from and joined back to s).
        ev (optional): new_events() of this step."""
        def mark(stage, i, st):
            if ev is not None:
                ev[stage][i].record(st)

        if side is not s:
            self.fork.record(s)
            side.wait_event(self.fork)
        for st, pl, name in ((side, self.plan_me, "build_me"), (s, self.plan_g, "build_g")):
            if pl:
                mark(name, 0, st)
                pl.build_ih(d_img, st)
                mark(name, 1, st)
        for k in self.kernels:  # the kernel's windows in one launch (multi-scale search)
            st = s if k == "gaussian" else side
            js = self.job_of[k]
            mark(f"gather_{k}", 0, st)
            self.plan_of[k].likelihood_scales(k, [(self.jobs[j][1], self.jobs[j][1]) for j in js],
                                              [targets[j] for j in js], [maps[j] for j in js], st)
            mark(f"gather_{k}", 1, st)
        if side is not s:
            self.join.record(side)
            s.wait_event(self.join)

    def step(self, ev=None):
        """ev (optional): new_events() of this step."""
        self.run_maps(self.d_img, self.targets, self.maps, self.stream, self.side, ev)

    @staticmethod
    def stage_ms(events):
        """Mean duration of each stage over the steps' events."""
        out = {}
        for ev in events:
            for st, (e0, e1) in ev.items():
                out.setdefault(st, []).append(e0.elapsed_time(e1))
        return {k: float(np.mean(v)) for k, v in out.items()}

    @staticmethod
    def step_ms(events):
        """Median, p99 and max of the step periods: from one step's first event
        on the main stream (the Gaussian build's, else the only plan's) to the
        next step's (no extra events: one recorded ahead of the fork changed how
        the two streams were scheduled)."""
        if not events:
            return None
        first = "build_g" if "build_g" in events[0] else next(iter(events[0]))
        t = np.array([a[first][0].elapsed_time(b[first][0]) for a, b in zip(events, events[1:])])
        if t.size == 0:
            return None
        return {"p50": float(np.median(t)), "p99": float(np.percentile(t, 99)), "max": float(t.max()),
                "periods": int(t.size)}

    def timed(self, steps, clocks=None):
        """Time `steps` steps with CUDA events (after a synchronize); returns
        (total ms, per-launch mean ms by stage, integral-histogram bytes the
        Gaussian gathers loaded per launch, clock summary or None)."""
        import torch

        events = [self.new_events() for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.start()
            clocks.wait_first()
        wall0 = time.time()
        for pl in self.plans:
            pl.load_bytes(reset=True)
        t0.record(self.stream)
        for i in range(steps):
            self.step(events[i])
        t1.record(self.stream)
        torch.cuda.synchronize()
        wall1 = time.time()
        clk = clocks.stop(wall0, wall1) if clocks is not None else None
        for pl in self.plans:
            pl.sync_status(self.stream)
        loaded_g = self.plan_g.load_bytes() / steps if self.plan_g else 0.0
        return t0.elapsed_time(t1), self.stage_ms(events), loaded_g, clk

    def close(self):
        for pl in self.plans:
            pl.close()


# inputs and final maps of the benchmark run, for the oracle comparison
_ORACLE_CHECK = []
# (block name, thunk) pairs: oracle comparisons of the extra measurements, run
# after every timed part; each thunk returns the block's "oracle_error"
_ORACLE_LATER = []


def run_swih(args, rank, world, local_rank):
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = synth.config2(seed=2 + rank, size=args.size)  # independent frame per rank
    img = cfg["image"]
    H, W = img.shape
    B = args.bins
    kernels = tuple(k for k in KERNELS if k in args.kernels.split(","))
    tx, ty = cfg["target_centre"]
    stream = torch.cuda.Stream(device=dev)
    fr = FrameStep(S, dev, img, B, kernels, tx, ty, stream, streams=args.streams)
    d_img = fr.d_img
    plan_me, plan_g, plans, plan_of = fr.plan_me, fr.plan_g, fr.plans, fr.plan_of
    info_me, info_g = fr.info_me, fr.info_g
    jobs, job_of, targets, maps = fr.jobs, fr.job_of, fr.targets, fr.maps
    step = fr.step

    for _ in range(args.warmup):
        step()
    for pl in plans:
        pl.sync_status(stream)

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    events = [fr.new_events() for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.wait_first()
    wall0 = time.time()
    for pl in plans:
        pl.load_bytes(reset=True)  # integral-histogram bytes the gathers request, counted by the kernels
    launches0 = S.swih_launch_count()
    t_start.record(stream)
    for s in range(args.steps):
        step(events[s])
    t_end.record(stream)
    launches = S.swih_launch_count() - launches0  # the library's own count of what it enqueued
    torch.cuda.synchronize()
    wall1 = time.time()
    clk = clocks.stop(wall0, wall1)
    if dist:
        tdist.barrier()
    ms = t_start.elapsed_time(t_end)
    for pl in plans:
        pl.sync_status(stream)
    loaded_g = plan_g.load_bytes() if plan_g else 0

    # per-launch durations inside the timed region (each gather stage is one
    # launch: the kernel's three windows), on the stream each stage runs on;
    # with two streams a stage's span includes the time it shares the GPU with
    # the other plan's stages
    seg_ms = FrameStep.stage_ms(events)

    # the same step with both plans on one stream, right after the timed region:
    # each stage alone on the GPU (the per-kernel figures beside the overlapped ones)
    solo = None
    if fr.side is not fr.stream:
        side, fr.side = fr.side, fr.stream
        n_solo = max(50, min(args.steps, 200))
        solo_ms, solo_seg, solo_loaded, _ = fr.timed(n_solo)
        fr.side = side
        solo = {"steps": n_solo, "ms_per_step": solo_ms / n_solo, "per_launch_ms": solo_seg,
                "loaded_g": solo_loaded}

    # algorithmic bytes per launch
    def ih_bytes(info, n_terms_used):
        return n_terms_used * B * H * W * info.elem_bytes

    algo = {
        # image read + bins written, every integral-histogram element written once
        "build_me": 2 * H * W + ih_bytes(info_me, info_me.n_terms) if info_me else 0,
        "build_g": 2 * H * W + ih_bytes(info_g, info_g.n_terms) if info_g else 0,
    }
    used_terms = {"manhattan": 3, "euclidean": 5, "gaussian": info_g.n_terms if info_g else 0}
    for k in kernels:  # each window reads the kernel's planes once, and writes its map
        algo[f"gather_{k}"] = sum(ih_bytes(info_g if k == "gaussian" else info_me, used_terms[k])
                                  + 4 * (H - w + 1) * (W - w + 1) for w in WINDOWS)
    # dominant kernel class by total time per step
    classes = {"ih_scan (Gaussian plan, 64-bit ring)": ["build_g"],
               "ih_scan (Manhattan+Euclidean plan, 32-bit ring)": ["build_me"],
               "gather Gaussian": ["gather_gaussian"],
               "gather Euclidean": ["gather_euclidean"],
               "gather Manhattan": ["gather_manhattan"]}
    stage_alone = solo["per_launch_ms"] if solo else seg_ms  # which kernel dominates on its own
    totals = {c: sum(stage_alone.get(k, 0.0) for k in ks) for c, ks in classes.items()}
    dom = max(totals, key=totals.get)
    dom_keys = classes[dom]
    dom_keys = [k for k in dom_keys if k in seg_ms]
    dense_bytes = float(np.mean([algo[k] for k in dom_keys]))
    dom_bytes = dense_bytes
    basis = "dense: every integral-histogram element the kernel's terms use, once, plus the map"
    maps_b = float(sum(4 * (H - w + 1) * (W - w + 1) for w in WINDOWS))
    if dom == "gather Gaussian" and loaded_g:
        # the gather skips bins and rows absent from its windows: its algorithmic
        # bytes are the row segments it must load (counted by the kernel) + the map
        dom_bytes = loaded_g / args.steps + maps_b  # one launch per step: the three windows
        basis = ("integral-histogram row segments the sparse gather loads (rows of windows holding "
                 "each bin, counted by the kernel over the timed launches) + the map")
    dom_ms = float(np.mean([seg_ms[k] for k in dom_keys]))
    peak, peak_kind = read_peaks()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    src = "k2_ih_scan.cuh" if dom.startswith("ih_scan") else "k3_tiled_kernels.cuh"
    prof = "ih_scan_gaussian_1024" if dom.startswith("ih_scan (G") else (
        "gather_gaussian_1024" if dom == "gather Gaussian" else None)
    if H != 1024 or B != 32:
        prof = None  # the committed counters are for the benchmark workload only
    traffic = profile_traffic(prof, src) if prof else None
    # the gathers (K3) alone: the step's windows over the sum of its gather
    # launches, each alone on the GPU (the one-stream pass)
    alone = solo["per_launch_ms"] if solo else seg_ms
    g_ms = sum(v for k, v in alone.items() if k.startswith("gather_"))
    gather_only = {"value": fr.windows_per_step / (g_ms * 1e-3) if g_ms else None, "unit": "windows/s",
                   "ms_per_step": g_ms,
                   "basis": ("the step's windows over the sum of its gather launches' CUDA-event times, "
                             "each launch alone on the GPU")}
    roof_solo = None
    if solo:
        s_ms = float(np.mean([solo["per_launch_ms"][k] for k in dom_keys]))
        s_bytes = dom_bytes
        if dom == "gather Gaussian" and solo["loaded_g"]:
            s_bytes = solo["loaded_g"] + maps_b
        roof_solo = {"avg_launch_ms": s_ms, "achieved": s_bytes / (s_ms * 1e-3) / 1e9,
                     "frac": s_bytes / (s_ms * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": s_bytes,
                     "steps": solo["steps"], "ms_per_step": solo["ms_per_step"],
                     "per_launch_ms": solo["per_launch_ms"],
                     "note": ("the same step with both plans on one stream, timed right after the timed "
                              "region: the kernel alone on the GPU")}

    # ---- the same step over a timed region of at least 1.5 s (>= 400 steps),
    # with the clocks sampled throughout: the sustained rate beside the K-step line
    sustained = None
    if world == 1 and not args.no_extras:
        n_sus = max(400, int(np.ceil(1500.0 / max(ms / args.steps, 1e-3))))
        sus_ms, sus_seg, _, sus_clk = fr.timed(n_sus, ClockSampler(local_rank))
        sustained = {"steps": n_sus, "timed_s": sus_ms * 1e-3, "ms_per_step": sus_ms / n_sus,
                     "value": fr.windows_per_step * n_sus / (sus_ms * 1e-3), "unit": "windows/s",
                     "per_launch_ms": sus_seg, "clocks": sus_clk}

    # ---- end to end through the C ABI from pinned host buffers. Every step
    # uploads its frame and targets and downloads its nine maps. Uploads and
    # downloads run on two copy streams of their own (so that an upload never
    # queues behind a download): a step's upload overlaps the previous step's
    # kernels, and its maps (one contiguous buffer) leave in one copy while the
    # next step computes; two device buffer sets alternate between steps, and
    # events keep every buffer from being overwritten before it is consumed.
    # The timed region opens before the first upload and closes after the last
    # download.
    sizes = [m.numel() for m in maps]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)

    def map_views(flat):
        return [flat[offs[j]: offs[j + 1]].view(m.shape) for j, m in enumerate(maps)]

    h_img = torch.from_numpy(img).pin_memory()
    h_flat = torch.empty(int(offs[-1]), dtype=torch.float32).pin_memory()
    h_maps = map_views(h_flat)
    h_targets = targets.cpu().pin_memory()
    up = torch.cuda.Stream(device=dev)
    down = torch.cuda.Stream(device=dev)
    d_imgs = [d_img, torch.empty_like(d_img)]
    d_tgts = [targets, torch.empty_like(targets)]
    d_flat = [torch.empty(int(offs[-1]), dtype=torch.float32, device=dev) for _ in range(2)]
    d_maps = [map_views(f) for f in d_flat]
    ev_in = [torch.cuda.Event() for _ in range(2)]      # set i uploaded
    ev_used = [torch.cuda.Event() for _ in range(2)]    # set i's kernels done (inputs read, maps written)
    ev_out = [torch.cuda.Event() for _ in range(2)]     # set i's maps downloaded
    for i in range(2):  # nothing pending yet
        ev_used[i].record(stream)
        ev_out[i].record(stream)

    def upload(i):
        with torch.cuda.stream(up):
            up.wait_event(ev_used[i])
            d_imgs[i].copy_(h_img, non_blocking=True)
            d_tgts[i].copy_(h_targets, non_blocking=True)
            ev_in[i].record(up)

    def compute_and_download(i):
        stream.wait_event(ev_in[i])
        stream.wait_event(ev_out[i])  # set i's maps downloaded two steps ago
        fr.run_maps(d_imgs[i], d_tgts[i], d_maps[i], stream, fr.side)
        ev_used[i].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev_used[i])
            h_flat.copy_(d_flat[i], non_blocking=True)
            ev_out[i].record(down)

    def e2e_run(n):
        upload(0)
        for n_ in range(n):
            i = n_ % 2
            compute_and_download(i)
            if n_ + 1 < n:
                upload(1 - i)
        stream.wait_stream(down)

    e2e_run(max(1, args.warmup))
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    up.wait_event(e0)
    down.wait_event(e0)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    for pl in plans:
        pl.sync_status(stream)
    bi = h_img.numel() * h_img.element_size() + h_targets.numel() * 4
    bo = sum(m.numel() * 4 for m in h_maps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:  # every step computes the same maps; compared with the oracle after the timed parts
            _ORACLE_CHECK[:] = [img, B, list(jobs), [m.numpy().copy() for m in h_maps], h_targets.numpy().copy()]
        except Exception:
            _ORACLE_CHECK[:] = []

    if dist:
        ms, e2e_ms = reduce_max_over_ranks([ms, e2e_ms])

    for pl in plans:
        pl.close()
    wps = len(kernels) * sum((H - w + 1) * (W - w + 1) for w in WINDOWS)
    rate = whole_job_rate(wps, args.steps, world, ms)
    rate_e2e = whole_job_rate(wps, args.steps, world, e2e_ms)
    if H != 1024 or B != 32 or len(kernels) != 3:
        line_note = f"profiling case {H}x{W}, B={B}, kernels {kernels}: not the benchmark workload"
    else:
        line_note = None
    line = {
        "metric": METRIC,
        "value": rate,
        "unit": "windows/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/u64-ring+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "windows_per_step_per_gpu": wps, "bins": B,
                   "image": f"{H}x{W} u8", "kernels": list(KERNELS), "window_sizes": list(WINDOWS),
                   "parallelism": f"replicas x{world} (independent frames, no collective)",
                   "streams": ("2 (Gaussian plan | Manhattan+Euclidean plan, forked and joined each step)"
                               if fr.side is not fr.stream else "1"),
                   "l2": "working set (integral histograms 7.1 GB/step) >> L2; no flush"},
        "e2e": {"value": rate_e2e, "unit": "windows/s",
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": dom_bytes,
                     "bytes_basis": basis, "dense_bytes_per_launch": dense_bytes,
                     "avg_launch_ms": dom_ms, "solo": roof_solo},
        "per_launch_ms": seg_ms,
        "step_ms": FrameStep.step_ms(events),
        "gather_only": gather_only,
        "clocks": clk,
    }
    if sustained:
        line["sustained"] = sustained
    if line_note:
        line["note"] = line_note
    return line



# ----------------------------------------------------------------------------- dense scene
def stage_bytes(fr, H, W, B):
    """Dense algorithmic bytes of each stage of one FrameStep: a build reads the
    pixels, writes the bins and every integral-histogram element of its plan
    once; a kernel's gather launch reads every element of the planes its kernel
    uses once per window and writes each window's map."""
    def ih(info, terms):
        return terms * B * H * W * info.elem_bytes

    out = {}
    if fr.info_me:
        out["build_me"] = 2 * H * W + ih(fr.info_me, fr.info_me.n_terms)
    if fr.info_g:
        out["build_g"] = 2 * H * W + ih(fr.info_g, fr.info_g.n_terms)
    used = {"manhattan": 3, "euclidean": 5, "gaussian": fr.info_g.n_terms if fr.info_g else 0}
    for k in fr.kernels:
        info = fr.info_g if k == "gaussian" else fr.info_me
        out[f"gather_{k}"] = sum(ih(info, used[k]) + 4 * (H - w + 1) * (W - w + 1) for w in fr.windows)
    return out


def run_dense_scene(args, dev):
    """The benchmark step on a frame without spatial structure: 1024x1024 u8
    pixels i.i.d. uniform over 0-255 (seed 1, the generator of the 128x128
    case), B = 32, the same kernels and windows. Every row holds nearly every
    bin and every window holds most bins, so the scans store every row and the
    gathers skip almost nothing: the worst case for the method's exact
    skipping of absent bins and rows. Timed like the main line (CUDA events,
    the two plans on two streams); the per-stage figures and the roofline come
    from the same steps run on one stream (each stage alone on the GPU) and use
    the dense bytes of each stage."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    H = W = 1024
    B = 32
    img = synth.uniform_image(H, W, 8, seed=1)
    stream = torch.cuda.Stream(device=dev)
    fr = FrameStep(S, dev, img, B, KERNELS, W // 2, H // 2, stream, streams=args.streams)
    try:
        for _ in range(max(3, args.warmup)):
            fr.step()
        steps = max(args.steps, 50)
        ms, seg_overlap, loaded_g, _ = fr.timed(steps)
        seg = seg_overlap
        if fr.side is not fr.stream:  # per-stage figures with each stage alone on the GPU
            side, fr.side = fr.side, fr.stream
            _, seg, loaded_g, _ = fr.timed(steps)
            fr.side = side
        algo = stage_bytes(fr, H, W, B)
        if not args.no_cpu_baseline:  # the last step's maps, against the oracle after the timed parts
            torch.cuda.synchronize()
            d_jobs = list(fr.jobs)
            d_maps = [m.cpu().numpy() for m in fr.maps]
            d_tgts = [t.cpu().numpy() for t in fr.targets]
            _ORACLE_LATER.append(("dense_scene", lambda: oracle_errors(
                img, B, d_jobs, d_maps, d_tgts, n=256, source="the maps of the block's last step")))
    finally:
        fr.close()
    peak, peak_kind = read_peaks()
    dom = max(seg, key=seg.get)
    stages = {k: {"ms": seg[k], "dense_bytes": algo[k], "dense_gbs": algo[k] / (seg[k] * 1e-3) / 1e9,
                  "frac_dense": algo[k] / (seg[k] * 1e-3) / 1e9 / peak} for k in seg}
    stages["gather_gaussian"]["loaded_bytes"] = loaded_g
    ach = algo[dom] / (seg[dom] * 1e-3) / 1e9
    return {
        "workload": ("1024x1024 u8 i.i.d. uniform 0-255 (seed 1), B=32, Manhattan/Euclidean/Gaussian "
                     "x windows 21/41/81, full valid maps (no spatial structure: nothing to skip)"),
        "windows_per_step": fr.windows_per_step, "steps": steps, "ms_per_step": ms / steps,
        "windows_per_s": fr.windows_per_step * steps / (ms * 1e-3),
        "per_launch_ms_overlapped": seg_overlap,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_launch": algo[dom],
                     "bytes_basis": "dense: every integral-histogram element of the stage, once, plus the maps",
                     "avg_launch_ms": seg[dom]},
        "stages": stages,
    }


# ----------------------------------------------------------------------------- small frame latency
def run_small_frame(args, dev, reps=200):
    """Latency of one small search (128x128 u8 i.i.d. frame, B = 16, one 31x31
    Manhattan map, 9,604 windows): its integral histograms fit in L2 and the
    GPU is far from full, so the figure of merit is the time per call. Device
    latency = CUDA events around build + likelihood on device-resident input;
    end-to-end latency = host time from the upload of the frame from pinned
    memory to the map copied back, synchronised per call. The map is compared
    with the FP64 oracle after the timed parts."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    cfg = synth.config1()
    img = cfg["image"]
    H, W = img.shape
    B, w = cfg["B"], cfg["windows"][0]
    tx, ty = cfg["target_centre"]
    stream = torch.cuda.Stream(device=dev)
    h_img = torch.from_numpy(img).pin_memory()
    d_img = h_img.to(dev)
    h_map = torch.empty((H - w + 1, W - w + 1), dtype=torch.float32).pin_memory()
    d_map = torch.empty((H - w + 1, W - w + 1), dtype=torch.float32, device=dev)
    q = torch.empty((1, 1, B), dtype=torch.float32, device=dev)
    dev_ms, e2e_ms = [], []
    with S.Plan(S.make_desc(H, W, bins=B, kernels=("manhattan",), max_win=(w, w))) as p:
        p.build_ih(d_img, stream)
        p.local_hist("manhattan", w, w, tx, ty, 1, 1, q, stream)  # set-up: the target window
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(reps + 10):
            e0.record(stream)
            p.build_ih(d_img, stream)
            p.likelihood("manhattan", w, w, q.reshape(B), d_map, stream)
            e1.record(stream)
            e1.synchronize()
            if i >= 10:
                dev_ms.append(e0.elapsed_time(e1))
        for i in range(reps + 10):
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                d_img.copy_(h_img, non_blocking=True)
                p.build_ih(d_img, stream)
                p.likelihood("manhattan", w, w, q.reshape(B), d_map, stream)
                h_map.copy_(d_map, non_blocking=True)
            stream.synchronize()
            if i >= 10:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
        p.sync_status(stream)
        eager_map = h_map.clone()
        # the same call (upload, build, likelihood, download) captured once into
        # a CUDA graph and replayed: one launch per call instead of six
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
            d_img.copy_(h_img, non_blocking=True)
            p.build_ih(d_img, stream)
            p.likelihood("manhattan", w, w, q.reshape(B), d_map, stream)
            h_map.copy_(d_map, non_blocking=True)
        g_dev, g_e2e = [], []
        for i in range(reps + 10):
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):  # replay() launches on the current stream
                e0.record(stream)
                graph.replay()
                e1.record(stream)
            stream.synchronize()
            if i >= 10:
                g_e2e.append((time.perf_counter() - t0) * 1e3)
                g_dev.append(e0.elapsed_time(e1))
        # one more replay into cleared maps: it recomputes and copies the map
        d_map.fill_(-1.0)
        h_map.fill_(-1.0)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            graph.replay()
        stream.synchronize()
        p.sync_status(stream)
        graph_equal = bool(torch.equal(h_map, eager_map))
        del graph
        target = q.reshape(B).cpu().numpy().astype(np.float64)
    out = {
        "workload": "128x128 u8 i.i.d. uniform (seed 1), B=16, one 31x31 Manhattan map (9,604 windows)",
        "reps": reps,
        "device_latency_ms": {"p50": float(np.percentile(dev_ms, 50)), "p99": float(np.percentile(dev_ms, 99))},
        "e2e_latency_ms": {"p50": float(np.percentile(e2e_ms, 50)), "p99": float(np.percentile(e2e_ms, 99)),
                           "h2d_bytes": H * W, "d2h_bytes": h_map.numel() * 4},
        "graph_replay_ms": {"device_p50": float(np.percentile(g_dev, 50)),
                            "device_p99": float(np.percentile(g_dev, 99)),
                            "e2e_p50": float(np.percentile(g_e2e, 50)), "e2e_p99": float(np.percentile(g_e2e, 99)),
                            "map_equals_eager": graph_equal,
                            "note": "upload + build + likelihood + download captured into one CUDA graph"},
        "windows_per_call": h_map.numel(),
    }
    if not args.no_cpu_baseline:
        _ORACLE_LATER.append(("small_frame", lambda: small_frame_error(img, B, w, target, h_map.numpy().copy())))
    return out


def small_frame_error(img, B, w, target, got):
    """Largest |GPU - oracle| over the whole 128x128 map (FP64 brute force)."""
    from oracle import swih_oracle as O

    bins = O.quantize(img, 8, B)
    ref = O.likelihood_map(bins, B, O.kernel_weights("manhattan", w, w), target)
    return {"max_abs": float(np.abs(got.astype(np.float64) - ref).max()), "tolerance": 1e-5,
            "sample": "every valid centre"}

# ----------------------------------------------------------------------------- batches
def run_regions(args, dev, per_region=True):
    """64 search regions of 96-768 px from a 4096x4096 u16 frame (B = 64,
    Gaussian, 3 scales): one batch (CUDA graph: one quantise, one scan, one
    gather launch per job group) against one plan per region (its own
    quantise, scan and three gathers), each timed with CUDA events over
    whole steps. per_region = False leaves out the per-region plans (a short
    run that profiles the batch alone)."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    cfg = synth.config3()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    d_img = torch.from_numpy(img.view(np.int16)).to(dev)
    ptr, pitch = d_img.data_ptr(), W * 2
    stream = torch.cuda.Stream(device=dev)
    rois, wins = cfg["rois"], cfg["windows"]
    wps = sum((w - k + 1) * (h - k + 1) for (_, _, w, h), ks in zip(rois, wins) for k in ks)
    maps = [[torch.empty((h - k + 1, w - k + 1), device=dev) for k in ks] for (_, _, w, h), ks in zip(rois, wins)]
    targets = torch.empty((len(rois), B), device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(3, min(args.steps, 10))

    # one plan per region; targets = each region's object window at scale 1 (set-up)
    plans = []
    for i, ((x0, y0, w, h), ks, (ox, oy)) in enumerate(zip(rois, wins, cfg["object_centres"])):
        if not per_region:
            targets[i].fill_(1.0 / B)
            continue
        p = S.Plan(S.make_desc(h, w, pitch_bytes=pitch, pixel_type=S.SWIH_PIXEL_U16, bitdepth=16, bins=B,
                               kernels=("gaussian",), max_win=(max(ks), max(ks))))
        p.build_ih(ptr + y0 * pitch + x0 * 2, stream)
        r = ks[1] // 2
        p.local_hist("gaussian", ks[1], ks[1], min(max(ox - x0, r), w - 1 - r), min(max(oy - y0, r), h - 1 - r),
                     1, 1, targets[i], stream)
        plans.append(p)

    def per_roi_step():
        for p, (x0, y0, w, h), ks, ms, i in zip(plans, rois, wins, maps, range(len(rois))):
            p.build_ih(ptr + y0 * pitch + x0 * 2, stream)
            for k, m in zip(ks, ms):
                p.likelihood("gaussian", k, k, targets[i], m, stream)

    per_roi_ms = float("nan")
    if per_region:
        for _ in range(2):
            per_roi_step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            per_roi_step()
        e1.record(stream)
        torch.cuda.synchronize()
        per_roi_ms = e0.elapsed_time(e1) / steps
    for p in plans:
        p.sync_status(stream)
        p.close()
    ref = [[m.clone() for m in ms] for ms in maps]
    plans = None
    torch.cuda.empty_cache()

    desc = S.make_batch_desc(H, W, pitch_bytes=pitch, pixel_type=S.SWIH_PIXEL_U16, bitdepth=16, bins=B,
                             kernels=("gaussian",))
    rl = [S.make_roi(x0, y0, w, h, "gaussian", [(k, k) for k in ks], targets[i], ms)
          for i, ((x0, y0, w, h), ks, ms) in enumerate(zip(rois, wins, maps))]
    ws_bytes = S.swih_batch_workspace_bytes(desc, rl)
    with S.Batch(desc, rl, ptr) as b:
        b.autotune(stream)
        for _ in range(2):
            b.run(stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            b.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        b.sync_status(stream)
        batch_ms = e0.elapsed_time(e1) / steps
    diff = (max((m - r).abs().max().item() for ms, rs in zip(maps, ref) for m, r in zip(ms, rs))
            if per_region else None)
    if per_region and not args.no_cpu_baseline:
        # sampled centres of every (region, scale) map, copied back for the oracle
        rng = np.random.default_rng(13)
        samples = []
        for i, ((x0, y0, w, h), ks, ms) in enumerate(zip(rois, wins, maps)):
            for k, m in zip(ks, ms):
                r = (k - 1) // 2
                cx = rng.integers(r, w - r, 64)
                cy = rng.integers(r, h - r, 64)
                idx = torch.from_numpy((cy - r) * (w - k + 1) + (cx - r)).to(dev)
                samples.append((i, k, cx, cy, m.reshape(-1)[idx].cpu().numpy()))
        tg = targets.cpu().numpy().astype(np.float64)
        _ORACLE_LATER.append(("batched_regions", lambda: regions_error(img, B, rois, samples, tg)))
    del maps, ref
    torch.cuda.empty_cache()
    return {
        "workload": ("64 regions of U{96..768}^2 px from a 4096x4096 u16 frame, B=64, Gaussian "
                     "(sigma=w/4), 3 scales 0.8/1/1.25 x a 24-64 px box, full valid maps"),
        "windows_per_step": wps, "steps": steps,
        "batch": {"ms_per_step": batch_ms, "windows_per_s": wps / (batch_ms * 1e-3),
                  "launches_per_step": "1 quantise + 1 scan + 1 gather per job group (graph replay)",
                  "workspace_gb": ws_bytes / 1e9},
        "per_region_plans": {"ms_per_step": per_roi_ms, "windows_per_s": wps / (per_roi_ms * 1e-3) if per_region else None,
                             "launches_per_step": 6 * len(rois)},
        "speedup": per_roi_ms / batch_ms if per_region else None,
        "max_abs_diff_batch_vs_per_region": diff,
    }


# ----------------------------------------------------------------------------- large frame
def run_large_frame(args, dev, budget_gb=100, passes=3):
    """8192x8192 u16 frame, B = 64, Gaussian and Euclidean kernels at windows
    15/25/43/75/127: the integral histograms (25 terms, 64-bit) would need
    ~860 GB, so the frame is streamed in bands within budget_gb of device
    memory; one pass = every band's quantise + scan + 10 gathers (CUDA graph).

    Reported: windows/s of the graph replay (CUDA events, inputs resident);
    per-stage times of one pass launched stage by stage with events between
    stages, and the roofline of the dominant stage (bytes the gathers loaded,
    counted by the kernels, or the scan's dense bytes); an end-to-end rate
    with the frame uploaded from pinned host memory and all ten maps copied
    back every pass; and the largest |GPU - oracle| over a 512x512 block of
    centres that straddles the first band boundary (after the timed parts)."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    cfg = synth.config4()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    h_img = torch.from_numpy(img.view(np.int16)).pin_memory()
    d_img = h_img.to(dev)
    stream = torch.cuda.Stream(device=dev)
    n_jobs = len(cfg["kernels"]) * len(cfg["windows"])
    g = torch.Generator(device="cpu").manual_seed(4)
    tgt = (torch.rand((n_jobs, B), generator=g) + 0.01).to(dev)
    tgt /= tgt.sum(1, keepdim=True)  # targets: positive normalised histograms (set-up)
    jobs, maps, job_kw = [], [], []
    for k in cfg["kernels"]:
        for w in cfg["windows"]:
            m = torch.empty((H - w + 1, W - w + 1), device=dev)
            jobs.append(S.make_frame_job(k, w, w, tgt[len(maps)], m))
            maps.append(m)
            job_kw.append((k, w))
    wpp = sum(m.numel() for m in maps)
    desc = S.make_desc(H, W, pixel_type=S.SWIH_PIXEL_U16, bitdepth=16, bins=B, kernels=cfg["kernels"],
                       max_win=(127, 127), hbm_budget_bytes=budget_gb << 30)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h_maps = [torch.empty(m.shape, dtype=torch.float32).pin_memory() for m in maps]
    with S.Stream(desc, jobs, d_img) as st:
        info = st.info()
        st.run(stream)
        st.sync_status(stream)
        st.load_bytes(reset=True)
        e0.record(stream)
        for _ in range(passes):
            st.run(stream)
        e1.record(stream)
        st.sync_status(stream)
        ms = e0.elapsed_time(e1) / passes
        loaded = {k: v / passes for k, v in st.load_bytes(reset=True).items() if v}
        stages = st.run_timed(stream)
        st.sync_status(stream)
        # end to end: frame up from pinned memory, the pass with every map's
        # rows copied back band by band as each band completes (the pass's
        # own host copies, beside the next band's work); one untimed pass first
        st.set_host_maps(h_maps)

        def e2e_pass():
            with torch.cuda.stream(stream):
                d_img.copy_(h_img, non_blocking=True)
                st.run(stream)

        e2e_pass()
        st.sync_status(stream)
        e2e_passes = 2
        e0.record(stream)
        for _ in range(e2e_passes):
            e2e_pass()
        e1.record(stream)
        st.sync_status(stream)
        e2e_ms = e0.elapsed_time(e1) / e2e_passes
    # dense bytes of a pass: each band region's planes once per job (gathers),
    # every element of the band's planes written once (scan)
    R, Hb, nb = 63, info["band_height"], info["n_bands"]
    rows = [(H if k == nb - 1 else min(H, (k + 1) * Hb + 2 * R)) - k * Hb for k in range(nb)]
    terms = {"gaussian": 25, "euclidean": 5}
    dense = {"scan": sum(r * W * (2 + 1 + 25 * B * 8) for r in rows)}
    for k in cfg["kernels"]:
        dense[k] = sum(len(cfg["windows"]) * terms[k] * B * r * W * 8 for r in rows)
    peak, peak_kind = read_peaks()
    dom = max(stages, key=stages.get)
    if dom in loaded:
        dom_bytes, basis = loaded[dom] + 4.0 * sum(
            m.numel() for (k, _), m in zip(job_kw, maps) if k == dom), (
            "integral-histogram row segments the gathers of this kernel loaded over all bands "
            "(counted by the kernels) + the maps")
    else:
        dom_bytes, basis = dense[dom], "dense: every element of every band's planes written once, plus pixels and bins"
    ach = dom_bytes / (stages[dom] * 1e-3) / 1e9
    out = {
        "workload": ("8192x8192 u16 fractal terrain + 200 blobs, B=64, Gaussian + Euclidean x windows "
                     "15/25/43/75/127, full valid maps, streamed in bands"),
        "windows_per_pass": wpp, "ms_per_pass": ms, "windows_per_s": wpp / (ms * 1e-3), "passes": passes,
        "band_height": Hb, "n_bands": nb,
        "workspace_gb": info["workspace_bytes"] / 1e9,
        "halo_rows_per_band": 2 * R,
        "whole_frame_ih_gb": 25 * B * H * W * 8 / 1e9,
        "stage_ms_per_pass": stages,
        "loaded_bytes_per_pass": loaded, "dense_bytes_per_pass": dense,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_launch": dom_bytes,
                     "bytes_basis": basis, "launch": "one pass, summed over bands (stage by stage)",
                     "avg_launch_ms": stages[dom]},
        "e2e": {"value": wpp / (e2e_ms * 1e-3), "unit": "windows/s", "ms_per_pass": e2e_ms,
                "h2d_bytes_per_step": h_img.numel() * 2, "d2h_bytes_per_step": sum(m.numel() * 4 for m in h_maps)},
    }
    if not args.no_cpu_baseline:
        rng = np.random.default_rng(4)
        bx = int(rng.integers(R, W - R - 512))
        by = max(R, min(H - R - 512, R + Hb - 256))  # rows on both sides of the first band boundary
        sub = img[by - R: by + 512 + R, bx - R: bx + 512 + R].copy()
        blocks = [hm.numpy()[by - (w - 1) // 2: by - (w - 1) // 2 + 512, bx - (w - 1) // 2: bx - (w - 1) // 2 + 512].copy()
                  for hm, (_, w) in zip(h_maps, job_kw)]
        targets = tgt.cpu().numpy().astype(np.float64)
        _ORACLE_LATER.append(("large_frame", lambda: large_frame_error(sub, B, job_kw, targets, blocks, bx, by, R)))
    del maps, h_maps
    torch.cuda.empty_cache()
    return out


def large_frame_error(sub, B, job_kw, targets, blocks, bx, by, R, n=512):
    """Largest |GPU - oracle| per map over an n x n block of centres; sub is
    the frame's pixels around the block (an R-pixel halo on every side) and
    blocks[j] the GPU's values of map j at those centres."""
    from oracle import swih_oracle as O

    bins = O.quantize(sub, 16, B)
    per = {}
    for j, ((k, w), got) in enumerate(zip(job_kw, blocks)):
        ref = O.likelihood_rect(bins, B, O.kernel_weights(k, w, w), targets[j], R, R, n, n)
        per[f"{k}_{w}"] = float(np.abs(got.astype(np.float64) - ref).max())
    return {"max_abs": max(per.values()), "tolerance": 1e-5, "per_map": per,
            "sample": (f"{n}x{n} centres at x {bx}..{bx + n - 1}, y {by}..{by + n - 1} (across the first band "
                       "boundary), every map, FP64 brute force with the targets the GPU used")}


# ----------------------------------------------------------------------------- exponential kernel
CHANNEL_BINS = (16, 16, 16)


def run_channels(args, dev, steps=50):
    """Feature channels (Sec. 4: one likelihood map per feature): three
    features of the benchmark frame (the 1024x1024 u8 scene at 16 bins, a
    12-bit texture-like u16 channel at 16 bins and a 6-bit u8 channel at 16
    bins; synth.feature_channels), Manhattan/Euclidean/Gaussian at windows
    21/41/81. One step = both channel plans' builds (K1 per channel, one K2
    over all 48 bins; the Manhattan+Euclidean plan on a second stream as in the
    main step) + 9 gathers, each writing the three channels' maps in one
    launch. Targets: each channel's window at the object (per-channel
    normalised, set up untimed). Counted: (centre, window, channel) triples."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    cfg = synth.config2()
    img = cfg["image"]
    H, W = img.shape
    tx, ty = cfg["target_centre"]
    feats = synth.feature_channels(img, seed=12)
    bufs, chans = [], []
    for (a, bd), B in zip(feats, CHANNEL_BINS):
        u16 = a.dtype == np.uint16
        bufs.append(torch.from_numpy(a.view(np.int16) if u16 else a).to(dev))
        chans.append(S.make_channel(W, pixel_type=S.SWIH_PIXEL_U16 if u16 else S.SWIH_PIXEL_U8, bitdepth=bd,
                                    bins=B))
    ptrs = [b.data_ptr() for b in bufs]
    C, Bt = len(chans), sum(CHANNEL_BINS)
    stream = torch.cuda.Stream(device=dev)
    side = torch.cuda.Stream(device=dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()
    plans = {"me": S.ChannelPlan(S.make_desc(H, W, bins=1, kernels=("manhattan", "euclidean"), max_win=(81, 81)),
                                 chans),
             "g": S.ChannelPlan(S.make_desc(H, W, bins=1, kernels=("gaussian",), max_win=(81, 81)), chans)}
    jobs = [(k, w) for k in KERNELS for w in WINDOWS]
    plan_of = {"manhattan": "me", "euclidean": "me", "gaussian": "g"}
    try:
        for pl in plans.values():
            pl.build_ih(ptrs, stream)
        targets = torch.empty((len(jobs), Bt), device=dev)
        for j, (k, w) in enumerate(jobs):
            plans[plan_of[k]].local_hist(k, w, w, tx, ty, 1, 1, targets[j], stream)
        maps = [torch.empty((C, H - w + 1, W - w + 1), device=dev) for _, w in jobs]

        def step():
            fork.record(stream)
            side.wait_event(fork)
            for name, st in (("me", side), ("g", stream)):
                plans[name].build_ih(ptrs, st)
                for j, (k, w) in enumerate(jobs):
                    if plan_of[k] == name:
                        plans[name].likelihood_channels(k, w, w, targets[j], maps[j], st)
            join.record(side)
            stream.wait_event(join)

        for _ in range(max(3, args.warmup)):
            step()
        for pl in plans.values():
            pl.sync_status(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        for pl in plans.values():
            pl.sync_status(stream)
        n_win = sum(m.numel() for m in maps)
        out = {"workload": ("1024x1024 benchmark scene as 3 feature channels (u8 8-bit, u16 12-bit, u8 6-bit; "
                            "16 bins each), Manhattan/Euclidean/Gaussian x windows 21/41/81, one map per "
                            "channel"),
               "channels": C, "bins": list(CHANNEL_BINS), "windows_per_step": n_win, "steps": steps,
               "ms_per_step": ms, "windows_per_s": n_win / (ms * 1e-3),
               "launches_per_step": "K1 per channel and one K2 per plan; one gather per (kernel, window)"}
        if not args.no_cpu_baseline:
            rng = np.random.default_rng(14)
            samples = []
            for j, (k, w) in enumerate(jobs):
                r = w // 2
                cx = rng.integers(r, W - r, 128)
                cy = rng.integers(r, H - r, 128)
                got = maps[j][:, torch.from_numpy(cy - r).to(dev), torch.from_numpy(cx - r).to(dev)].cpu().numpy()
                samples.append((k, w, cx, cy, got, targets[j].cpu().numpy().astype(np.float64)))
            feats_np = [(a, bd) for a, bd in feats]
            _ORACLE_LATER.append(("channels", lambda: channels_error(feats_np, samples)))
    finally:
        for pl in plans.values():
            pl.close()
    return out


def channels_error(feats, samples):
    """Largest |GPU - oracle| over 128 sampled centres of every (kernel, window,
    channel) map, each channel scored over its own bins against its slice of
    the target the GPU used."""
    from oracle import swih_oracle as O

    bins = [O.quantize(a, bd, B) for (a, bd), B in zip(feats, CHANNEL_BINS)]
    worst, n = 0.0, 0
    for k, w, cx, cy, got, q in samples:
        K = O.kernel_weights(k, w, w)
        off = 0
        for c, B in enumerate(CHANNEL_BINS):
            ref = O.likelihood_at(bins[c], B, K, q[off:off + B], cx, cy)
            worst = max(worst, float(np.abs(got[c].astype(np.float64) - ref).max()))
            n += cx.size
            off += B
    return {"max_abs": worst, "tolerance": 1e-5,
            "sample": f"{n} centres: 128 random valid centres of every (kernel, window, channel) map, FP64 brute force"}


def run_exponential(args, dev, lam=0.1, steps=50):
    """The exponential kernel exp(-lambda (|dx| + |dy|)), lambda = 0.1 per pixel,
    on the benchmark frame (1024x1024 u8, B = 32) at windows 21/41/81. One step =
    quantise + the plain integral histogram (the count gate) + the four
    directional tables + the 3 likelihood maps, timed with CUDA events; the
    tables (1.2 GB) exceed L2."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    cfg = synth.config2()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    tx, ty = cfg["target_centre"]
    d_img = torch.from_numpy(img).to(dev)
    stream = torch.cuda.Stream(device=dev)
    desc = S.make_desc(H, W, bins=B, kernels=("exponential",), max_win=(81, 81), exp_lambda=lam)
    maps = {w: torch.empty((H - w + 1, W - w + 1), device=dev) for w in WINDOWS}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 + len(WINDOWS))]
    with S.Plan(desc) as p:
        p.build_ih(d_img, stream)
        tgt = torch.empty((1, 1, B), device=dev)  # set-up: the target is the window at the object
        p.local_hist("exponential", 41, 41, tx, ty, 1, 1, tgt, stream)
        q = tgt.reshape(B)
        for _ in range(3):
            p.build_ih(d_img, stream)
            for w in WINDOWS:
                p.likelihood("exponential", w, w, q, maps[w], stream)
        t_build, t_map = 0.0, {w: 0.0 for w in WINDOWS}
        for _ in range(steps):
            ev[0].record(stream)
            p.build_ih(d_img, stream)
            ev[1].record(stream)
            for i, w in enumerate(WINDOWS):
                p.likelihood("exponential", w, w, q, maps[w], stream)
                ev[2 + i].record(stream)
            torch.cuda.synchronize()
            t_build += ev[0].elapsed_time(ev[1])
            prev = ev[1]
            for i, w in enumerate(WINDOWS):
                t_map[w] += prev.elapsed_time(ev[2 + i])
                prev = ev[2 + i]
        p.sync_status(stream)
        info = p.info()
        if not args.no_cpu_baseline:  # the last step's maps, against the oracle after the timed parts
            e_maps = [maps[w].cpu().numpy() for w in WINDOWS]
            e_q = q.cpu().numpy()
            _ORACLE_LATER.append(("exponential", lambda: oracle_errors(
                img, B, [("exponential", w) for w in WINDOWS], e_maps, [e_q] * len(WINDOWS), n=256,
                source="the maps of the block's last step")))
    build = t_build / steps
    gathers = {w: t / steps for w, t in t_map.items()}
    step_ms = build + sum(gathers.values())
    n_win = sum(m.numel() for m in maps.values())
    pitch = info.ih_pitch
    written = 4 * B * H * pitch * 8 + B * H * pitch * info.elem_bytes  # tables + count plane
    peak = read_peaks()[0]
    return {
        "workload": ("1024x1024 u8 benchmark frame, B=32, exponential kernel exp(-0.1 (|dx|+|dy|)) "
                     "x windows 21/41/81, full valid maps"),
        "windows_per_step": n_win, "ms_per_step": step_ms, "windows_per_s": n_win / (step_ms * 1e-3),
        "build_ms": build, "gather_ms": {str(w): v for w, v in gathers.items()},
        "build_bytes_written": written, "build_gbs": written / (build * 1e-3) / 1e9,
        "build_frac_of_copy_peak": written / (build * 1e-3) / 1e9 / peak,
        "steps": steps,
    }


def run_exp_profile():
    """A small exponential-kernel run to capture under ncu: the benchmark frame
    with B = 8 (268 MB of tables, above L2), two builds and two w = 41 maps."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    dev = torch.device("cuda", 0)
    img = synth.config2()["image"]
    H, W = img.shape
    B = 8
    d_img = torch.from_numpy(img).to(dev)
    q = torch.full((B,), 1.0 / B, device=dev)
    m = torch.empty((H - 40, W - 40), device=dev)
    with S.Plan(S.make_desc(H, W, bins=B, kernels=("exponential",), max_win=(81, 81), exp_lambda=0.1)) as p:
        for _ in range(2):
            p.build_ih(d_img)
            p.likelihood("exponential", 41, 41, q, m)
        p.sync_status()
    print(json.dumps({"exp_profile": "ok", "bins": B}), flush=True)


def run_wide_profile(degree=3, w=151, timed=False):
    """A small run of the any-degree Gaussian gather to capture under ncu: the
    benchmark frame with B = 8, a degree-3 plan at a 151 px window (128-bit
    ring), two builds and two maps."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    dev = torch.device("cuda", 0)
    img = synth.config2()["image"]
    H, W = img.shape
    B = 8
    d_img = torch.from_numpy(img).to(dev)
    q = torch.full((B,), 1.0 / B, device=dev)
    m = torch.empty((H - w + 1, W - w + 1), device=dev)
    desc = S.make_desc(H, W, bins=B, kernels=("gaussian",), max_win=(w, w), gauss_degree=degree)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with S.Plan(desc) as p:
        for _ in range(2):
            p.build_ih(d_img)
            p.likelihood("gaussian", w, w, q, m)
        p.sync_status()
        elem = p.info().elem_bytes
        if timed:
            e0.record()
            for _ in range(5):
                p.likelihood("gaussian", w, w, q, m)
            e1.record()
            p.sync_status()
    out = {"wide_profile": "ok", "bins": B, "degree": degree, "window": w, "ring_bits": 8 * elem}
    if timed:
        out["gather_ms"] = e0.elapsed_time(e1) / 5
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- serving
def run_serving(args, dev, n_queries=400, rate=2000.0):
    """A Poisson stream of tracking queries against 16 resident 2048x2048
    frames: the server (continuous batching) against the plain path (one plan
    per query, processed one at a time in arrival order). Latency = completion
    - arrival (host monotonic clock); the same stream and arrival times for
    both."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    frames = synth.config5_frames()
    qs = synth.config5_queries(n=n_queries, rate=rate)
    d_frames = [torch.from_numpy(img if img.dtype == np.uint8 else img.view(np.int16)).to(dev) for img, _ in frames]
    targets = [torch.from_numpy(q["targets"]).to(dev) for q in qs]

    def n_eval(q):
        return len(q["targets"]) * sum((q["h"] - h + 1) * (q["w"] - w + 1) for w, h in q["windows"])

    total = sum(n_eval(q) for q in qs)
    outs = [torch.empty(n_eval(q), device=dev) for q in qs]
    torch.cuda.synchronize()

    def stats(lat_ms, span_s):
        return {"queries_per_s": len(lat_ms) / span_s, "windows_per_s": total / span_s,
                "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "span_s": span_s}

    srv_cfg = dict(hbm_budget_bytes=96 << 30, max_inflight=8, max_batch_queries=8, merge_regions=True,
                   keep_ih=True)

    def serve_stream(srv, qq):
        t0 = time.monotonic_ns()
        arrival = []
        for i, q in enumerate(qs):
            a = t0 + int(q["t"] * 1e9)
            while time.monotonic_ns() < a:
                pass
            arrival.append(a)
            srv.submit(qq[i])
        srv.drain()
        comps = srv.poll(n_queries + 16)
        lat = [(c.done_ns - arrival[c.user_tag]) / 1e6 for c in comps]
        out = stats(lat, (max(c.done_ns for c in comps) - t0) / 1e9)
        out.update({"mean_queries_per_micro_batch": float(np.mean([c.batch_queries for c in comps])),
                    "failed": sum(c.status != 0 for c in comps),
                    "ih_reused_fraction": float(np.mean([c.ih_reused for c in comps]))})
        return out

    with S.Server(**srv_cfg) as srv:
        ids = []
        for (img, bd), d in zip(frames, d_frames):
            pt = S.SWIH_PIXEL_U8 if img.dtype == np.uint8 else S.SWIH_PIXEL_U16
            ids.append(srv.add_frame(d, img.shape[0], img.shape[1], pixel_type=pt, bitdepth=bd))
        qq = [S.make_query(ids[q["frame"]], q["x0"], q["y0"], q["w"], q["h"], q["B"], q["kernel"], q["windows"],
                           targets[i], outs[i], n_targets=len(q["targets"]), user_tag=i) for i, q in enumerate(qs)]
        for i in range(8):  # warm-up
            srv.submit(qq[i])
        srv.drain()
        srv.poll(64)
        for f in ids:  # the stream starts with nothing resident
            srv.frame_changed(f)
        server = serve_stream(srv, qq)
        server["config"] = {k: v for k, v in srv_cfg.items()}
        server["ih_stats"] = srv.stats()
        # the same stream again over the unchanged frames: integral histograms resident
        warm = serve_stream(srv, qq)
        warm["ih_stats"] = srv.stats()
    server_out = [o.clone() for o in outs]
    if not args.no_cpu_baseline:
        rng = np.random.default_rng(17)
        samples = []
        for i, q in enumerate(qs):
            off = 0
            for t in range(len(q["targets"])):
                for (w, h) in q["windows"]:
                    nx, ny = q["w"] - w + 1, q["h"] - h + 1
                    cx = rng.integers(0, nx, 16)
                    cy = rng.integers(0, ny, 16)
                    idx = torch.from_numpy(off + cy * nx + cx).to(dev)
                    samples.append((i, t, w, h, cx + (w - 1) // 2, cy + (h - 1) // 2,
                                    server_out[i][idx].cpu().numpy()))
                    off += nx * ny
        _ORACLE_LATER.append(("serving", lambda: serving_error(frames, qs, samples)))

    stream = torch.cuda.Stream(device=dev)
    lat = []
    t0 = time.monotonic_ns()
    for i, q in enumerate(qs):
        a = t0 + int(q["t"] * 1e9)
        while time.monotonic_ns() < a:
            pass
        img, bd = frames[q["frame"]]
        pb = img.dtype.itemsize
        W = img.shape[1]
        mw = max(w for w, _ in q["windows"])
        desc = S.make_desc(q["h"], q["w"], pitch_bytes=W * pb, pixel_type=S.SWIH_PIXEL_U8 if pb == 1 else S.SWIH_PIXEL_U16,
                           bitdepth=bd, bins=q["B"], kernels=(q["kernel"],), max_win=(mw, mw))
        with S.Plan(desc) as p:
            p.build_ih(d_frames[q["frame"]].data_ptr() + (q["y0"] * W + q["x0"]) * pb, stream)
            off = 0
            for t in range(len(q["targets"])):
                for (w, h) in q["windows"]:
                    p.likelihood(q["kernel"], w, h, targets[i][t], outs[i].data_ptr() + 4 * off, stream)
                    off += (q["h"] - h + 1) * (q["w"] - w + 1)
            p.sync_status(stream)
        lat.append((time.monotonic_ns() - a) / 1e6)
    plain = stats(lat, (time.monotonic_ns() - t0) / 1e9)
    diff = max((a - b).abs().max().item() for a, b in zip(outs, server_out))
    repeats = run_serving_repeats(S, synth, dev, frames, d_frames, stats_fn=stats)
    return {
        "workload": (f"{n_queries} queries, Poisson {rate:.0f}/s, 16 resident 2048x2048 u8/u16 frames, crops "
                     "U{64..1024}^2, B in {16,32,64}, M/E/G kernel, 1-8 targets, 1-5 windows of "
                     "15/25/43/75/127"),
        "windows_per_query_mean": total / n_queries,
        "server": server, "server_warm_replay": warm, "plain_per_query": plain,
        "p99_ratio_plain_over_server": plain["p99_ms"] / server["p99_ms"],
        "throughput_ratio_server_over_plain": server["queries_per_s"] / plain["queries_per_s"],
        "max_abs_diff_server_vs_plain": diff,
        "revisited_regions": repeats,
    }


def run_serving_repeats(S, synth, dev, frames, d_frames, stats_fn):
    """A stream that comes back to the same search regions (80 regions on the
    16 resident frames, 5 queries each, Poisson 2000/s), served with the
    integral histograms kept resident between micro-batches and without: the
    hit rate, latency and throughput of each, and the largest difference
    between their maps (0: the integer integral histograms are exact)."""
    import torch

    qs = synth.config5_repeat_queries()

    def n_eval(q):
        return len(q["targets"]) * sum((q["h"] - h + 1) * (q["w"] - w + 1) for w, h in q["windows"])

    targets = [torch.from_numpy(q["targets"]).to(dev) for q in qs]
    res, outs_by = {}, {}
    for keep in (True, False):
        outs = [torch.empty(n_eval(q), device=dev) for q in qs]
        cfg = dict(hbm_budget_bytes=96 << 30, max_inflight=8, max_batch_queries=8, merge_regions=True,
                   keep_ih=keep)
        with S.Server(**cfg) as srv:
            ids = []
            for (img, bd), d in zip(frames, d_frames):
                pt = S.SWIH_PIXEL_U8 if img.dtype == np.uint8 else S.SWIH_PIXEL_U16
                ids.append(srv.add_frame(d, img.shape[0], img.shape[1], pixel_type=pt, bitdepth=bd))
            qq = [S.make_query(ids[q["frame"]], q["x0"], q["y0"], q["w"], q["h"], q["B"], q["kernel"],
                               q["windows"], targets[i], outs[i], n_targets=len(q["targets"]), user_tag=i)
                  for i, q in enumerate(qs)]
            for i in range(8):  # warm-up, then nothing resident
                srv.submit(qq[i])
            srv.drain()
            srv.poll(64)
            for f in ids:
                srv.frame_changed(f)
            t0 = time.monotonic_ns()
            arrival = []
            for i, q in enumerate(qs):
                a = t0 + int(q["t"] * 1e9)
                while time.monotonic_ns() < a:
                    pass
                arrival.append(a)
                srv.submit(qq[i])
            srv.drain()
            comps = srv.poll(len(qs) + 16)
            st = stats_fn([(c.done_ns - arrival[c.user_tag]) / 1e6 for c in comps],
                          (max(c.done_ns for c in comps) - t0) / 1e9)
            st.update({"ih_reused_fraction": float(np.mean([c.ih_reused for c in comps])),
                       "failed": sum(c.status != 0 for c in comps), "ih_stats": srv.stats()})
            # windows/s of this stream (the stats helper's figure is the main stream's)
            st["windows_per_s"] = sum(n_eval(q) for q in qs) / st["span_s"]
        res["resident_ih" if keep else "rebuilt_each_micro_batch"] = st
        outs_by[keep] = outs
    res["max_abs_diff"] = max((a - b).abs().max().item() for a, b in zip(outs_by[True], outs_by[False]))
    res["workload"] = ("400 queries, Poisson 2000/s: 80 search regions (U{256..512}^2, B in {16,32}, "
                       "Manhattan/Euclidean) on the 16 resident frames, each queried 5 times in random order, "
                       "1-4 targets, 1-3 windows of 15/25/43/75/127")
    return res


# ----------------------------------------------------------------------------- Fig. 6
FIG6_KINDS = (("manhattan", 2), ("euclidean", 2), ("gaussian", 2), ("gaussian", 3), ("exponential", 2))
FIG6_WINDOWS = (11, 21, 41, 61, 81, 121, 161, 201, 301, 401)


def run_fig6(args, frames=((480, 640), (1024, 1024)), cpu=True, reps=10):
    """Time per likelihood map against window size (the experiment of Fig. 6):
    SWIH on the GPU (quantise + integral histograms + gather, CUDA events, and
    the gather alone) for the Manhattan, Euclidean, Gaussian (degree 2 and 3)
    and exponential kernels, and with cpu the brute-force oracle on the host
    cores (timed on a sample of centres and scaled to the whole map), on
    frames of the benchmark's scene generator, B = 32. Gaussian windows whose
    exact moments pass 2^64 use the 128-bit ring and the any-degree gather."""
    import torch

    from paper_1705_03524_gb300 import swih as S
    from paper_1705_03524_gb300 import synth

    if cpu:
        from oracle import swih_oracle as O
        O.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    B = 32
    rows = []
    for (H, W) in frames:
        sc = synth.blob_scene(H, W, 8, seed=2, n_blobs=8)
        img = sc.image
        d_img = torch.from_numpy(img).to(dev)
        bins = O.quantize(img, 8, B) if cpu else None
        for kind, degree in FIG6_KINDS:
            for w in (w for w in FIG6_WINDOWS if w < min(H, W)):
                desc = S.make_desc(H, W, bins=B, kernels=(kind,), max_win=(w, w), gauss_degree=degree)
                with S.Plan(desc) as p:
                    elem = p.info().elem_bytes
                    q = torch.full((B,), 1.0 / B, device=dev)
                    m = torch.empty((H - w + 1, W - w + 1), device=dev)
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    for _ in range(3):
                        p.build_ih(d_img, stream)
                        p.likelihood(kind, w, w, q, m, stream)
                    t_all, t_g = 0.0, 0.0
                    for _ in range(reps):
                        ev[0].record(stream)
                        p.build_ih(d_img, stream)
                        ev[1].record(stream)
                        p.likelihood(kind, w, w, q, m, stream)
                        ev[2].record(stream)
                        torch.cuda.synchronize()
                        t_all += ev[0].elapsed_time(ev[2])
                        t_g += ev[1].elapsed_time(ev[2])
                    p.sync_status(stream)
                n_c = (H - w + 1) * (W - w + 1)
                row = {"frame": f"{W}x{H}", "kernel": kind if kind != "gaussian" else f"gaussian_d{degree}",
                       "window": w, "centres": n_c, "ring_bits": 8 * elem,
                       "swih_ms": t_all / reps, "swih_gather_ms": t_g / reps}
                if cpu:
                    K = O.kernel_weights(kind, w, w, degree=degree)
                    r = w // 2
                    rng = np.random.default_rng(w)
                    n_s = int(max(256, min(n_c, 2e8 / (w * w))))
                    cx = rng.integers(r, W - r, n_s)
                    cy = rng.integers(r, H - r, n_s)
                    t0 = time.perf_counter()
                    O.likelihood_at(bins, B, K, np.full(B, 1.0 / B), cx, cy)
                    row.update({"brute_force_cpu_ms": (time.perf_counter() - t0) / n_s * n_c * 1e3,
                                "cpu_threads": O.threads(), "cpu_sample_centres": n_s})
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
    return {"fig6": rows, "bins": B,
            "note": ("SWIH: GPU time per map (quantise + integral histograms + gather) and the gather "
                     "alone" + ("; brute force: the FP64 oracle on the host cores, timed on a sample of "
                                "centres and scaled to the map" if cpu else ""))}


# ----------------------------------------------------------------------------- oracle
def oracle_errors(img, B, jobs, maps, targets, n=2048, seed=11,
                  source="the maps copied back at the end of the end-to-end run"):
    """Largest |GPU - oracle| of each likelihood map at n random valid centres.

    The FP64 brute-force oracle is evaluated with the target histograms the GPU
    used (float32, as copied back) and compared with the map values copied back
    from the device; maps[j] is [H - w + 1, W - w + 1] for job (kernel, w)."""
    from oracle import swih_oracle as O

    bins = O.quantize(img, 8, B)
    H, W = bins.shape
    rng = np.random.default_rng(seed)
    per, approx = {}, {}
    for j, (k, w) in enumerate(jobs):
        r = (w - 1) // 2
        cx = rng.integers(r, W - r, n)
        cy = rng.integers(r, H - r, n)
        ref = O.likelihood_at(bins, B, O.kernel_weights(k, w, w), np.asarray(targets[j], dtype=np.float64), cx, cy)
        got = np.asarray(maps[j], dtype=np.float64)[cy - r, cx - r]
        per[f"{k}_{w}"] = float(np.abs(got - ref).max())
        if k == "gaussian":
            true = O.likelihood_at(bins, B, O.true_gaussian(w, w), np.asarray(targets[j], dtype=np.float64),
                                   cx, cy)
            approx[f"{k}_{w}"] = float(np.abs(got - true).max())
    out = {"max_abs": max(per.values()), "tolerance": 1e-5, "per_map": per,
           "sample": (f"{n} random valid centres per map (seed {seed}), FP64 brute-force oracle with the "
                      f"targets the GPU used, against {source}")}
    if approx:
        out["gaussian_vs_true_gaussian"] = {
            "per_map": approx,
            "note": ("approximation error, not parity: the Gaussian kernel is the degree-2 polynomial "
                     "stand-in P(dx^2/rx^2) P(dy^2/ry^2) fitted to exp(-d^2/2 sigma^2), sigma = w/4; this "
                     "is the largest |L_gpu - L| with L the brute-force likelihood under the exact "
                     "Gaussian weights, same centres and targets")}
    return out


def regions_error(img, B, rois, samples, targets):
    """Largest |GPU - oracle| over 64 sampled centres of each (region, scale) map."""
    from oracle import swih_oracle as O

    worst = 0.0
    n = 0
    for i, k, cx, cy, got in samples:
        x0, y0, w, h = rois[i]
        bins = O.quantize(img[y0:y0 + h, x0:x0 + w], 16, B)
        ref = O.likelihood_at(bins, B, O.kernel_weights("gaussian", k, k), targets[i], cx, cy)
        worst = max(worst, float(np.abs(got.astype(np.float64) - ref).max()))
        n += cx.size
    return {"max_abs": worst, "tolerance": 1e-5,
            "sample": f"{n} centres: 64 random valid centres of every (region, scale) map, FP64 brute force"}


def serving_error(frames, qs, samples):
    """Largest |GPU - oracle| over 16 sampled centres of every (query, target,
    window) map the server returned."""
    from oracle import swih_oracle as O

    worst = 0.0
    n = 0
    cache = {}
    for i, t, w, h, cx, cy, got in samples:
        q = qs[i]
        img, bd = frames[q["frame"]]
        key = i
        if key not in cache:
            cache.clear()
            cache[key] = O.quantize(img[q["y0"]:q["y0"] + q["h"], q["x0"]:q["x0"] + q["w"]], bd, q["B"])
        ref = O.likelihood_at(cache[key], q["B"], O.kernel_weights(q["kernel"], w, h),
                              q["targets"][t].astype(np.float64), cx, cy)
        worst = max(worst, float(np.abs(got.astype(np.float64) - ref).max()))
        n += cx.size
    return {"max_abs": worst, "tolerance": 1e-5,
            "sample": f"{n} centres: 16 random valid centres of every (query, target, window) map, FP64 brute force"}



_ORACLE_SETUP = {}


def cpu_model() -> str:
    """The host CPU's name (model name, else implementer/part codes), for the
    CPU baseline's record."""
    import platform

    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        m = re.search(r"^model name\s*:\s*(.+)$", info, re.M)
        if m:
            return m.group(1).strip()
        imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
        part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
        if imp and part:
            return f"{platform.machine()} (implementer {imp.group(1)}, part {part.group(1)})"
    except OSError:
        pass
    return platform.machine() or "unknown"


def oracle_sample(budget_s: float, seed: int = 7):
    """Time the CPU oracle on random valid centres of the same workload (all nine
    kernel/window maps, round robin) for about budget_s seconds (at least one
    chunk per map). The frame, its bins, the kernels and the targets are set up
    once per process, untimed."""
    from oracle import swih_oracle as O
    from paper_1705_03524_gb300 import synth

    if not _ORACLE_SETUP:
        cfg = synth.config2()
        img = cfg["image"]
        B = cfg["B"]
        tx, ty = cfg["target_centre"]
        bins = O.quantize(img, 8, B)
        jobs = []
        for k in KERNELS:
            for w in WINDOWS:
                K = O.kernel_weights(k, w, w)
                jobs.append((k, w, K, O.target_hist(bins, B, K, tx, ty)))
        _ORACLE_SETUP.update(bins=bins, B=B, jobs=jobs)
    bins, B, jobs = _ORACLE_SETUP["bins"], _ORACLE_SETUP["B"], _ORACLE_SETUP["jobs"]
    H, W = bins.shape
    rng = np.random.default_rng(seed)
    n_chunk = 2048
    done = 0
    by_job = {}
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        for (k, w, K, q) in jobs:
            r = (w - 1) // 2
            cx = rng.integers(r, W - r, n_chunk)
            cy = rng.integers(r, H - r, n_chunk)
            O.likelihood_at(bins, B, K, q, cx, cy)
            done += n_chunk
            by_job[(k, w)] = by_job.get((k, w), 0) + n_chunk
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "windows/s", "cores": O.threads(), "kind": "oracle",
            "sample": (f"{done} random valid centres over the 9 kernel/window maps of the same "
                       f"1024x1024 frame, round robin in chunks of {n_chunk}, {el:.1f} s "
                       "(FP64 brute force, OpenMP over centres)"),
            "seconds": el, "by_job": {f"{k}_{w}": n for (k, w), n in by_job.items()}}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    # per step a bounded sample: about a minute for the whole run, at most 2 s a step
    budget = max(0.05, min(2.0, 60.0 / max(1.0, args.steps + 0.25 * args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(budget * 0.25)
    vals = []
    t0 = time.perf_counter()
    res = None
    for _ in range(args.steps):
        res = oracle_sample(budget)
        vals.append(res["value"])
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    cpu = {"value": value, "unit": "windows/s", "cores": res["cores"], "kind": "oracle",
           "sample": res["sample"], "cpu_model": cpu_model()}
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "windows/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "note": "CPU FP64 brute-force oracle on the host cores, "
                   "bounded sample of the workload per step"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "windows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--size", type=int, default=1024,
                    help="frame side; 1024 is the benchmark workload, smaller sizes are for profiling")
    ap.add_argument("--streams", type=int, default=2, choices=(1, 2),
                    help="2: the two plans' builds and gathers on two streams within a step")
    ap.add_argument("--kernels", default="manhattan,euclidean,gaussian",
                    help="subset of kernels (profiling); the benchmark runs all three")
    ap.add_argument("--bins", type=int, default=32,
                    help="bin count; 32 is the benchmark workload, fewer bins shrink profiling captures")
    ap.add_argument("--impl", choices=("swih", "reference"), default="swih")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-regions and serving measurements (profiling runs)")
    ap.add_argument("--serve-queries", type=int, default=400)
    ap.add_argument("--fig6", action="store_true",
                    help="time per map against window size (SWIH on the GPU vs the brute-force oracle)")
    ap.add_argument("--exp-profile", action="store_true",
                    help="small exponential-kernel run for ncu captures: B = 8, two builds and two w = 41 maps")
    ap.add_argument("--wide-profile", action="store_true",
                    help="small any-degree Gaussian run for ncu captures: B = 8, degree 3, 151 px window")
    ap.add_argument("--timed", action="store_true", help="with --wide-profile: time five maps with CUDA events")
    ap.add_argument("--wide-degree", type=int, default=3, help="with --wide-profile: the Gaussian's degree")
    ap.add_argument("--wide-window", type=int, default=151, help="with --wide-profile: the window side")
    ap.add_argument("--regions-only", action="store_true",
                    help="only the batched search-regions measurement (for launch lists of the batch)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "swih":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.fig6:
        print(json.dumps(run_fig6(args)), flush=True)
        return
    if args.exp_profile:
        run_exp_profile()
        return
    if args.wide_profile:
        run_wide_profile(degree=args.wide_degree, w=args.wide_window, timed=args.timed)
        return
    if args.regions_only:
        import torch
        print(json.dumps({"batched_regions": run_regions(args, torch.device("cuda", 0), per_region=False)}),
              flush=True)
        return

    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    # the oracle's OpenMP pool is started before any CUDA work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import swih_oracle as O
        O.build()
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    t0 = time.perf_counter()
    line = run_swih(args, rank, world, local_rank)
    progress(f"frame benchmark: {time.perf_counter() - t0:.1f} s")
    if world == 1 and not args.no_extras:
        import torch
        torch.cuda.empty_cache()
        dev = torch.device("cuda", local_rank)
        for name, fn in (("small_frame", run_small_frame), ("dense_scene", run_dense_scene),
                         ("batched_regions", run_regions),
                         ("serving", lambda a, d: run_serving(a, d, n_queries=a.serve_queries)),
                         ("large_frame", run_large_frame), ("exponential", run_exponential),
                         ("channels", run_channels),
                         ("fig6", lambda a, d: run_fig6(a, frames=((1024, 1024),), cpu=False, reps=5))):
            t0 = time.perf_counter()
            line[name] = fn(args, dev)
            progress(f"{name}: {time.perf_counter() - t0:.1f} s")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        res = oracle_sample(args.cpu_seconds)
        progress(f"cpu baseline: {time.perf_counter() - t0:.1f} s")
        cpu = {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["cpu_model"] = cpu_model()
        if _ORACLE_CHECK:
            try:
                line["oracle_error"] = oracle_errors(*_ORACLE_CHECK)
            except Exception as e:  # the bench line is printed either way
                line["oracle_error"] = {"error": repr(e)}
        for name, thunk in _ORACLE_LATER:
            if name in line:
                t0 = time.perf_counter()
                try:
                    line[name]["oracle_error"] = thunk()
                except Exception as e:
                    line[name]["oracle_error"] = {"error": repr(e)}
                progress(f"oracle check of {name}: {time.perf_counter() - t0:.1f} s")
    if rank == 0:
        line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
