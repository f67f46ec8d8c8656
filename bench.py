#!/usr/bin/env python3
"""Throughput of the FGBD per-frame path on one GB300 (or N replicas under torchrun).

One step = one frame through the whole path of Section 2.1 (scan-line graph,
NE-GBP noise estimate, FSLR selection, Eq. 5 filter written back in input
order) via ``fgbd_run``.  The workload is the 1M-point plain-method frame:
a densely voxelized union of 6 ellipsoids and 4 capped cylinders at 10 bits,
piecewise-smooth uint8 colour, Gaussian colour noise with sigma cycling over
{10, 20, 30, 40, 50} from step to step (5 noise draws of the same geometry).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoints/s and frames/s at 1M pts/frame (plain vs batched); % HBM roofline"
SIGMAS = (10.0, 20.0, 30.0, 40.0, 50.0)
N_POINTS = 1_000_000
BITS = 10
L2_FLUSH_BYTES = 512 << 20
SPEC_STEPS = 3          # filter steps the noise-estimate launch stores (kSpecMax)
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["fgbd", "reference"], default="fgbd")
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-path measurement")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiable-filter measurement")
    ap.add_argument("--stream-frames", type=int, default=300, help="frames of the streaming measurement (0: skip)")
    return ap.parse_args()


def make_frames(n_points, seed=0):
    from paper_2401_09721_gb300 import synth
    xyz = synth.torso_points(n_points, BITS, seed)
    clean = synth.piecewise_colors(xyz, BITS, seed)
    noisy = [synth.add_noise_u8(clean, s, seed + 11 * k) for k, s in enumerate(SIGMAS)]
    return xyz, clean, noisy


# ------------------------------------------------------------------ input generation

_STREAM_SEQ = None


def _stream_frame(t):
    global _STREAM_SEQ
    from paper_2401_09721_gb300 import synth
    if _STREAM_SEQ is None:
        _STREAM_SEQ = synth.StreamSequence(frames=300)
    return _STREAM_SEQ.frame(t)


def _batch_frame(f):
    from paper_2401_09721_gb300 import synth
    return synth.batch_frame(f)


def generate(fn, items):
    """[fn(i) for i in items], computed by a pool of spawned processes (one per
    host core); spawned, not forked, so that it is safe after CUDA is in use."""
    import multiprocessing as mp
    items = list(items)
    workers = max(1, min(len(items), len(os.sched_getaffinity(0))))
    # never from inside a pool worker (a script without a __main__ guard would
    # otherwise spawn pools recursively)
    if workers == 1 or mp.current_process().name != "MainProcess":
        return [fn(i) for i in items]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(fn, items, chunksize=1)


# ------------------------------------------------------------------ batched path

def measure_batched(fgbd, torch, dev, stream, flush, frames, workload, repeats=3):
    """A batch of frames through (a) one fgbd_run per frame, (b) fgbd_run_batch
    with every frame on its own stream, (c) fgbd_run_batch segmented (one
    launch per stage over 16 frames), then (d) fgbd_tune_batch's choice among
    those (and the block shapes), run directly and replayed from a CUDA graph.
    Device time per pass over the frames, L2 flushed before each pass (not
    timed); every output is checked against (a)'s bit for bit."""
    ctxs = [fgbd.Context(fr.n, bits=fr.bits) for fr in frames]
    xs = [torch.from_numpy(fr.xyz).to(dev) for fr in frames]
    cs = [torch.from_numpy(fr.noisy).to(dev) for fr in frames]
    outs = [torch.empty((fr.n, 3), dtype=torch.uint8, device=dev) for fr in frames]
    total = sum(fr.n for fr in frames)
    mean = int(total / len(frames))
    didx = dev.index if dev.index is not None else torch.cuda.current_device()

    def plain():
        for c, x, ci, co in zip(ctxs, xs, cs, outs):
            c.run(x, ci, out=co)

    def batched():
        fgbd.Context.run_batch(ctxs, xs, cs, outs=outs)

    def timed(fn):
        for _ in range(2):
            fn()
        ms = []
        for _ in range(repeats):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    res = {"frames": len(frames), "points": total, "sizes": [fr.n for fr in frames], "workload": workload}
    res["plain_ms"] = timed(plain)
    ref = [o.clone() for o in outs]
    same = True
    base = fgbd.fgbd_get_batch_shape(didx, mean)
    for name, sf in (("streams", 0), ("segmented", 16)):
        fgbd.fgbd_set_batch_shape(didx, mean, dict(base, seg_frames=sf))
        res[f"{name}_ms"] = timed(batched)
        same &= all(torch.equal(a, b) for a, b in zip(outs, ref))
    fgbd.fgbd_set_batch_shape(didx, mean, None)
    shape, _ = fgbd.Context.tune_batch(ctxs, xs, cs, outs=outs)
    res["tuned_shape"] = shape
    res["batched_ms"] = timed(batched)
    same &= all(torch.equal(a, b) for a, b in zip(outs, ref))
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            batched()
        res["graph_ms"] = timed(g.replay)
        same &= all(torch.equal(a, b) for a, b in zip(outs, ref))
    except RuntimeError as e:  # capture refused: report why, keep the other numbers
        res["graph_ms"] = None
        res["graph_error"] = str(e).splitlines()[0][:200]
    res["identical_to_plain"] = bool(same)
    for key in ("plain", "streams", "segmented", "batched", "graph"):
        ms = res.get(f"{key}_ms")
        if ms:
            res[f"{key}_frames_per_s"] = len(frames) / (ms / 1e3)
            res[f"{key}_mpoints_per_s"] = total / (ms / 1e3) / 1e6
    fgbd.fgbd_set_batch_shape(didx, mean, None)
    for c in ctxs:
        c.close()
    return res


def _small_batch_frame(f):
    from paper_2401_09721_gb300 import synth
    return synth.batch_frame(f, lo=20_000, hi=100_000, seed=501, bits=9)


# ------------------------------------------------------------------ differentiable filter

def measure_differentiable(fgbd, torch, dev, stream, steps=200, q=4):
    """Tuning of the filter strength alpha and the bandwidth scale s (sigma = s
    sigma_g) by Adam on 8 clean/noisy pairs (300k sphere points at b = 9,
    sigma = 30): loss = mean squared error of the filtered noisy colours against
    the clean ones, averaged over the pairs.  Reports the device time of one
    forward + backward pass and the loss before and after."""
    from paper_2401_09721_gb300 import synth
    pairs = synth.tuning_pairs()
    ctxs, ys, cl, sgs = [], [], [], []
    for fr in pairs:
        c = fgbd.Context(fr.n, bits=fr.bits)
        c.build_graph(torch.from_numpy(fr.xyz).to(dev))
        ctxs.append(c)
        ys.append(torch.from_numpy(fr.noisy).to(dev))
        cl.append(torch.from_numpy(fr.clean).to(dev))
        sgs.append(c.stats()["sigma_g"])
    alpha = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    scale = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([alpha, scale], lr=0.02)

    def loss_of(k):
        out = ctxs[k].filter(ys[k], alpha, scale * sgs[k], q=q)
        return ((out - cl[k]) ** 2).mean()

    # device time of one forward + backward on one pair
    for _ in range(3):
        loss_of(0).backward()
    ms = []
    for _ in range(10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        loss_of(0).backward()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    alpha.grad = None
    scale.grad = None
    with torch.no_grad():
        first = float(np.mean([loss_of(k).item() for k in range(len(pairs))]))
    t0 = time.perf_counter()
    for _ in range(steps):
        opt.zero_grad()
        total = sum(loss_of(k) for k in range(len(pairs))) / len(pairs)
        total.backward()
        opt.step()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    with torch.no_grad():
        last = float(np.mean([loss_of(k).item() for k in range(len(pairs))]))
    for c in ctxs:
        c.close()
    return {"workload": "8 pairs, 300k sphere points at b=9, float32 noise sigma=30, seeds 101..108, q=4",
            "fwd_bwd_ms": float(np.median(ms)), "fwd_bwd_mpoints_per_s": pairs[0].n / (np.median(ms) / 1e3) / 1e6,
            "adam_steps": steps, "tuning_wall_s": wall, "mse_before": first, "mse_after": last,
            "psnr_before": 10 * np.log10(255.0 ** 2 / first), "psnr_after": 10 * np.log10(255.0 ** 2 / last),
            "alpha": float(alpha.item()), "sigma_scale": float(scale.item())}


# ------------------------------------------------------------------ streaming mode

def measure_streaming(fgbd, torch, dev, stream, frames=300):
    """The first `frames` frames (all 300 by default) of a 300-frame moving sphere (~1.0M points at
    b = 10, sigma = 25, synth.StreamSequence): (a) the full method on every
    frame, (b) the noise estimate and q search on every 10th frame only, the
    others reusing the previous q (Section 3 (2)), (c) every frame in batches
    of 4 through the batched path.  Device-timed per frame (per batch in (c));
    PSNR of the uint8 output against the clean colours."""
    fr = generate(_stream_frame, range(frames))
    xs = [torch.from_numpy(f.xyz).to(dev) for f in fr]
    cs = [torch.from_numpy(f.noisy).to(dev) for f in fr]
    clean = [torch.from_numpy(f.clean).to(dev) for f in fr]
    cap = max(f.n for f in fr)
    outs = [torch.empty((f.n, 3), dtype=torch.uint8, device=dev) for f in fr]

    def psnr():
        mse = [((o.float() - c.float()) ** 2).mean().item() for o, c in zip(outs, clean)]
        return float(np.mean([10 * np.log10(255.0 ** 2 / m) for m in mse]))

    def summary(lat, n_frames):
        total = sum(lat)
        return {"frames_per_s": n_frames / (total / 1e3), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "psnr_db": psnr()}

    res = {"workload": f"frames 0..{frames - 1} of a 300-frame moving sphere, ~1.0M points at b=10, sigma=25",
           "points_mean": float(np.mean([f.n for f in fr]))}
    ctx = fgbd.Context(cap, bits=10)
    for _ in range(2):
        ctx.run(xs[0], cs[0], out=outs[0])
    for mode in ("every_frame", "every_10th"):
        lat = []
        for t in range(frames):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if mode == "every_frame" or t % 10 == 0:
                ctx.run(xs[t], cs[t], out=outs[t])
            else:
                ctx.run_reuse(xs[t], cs[t], out=outs[t])
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
        res[mode] = summary(lat, frames)
    ctx.close()
    ctxs = [fgbd.Context(cap, bits=10) for _ in range(4)]
    fgbd.Context.run_batch(ctxs, xs[:4], cs[:4], outs=outs[:4])
    lat = []
    for t in range(0, frames - frames % 4, 4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fgbd.Context.run_batch(ctxs, xs[t:t + 4], cs[t:t + 4], outs=outs[t:t + 4])
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    res["batches_of_4"] = summary(lat, 4 * len(lat))
    res["batches_of_4"]["latency_is"] = "per batch of 4 frames"
    for c in ctxs:
        c.close()
    return res


# ------------------------------------------------------------------ CPU oracle

def _oracle_child(path, out_path, which):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import fgbd_oracle as orc
    d = np.load(path)
    xyz = d["xyz"]
    times = []
    for k in which:
        rgb = d[f"rgb{k}"]
        t0 = time.perf_counter()
        orc.fgbd(xyz, rgb, orc.Params(bits=BITS))
        times.append(time.perf_counter() - t0)
    with open(out_path, "w") as fh:
        json.dump({"times": times, "n": int(xyz.shape[0])}, fh)


def host_cores():
    """Cores this process may run on, and the CPU model (lscpu)."""
    cores = len(os.sched_getaffinity(0))
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return cores, model


def time_oracle(xyz, rgbs, procs=1):
    """Run the oracle (as it stands, NumPy float64, one thread per process) on
    every colour array of `rgbs` over the frame `xyz`, spread over `procs`
    concurrent fresh processes.  Returns (wall seconds of the whole run, the
    per-frame seconds).  With procs = 1 the frames run one after another."""
    procs = max(1, min(procs, len(rgbs)))
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "frame.npz")
        np.savez(path, xyz=xyz, **{f"rgb{k}": r for k, r in enumerate(rgbs)})
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        children = []
        t0 = time.perf_counter()
        for p in range(procs):
            which = list(range(p, len(rgbs), procs))
            out = os.path.join(td, f"t{p}.json")
            code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
                    f"bench._oracle_child({path!r}, {out!r}, {which!r})")
            children.append((out, subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT)))
        for _, ch in children:
            if ch.wait() != 0:
                raise RuntimeError("oracle process failed")
        wall = time.perf_counter() - t0
        times = []
        for out, _ in children:
            with open(out) as fh:
                times += json.load(fh)["times"]
        return wall, times


def cpu_baseline(xyz, noisy):
    """The oracle on full frames of the workload: one frame on one thread, then
    one frame per host core, all at once (every core busy)."""
    n = xyz.shape[0]
    cores, model = host_cores()
    _, t1 = time_oracle(xyz, [noisy[2]], procs=1)
    rgbs = [noisy[k % len(noisy)] for k in range(cores)]
    wall, tk = time_oracle(xyz, rgbs, procs=cores)
    return {"value": cores * n / wall / 1e6, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": f"{cores} full {n}-point frames of this workload (sigma cycling 10..50), one per host core, "
                      f"run at once in {cores} single-threaded processes of the NumPy float64 oracle: "
                      f"{wall:.1f} s wall",
            "one_core": {"value": n / t1[0] / 1e6, "unit": "Mpoints/s", "cores": 1,
                         "sample": f"one full {n}-point frame (sigma 30), one thread, {t1[0]:.1f} s"},
            "all_cores_frame_s": {"mean": float(np.mean(tk)), "max": float(np.max(tk))}}


def max_over_ranks(values, dist=None, device="cpu"):
    """Each of `values` maximised over the ranks of the job (the slowest rank
    sets the job's time); the values themselves when there is one rank."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(world, n_points, steps, seconds):
    """Whole-job Mpoints/s and frames/s: every rank takes one n_points frame per step
    (replicas), and the job's time is the slowest rank's."""
    return world * n_points * steps / seconds / 1e6, world * steps / seconds


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the full workload frame, one frame per step; the frames of the run are
    # spread over the host cores (one single-threaded oracle process per core)
    xyz, _, noisy = make_frames(args.points)
    n = xyz.shape[0]
    cores, model = host_cores()
    if args.warmup > 0:
        time_oracle(xyz, [noisy[k % len(noisy)] for k in range(min(args.warmup, cores))], procs=cores)
    rgbs = [noisy[k % len(noisy)] for k in range(args.steps)]
    wall, times = time_oracle(xyz, rgbs, procs=cores)
    value = n * len(rgbs) / wall / 1e6
    used = min(cores, len(rgbs))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / len(rgbs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n),
        "cpu_baseline": {"value": value, "unit": "Mpoints/s", "cores": used, "kind": "oracle", "cpu_model": model,
                         "sample": f"{len(rgbs)} full {n}-point torso frames of this workload, one per step "
                                   f"(sigma cycling 10..50), spread over {used} single-threaded processes of the "
                                   f"NumPy float64 oracle; {wall:.1f} s wall, {float(np.mean(times)):.1f} s a frame"},
        "e2e": {"value": value, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(n_points):
    return {"workload": f"torso_shell_{n_points // 1000}k_b{BITS}_u8_sigma10-50",
            "points_per_frame": n_points, "frames_per_step": 1, "bits": BITS,
            "colour": "piecewise-smooth uint8, Gaussian noise sigma in {10,20,30,40,50}",
            "parallelism": "replicas",
            "l2": "flushed between timed steps by a 512 MiB write, flush not timed"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:7]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline bookkeeping

def algorithmic_bytes(name, n, extra_steps=0.0, out_bytes=3):
    """Compulsory DRAM bytes of one launch: the per-point figure of each kernel times n."""
    per_point = {
        "slg_hist": 12,                                   # xyz
        # digit counts of pass 2 (passes 0 and 1 are counted by the histogram and the slab sort)
        "slg_counts2": 4,
        # scatter: keys and values in, keys and values (or the final arrays) out.
        # pass 0 (y-slabs) reads xyz; the slab sort reads the y-ordered pairs and
        # writes the C3 order; pass 1 (C1 on z) writes packed codes, input
        # indices, ranks and the C3 order as sorted ids; pass 2 (C2 on x) reads
        # the codes only and writes the C2 order, the C2 ranks and the codes
        # along C2
        "slg_scatter0": 12 + 8, "slg_slab": 8 + 8, "slg_scatter1": 8 + 16, "slg_scatter2": 4 + 12,
        # link: codes along C1, ids and codes along C2 and C3, C2 ranks of the C3
        # points; the neighbour slots out
        "slg_link": 4 + 8 + 12 + 16,
        "gather_colors": 11,
        # moments: codes 4, slots 16, colours 4, the spread out 4; x_0 of the filter steps out 16
        "ne_moments": 28 + 16,
    }
    if name in per_point:
        return per_point[name] * n
    if name == "ne_finalize":
        # the filter steps stored by the estimate launch (its eigen block moves no bytes):
        # step 1 reads x_0 16 (written by the moments launch) and c4 16, writes the six
        # normalised weights 24, x_1 16 and its power sum 4; each later step reads x 16, c4 16
        # and the weights 24, writes x 16 and its power sum 4
        return 76 * SPEC_STEPS * n
    if name == "filter_select":
        # keep flags: y 4, spread 4, keep 1; the stored steps' Eq. 6 terms 4 each and keep 1;
        # ordinary steps beyond the stored ones 72 each (x in, c4, weights, x out);
        # output: rank 4, x 16, colours out
        return (9 + 4 * SPEC_STEPS + 1 + 72 * extra_steps + 20 + out_bytes) * n
    return 0


def kernel_group(name):
    """Launches of the same kernel function share one group (the sort passes differ by digit)."""
    for g in ("slg_counts", "slg_scan", "slg_scatter"):
        if name.startswith(g):
            return g
    return name


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def read_traffic():
    """DRAM bytes per launch measured by ncu, keyed by kernel and library digest."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    out = {}
    try:
        with open(path) as fh:
            for line in fh:
                line = line.strip()
                if not line or line.startswith("#"):
                    continue
                kern, digest, n, b = line.split()
                out[kern] = (digest, int(n), float(b))
    except (OSError, ValueError):
        pass
    return out


# ------------------------------------------------------------------ GPU arm

def run_fgbd(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2401_09721_gb300 import build, fgbd
    build.build()

    xyz, clean, noisy = make_frames(args.points, seed=rank)
    n = xyz.shape[0]
    dev = torch.device("cuda", local)
    x = torch.from_numpy(xyz).to(dev)
    cols = [torch.from_numpy(c).to(dev) for c in noisy]
    out = torch.empty((n, 3), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = fgbd.Context(n, bits=BITS)
    stream = torch.cuda.current_stream()

    def step(k):
        ctx.run(x, cols[k % len(cols)], out=out)

    # fgbd_run keeps a CUDA graph per argument set from its second call on:
    # give each of the frames' colour buffers its graph before the warm-up
    for k in range(2 * len(cols)):
        step(k)
    for k in range(args.warmup):
        step(k)
    ctx.sync()

    # ---- timed region: device events around each step, L2 flushed in between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.stats()["launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step(args.warmup + k)
            ends[k].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    st = ctx.stats()
    launches = st["launches"] - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = max_over_ranks([sum(step_ms) / 1e3], dist, dev)[0]
    value, fps = job_throughput(world, n, args.steps, total_s)

    # ---- per-kernel timing pass (separate, instrumented)
    ctx.set_timing(True)
    per = {}
    qs = []
    for k in range(len(cols)):
        flush.zero_()
        step(k)
        qs.append(ctx.stats()["q"])
        for name, ms in ctx.timings():
            per.setdefault(name, []).append(ms)
    ctx.set_timing(False)
    q_mean = float(np.mean(qs))
    # steps the selection takes itself: J(q* + 1) decides, SPEC_STEPS come stored
    extra_steps = float(np.mean([max(0, min(q + 1, 64) - SPEC_STEPS) for q in qs]))
    kernels = {}
    for name, lst in per.items():
        avg = float(np.mean(lst))
        b = algorithmic_bytes(name, n, extra_steps=extra_steps)
        kernels[name] = {"ms": avg, "launches_per_step": len(lst) / len(cols),
                         "algo_bytes": b, "gbs": (b / (avg / 1e3) / 1e9) if b and avg > 0 else None}
    # the dominant kernel: the largest share of the step; the launches of one
    # kernel function (the sort passes) count as one kernel.  Every kernel in
    # the step has algorithmic bytes (the estimate launch: its stored filter
    # steps; its eigen block moves none).
    groups = {}
    for name, kd in kernels.items():
        groups.setdefault(kernel_group(name), []).append(kd)
    movers = [g for g in groups if all(kd["algo_bytes"] for kd in groups[g])]
    dom = max(movers, key=lambda g: sum(kd["ms"] * kd["launches_per_step"] for kd in groups[g]))
    members = groups[dom]
    dom_ms = float(np.mean([kd["ms"] for kd in members]))
    dom_bytes = float(np.mean([kd["algo_bytes"] for kd in members]))
    peak, peak_kind = read_peaks()
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic = None
    tr = read_traffic().get(dom)
    if tr is not None and tr[0] == build._digest()[:16]:
        traffic = tr[2] * n / tr[1]
    step_kernel_ms = sum(kd["ms"] * kd["launches_per_step"] for kd in kernels.values())
    table = {}
    for name, kd in sorted(kernels.items(), key=lambda it: -it[1]["ms"] * it[1]["launches_per_step"]):
        table[name] = {"ms": round(kd["ms"], 5), "per_step": kd["launches_per_step"],
                       "share": round(kd["ms"] * kd["launches_per_step"] / step_kernel_ms, 4),
                       "algo_bytes": kd["algo_bytes"],
                       "gbs": None if kd["gbs"] is None else round(kd["gbs"], 1),
                       "frac": None if kd["gbs"] is None else round(kd["gbs"] / peak, 4)}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "algo_bytes_per_launch": dom_bytes, "launch_ms": dom_ms,
                "kernels": table,
                "how": "per-kernel CUDA events on the launching stream in an instrumented pass over the five "
                       "noise draws (L2 flushed before each); achieved = algorithmic bytes / mean launch time; "
                       "share = of the summed kernel times of a step"}
    stages = {}
    for name, kd in kernels.items():
        stage = ("graph" if name.startswith("slg") else "noise" if name in ("gather_colors", "ne_moments", "ne_finalize")
                 else "select+filter")
        stages[stage] = stages.get(stage, 0.0) + kd["ms"] * kd["launches_per_step"]

    # ---- end to end through the C call on host buffers (fgbd_run_host): every step
    # copies its pinned inputs in and its output back.  Consecutive steps pipeline
    # (a step's copies overlap its neighbours' device work), so the wall-clock time of
    # K steps is measured; the L2 is not flushed in between (a step's device working
    # set, about 180 MB, exceeds the 129 MB L2 anyway).
    pin_x = torch.from_numpy(xyz).pin_memory()
    pin_c = [torch.from_numpy(c).pin_memory() for c in noisy]
    pin_o = [torch.empty((n, 3), dtype=torch.uint8).pin_memory() for _ in range(2)]
    for k in range(max(args.warmup, 4)):
        ctx.run_host(pin_x, pin_c[k % len(pin_c)], pin_o[k % 2])
    ctx.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        ctx.run_host(pin_x, pin_c[k % len(pin_c)], pin_o[k % 2])
    ctx.sync()
    e2e_s = time.perf_counter() - t0
    # the same copies issued one step at a time on the caller's stream, with the L2
    # flushed between steps (outside the timed regions): no overlap at all
    dx = torch.empty_like(x)
    dc = torch.empty_like(cols[0])
    e_st = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_en = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.warmup + args.steps):
        flush.zero_()
        if k >= args.warmup:
            e_st[k - args.warmup].record(stream)
        dx.copy_(pin_x, non_blocking=True)
        dc.copy_(pin_c[k % len(pin_c)], non_blocking=True)
        ctx.run(dx, dc, out=out)
        pin_o[0].copy_(out, non_blocking=True)
        if k >= args.warmup:
            e_en[k - args.warmup].record(stream)
    torch.cuda.synchronize()
    serial_s = sum(a.elapsed_time(b) for a, b in zip(e_st, e_en)) / 1e3
    e2e_s, serial_s = max_over_ranks([e2e_s, serial_s], dist, dev)
    e2e = {"value": job_throughput(world, n, args.steps, e2e_s)[0], "unit": "Mpoints/s",
           "h2d_bytes_per_step": int(pin_x.numel() * 4 + pin_c[0].numel()), "d2h_bytes_per_step": int(pin_o[0].numel()),
           "api": "fgbd_run_host (pinned host buffers, two steps in flight), host wall clock",
           "serial": {"value": job_throughput(world, n, args.steps, serial_s)[0],
                      "how": "copies and run in order on one stream, L2 flushed between steps, CUDA events"}}

    # ---- ablations of Tables 4 and 5 (and the same-line reading) on the same frames,
    # device-timed like the main steps; PSNR of the output against the clean colours
    ablations = {}
    clean_d = torch.from_numpy(clean).to(dev).float()
    for name, variant, window in (("as_published", 0, 1), ("no_fslr", fgbd.VARIANT_NO_FSLR, 1),
                                  ("unsorted_patch", fgbd.VARIANT_UNSORTED_PATCH, 1),
                                  ("same_line", fgbd.VARIANT_SAME_LINE, 1), ("window2", 0, 2), ("window3", 0, 3),
                                  ("sigma_g_node_mean", fgbd.VARIANT_SIGMA_NODE, 1),
                                  ("sigma_g_per_point", fgbd.VARIANT_SIGMA_PAIR, 1),
                                  ("pooled_patch_d7", fgbd.VARIANT_POOLED_PATCH, 1),
                                  ("q_global_argmin", fgbd.VARIANT_GLOBAL_Q, 1)):
        vctx = fgbd.Context(n, bits=BITS, variant=variant, window=window)
        for k in range(2 * len(cols)):  # every frame's graph is captured before the timed runs
            vctx.run(x, cols[k % len(cols)], out=out)
        ms, sig, qv, ps = [], [], [], []
        for k in range(len(cols)):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            vctx.run(x, cols[k], out=out)
            a1.record(stream)
            vst = vctx.stats()
            ms.append(a0.elapsed_time(a1))
            sig.append(vst["sigma_est"])
            qv.append(vst["q"])
            mse = float(((out.float() - clean_d) ** 2).mean().item())
            ps.append(round(10.0 * math.log10(255.0 ** 2 / max(mse, 1e-12)), 3))
        vctx.close()
        ablations[name] = {"ms_per_step": float(np.mean(ms)), "value": n / (float(np.mean(ms)) / 1e3) / 1e6,
                           "unit": "Mpoints/s", "window": window, "variant": int(variant), "sigma": list(SIGMAS),
                           "sigma_est": [round(v, 4) for v in sig], "sigma_g": round(vst["sigma_g"], 4),
                           "q": qv, "psnr_db": ps}

    batched = None
    batched_small = None
    if not args.no_batch:
        batched = measure_batched(fgbd, torch, dev, stream, flush, generate(_batch_frame, range(16)),
                                  "16 sphere frames, N ~ U[200k, 1.2M] at b=10, sigma ~ U[10, 50], seeds 1..16")
        batched_small = measure_batched(fgbd, torch, dev, stream, flush, generate(_small_batch_frame, range(64)),
                                        "64 sphere frames, N ~ U[20k, 100k] at b=9, sigma ~ U[10, 50], seeds 501..564")
    differentiable = None
    if not args.no_diff:
        differentiable = measure_differentiable(fgbd, torch, dev, stream)
    streaming = None
    if args.stream_frames > 0:
        streaming = measure_streaming(fgbd, torch, dev, stream, args.stream_frames)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(xyz, noisy)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(n), "frames_per_s": fps, "e2e": e2e,
            "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clocks.summary(), "stages_ms": stages,
            "q_mean": q_mean, "wall_s": wall, "step_ms_min": min(step_ms), "step_ms_max": max(step_ms),
            "ablations": ablations, "batched": batched, "batched_small": batched_small,
            "differentiable": differentiable,
            "streaming": streaming,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fgbd(args)


if __name__ == "__main__":
    main()
