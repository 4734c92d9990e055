#!/usr/bin/env python3
"""RSFT throughput on GB300: frames/s of the whole hot path on synthetic radar cubes.

Default workload: the 3-D radar cube 1024 x 256 x 64 complex64 (range x Doppler x
angle), bucket grid 64 x 32 x 8, L = 12 loops, 80 dB Chebyshev windows, system
P_fa = 1e-6, K = 32 off-grid Rayleigh targets at 5-25 dB.  The headline runs at the
operating point where the RSFT meets its P_fa: thresholds from eq. (opt) with the
binomial vote laws (the paper's Normal approximation of Claim 3 puts the false-alarm
rate near 1e-3 on this workload; it is reported beside it as `paper_design`), and the
dense detector is run at the RSFT's measured false-alarm rate.  A step is a chunk of
`--frames-per-step` frames (default 256), each one whole RSFT (fold, bucket FFT +
detection, votes, second stage, median estimate).  Frames rotate through a ring of 4
distinct cubes (537 MB, larger than the 129 MB L2).

Prints one JSON line (rank 0).  `--impl reference` times the CPU FP64 oracle on
the host instead (the only comparison system this method has).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RSFT frames/s on 1 GB300 at matched Pd/Pfa; % HBM roofline; vs plain and dense FFT"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--frames-per-step", type=int, default=256)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2_3d_radar")
    ap.add_argument("--frames", type=int, default=4)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", type=int, default=0,
                    help="run this many plain executes of the workload and exit without a JSON line: the small, "
                         "fixed command that the ncu captures under profiles/ are taken on")
    ap.add_argument("--profile-frames", type=int, default=0,
                    help="with --profile: run that many rsft_execute_frames calls of this many frames instead")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_frames(rank, frames):
    """Frame ids of one rank: ranks own disjoint frames (weak scaling, no data exchange)."""
    return [rank * frames + f for f in range(frames)]


def max_over_ranks(value, ws, device=None):
    """The largest of the ranks' values (the slowest rank's time); identity for one rank."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, steps, ms):
    """Frames per second of the whole job: every rank runs `steps` frames in at most `ms`."""
    return ws * steps / (ms / 1e3)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profile_traffic(workload, source):
    """DRAM bytes per fold launch from the committed ncu summary, if it matches the kernel source."""
    tag = "_tc" if source == "fold_tc.cu" else ""
    path = os.path.join(ROOT, "profiles", f"permute_window_fold{tag}_{workload}.txt")
    src = os.path.join(ROOT, "paper_1610_01050_gb300", "csrc", source)
    try:
        text = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        vals = dict(line.split(":", 1) for line in text.splitlines() if ":" in line)
        if vals.get("source", "").strip() != source or vals.get("source_sha256_16", "").strip() != digest:
            return None
        return float(vals["dram_bytes_per_launch"].strip())
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.out = tempfile.NamedTemporaryFile(prefix="clocks_", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd.insert(1, f"--id={gpu_id}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = self.t1 = None

    def mark(self, start):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.out.close()
        rows = []
        try:
            for line in open(self.out.name):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def workload_desc(R, wl, nv, seed, max_located=1 << 20, design=None):
    """The workload's descriptor; `design` None = the binomial vote-law design (the headline's
    operating point), else an RSFT_DESIGN_* value."""
    return R.make_desc(wl.shape, wl.buckets, wl.loops, atten_db=wl.atten_db, flat_support=wl.flat_support,
                       p_fa=wl.p_fa, k_max=wl.k_design, noise_var=nv, seed=seed, max_located=max_located,
                       design_mode=R.RSFT_DESIGN_BINOMIAL if design is None else design)


BATCH_CHUNK = 32      # frames per batched call
BATCH_CAP = 1 << 17   # located capacity per frame in batched calls


def batched_frames(R, bplan, ring, nframes, lanes, bcounts, bloc, bamp, stream):
    """nframes frames through rsft_execute_batch in calls of BATCH_CHUNK frames."""
    done = 0
    while done < nframes:
        m = min(BATCH_CHUNK, nframes - done)
        R.rsft_execute_batch(bplan, ring[:m], bcounts, lanes=lanes, located=bloc, amp=bamp, stream=stream)
        done += m


def graph_frames(R, graphs, nframes, stream):
    """nframes frames as recorded executes (frame f: graph f mod len(graphs), one per lane),
    BATCH_CHUNK per rsft_graph_launch_batch."""
    seq = [graphs[f % len(graphs)] for f in range(nframes)]
    for i in range(0, nframes, BATCH_CHUNK):
        R.rsft_graph_launch_batch(seq[i:i + BATCH_CHUNK], stream=stream)


def oracle_plan(wl, nv, seed):
    import oracle as O
    return O.make_plan(wl.shape, wl.buckets, wl.loops, seed=seed, atten_db=wl.atten_db,
                       flat_support=wl.flat_support, noise_var=nv, p_fa=wl.p_fa, k_max=wl.k_design,
                       design_mode="binomial")


def oracle_frame(op, x):
    """Time the FP64 oracle (as it stands) on one whole frame, all L loops; returns
    (wall seconds, threads used = CPU time / wall time)."""
    import oracle as O
    t0, c0 = time.perf_counter(), time.process_time()
    O.rsft(op, x, estimate=True, keep=False)
    wall = time.perf_counter() - t0
    return wall, max(1, int(round((time.process_time() - c0) / max(wall, 1e-9))))


def cpu_baseline(wl, cube, nv, seed, min_s=10.0, max_frames=3):
    """Whole frames through the oracle until about 10 s of CPU work (at most 3 frames)."""
    op = oracle_plan(wl, nv, seed)
    x = cube.astype(np.complex128)
    times, cores = [], 1
    while len(times) < max_frames and sum(times) < min_s:
        t, c = oracle_frame(op, x)
        times.append(t)
        cores = max(cores, c)
    per_frame = sum(times) / len(times)
    sample = (f"{len(times)} whole {'x'.join(map(str, wl.shape))} frame(s), all {wl.loops} loops of the FP64 "
              f"oracle (plan excluded), {sum(times):.1f} s")
    return {"value": 1.0 / per_frame, "unit": "frames/s", "cores": cores, "host_cores": os.cpu_count(),
            "kind": "oracle", "sample": sample}


def workload_name(wl):
    """The config's workload string, the same for both arms."""
    return (f"{wl.name}: {'x'.join(map(str, wl.shape))} complex64, B={'x'.join(map(str, wl.buckets))}, "
            f"L={wl.loops}, {wl.atten_db:g} dB Chebyshev, Pfa={wl.p_fa:g}, K={wl.k_range[0]}-{wl.k_range[1]} {wl.kind}")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import rsft_inputs as ri
    wl = ri.WORKLOADS[args.workload]
    cube, _, _, nv = ri.workload_frame(args.workload, 0)
    seed = ri.frame_seed(wl, 0)
    # a step is one whole frame through the oracle (about 3 s on one core): the bounded sample of the
    # workload; the warm-up and timed step counts are the ones given
    op = oracle_plan(wl, nv, seed)
    x = cube.astype(np.complex128)
    warmup = max(0, args.warmup)
    for _ in range(warmup):
        oracle_frame(op, x)
    steps = max(1, args.steps)
    runs = [oracle_frame(op, x) for _ in range(steps)]
    per_step = sum(t for t, _ in runs) / len(runs)
    cores = max(c for _, c in runs)
    value = 1.0 / per_step
    sample = (f"one whole {'x'.join(map(str, wl.shape))} frame per step (all {wl.loops} loops, binomial-design "
              f"thresholds), {steps} steps after {warmup} warm-up")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(wl), "shape": list(wl.shape), "buckets": list(wl.buckets),
                   "loops": wl.loops},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def detection_quality(wl, targets, shape, located):
    """Pd: targets with a located index within +-1 bin per dimension; Pfa: located cells
    outside every target's +-3-bin box over the cells outside those boxes."""
    n = np.asarray(shape)
    idx = np.stack(np.unravel_index(located, shape), axis=1) if len(located) else np.zeros((0, len(shape)), int)
    grid = np.rint(targets.freqs * n).astype(np.int64) % n
    hits, outside = 0, np.ones(len(idx), dtype=bool)
    for g in grid:
        diff = np.abs(idx - g)
        diff = np.minimum(diff, n - diff)
        if np.any(np.all(diff <= 1, axis=1)):
            hits += 1
        outside &= ~np.all(diff <= 3, axis=1)
    cells_out = float(np.prod(n)) - len(grid) * 7.0 ** len(shape)
    return hits / max(1, len(grid)), float(outside.sum()) / cells_out


def dense_comparator(R, torch, wl, nv, cubes, targets, stream, dev, ws, steps, warmup, cap, rsft_value,
                     matched_pfa=None):
    """The dense Bartlett detector (window + cuFFT N-D FFT + exact NP threshold) on the same
    frames: frames/s by CUDA events, its Pd/Pfa at the workload's P_fa and, when given, at the
    RSFT's measured false-alarm rate (the matched operating point), and the RSFT's speed-up."""
    def make(p_fa):
        d = R.make_desc(wl.shape, wl.buckets, wl.loops, atten_db=wl.atten_db, noise_var=nv, max_located=cap)
        d.p_fa = p_fa
        return R.rsft_bartlett_plan_create(d)

    located = torch.zeros(cap, dtype=torch.int64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)

    def quality(plan):
        pd, pfa, n_loc = [], [], []
        for f in range(len(cubes)):
            c = R.rsft_bartlett_execute(plan, cubes[f], located=located, allow_capacity=True)
            a, b = detection_quality(wl, targets[f], wl.shape, located[:min(c, cap)].cpu().numpy())
            pd.append(a)
            pfa.append(b)
            n_loc.append(c)
        return float(np.mean(pd)), float(np.mean(pfa)), float(np.mean(n_loc))

    plan = make(wl.p_fa)
    pd, pfa, n_loc = quality(plan)
    matched = None
    if matched_pfa is not None and 0.0 < matched_pfa < 1.0:
        mplan = make(matched_pfa)
        mpd, mpfa, mloc = quality(mplan)
        mplan.close()
        matched = {"p_fa_design": matched_pfa, "pd": mpd, "pfa": mpfa, "located_per_frame": mloc}
    for k in range(warmup):
        R.rsft_bartlett_execute_async(plan, cubes[k % len(cubes)], count, located=located, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        R.rsft_bartlett_execute_async(plan, cubes[k % len(cubes)], count, located=located, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    val = whole_job_rate(ws, steps, ms)
    plan.close()
    return {"method": "Bartlett (Algorithm 2, one segment): pre-window, cuFFT N-D FFT, exact NP threshold",
            "value": val, "unit": "frames/s", "ms_per_frame": ms / steps, "steps": steps,
            "pd": pd, "pfa": pfa, "located_per_frame": n_loc, "at_rsft_pfa": matched,
            "rsft_speedup": rsft_value / val}


def rsft_quality(R, plan, wl, cubes, targets, located, cap):
    """Pd / Pfa of a plan over the ring of frames (detection_quality per frame, averaged)."""
    pd, pfa, n_loc = [], [], []
    for f in range(len(cubes)):
        c = R.rsft_execute(plan, cubes[f], located=located, allow_capacity=True)
        a, b = detection_quality(wl, targets[f], wl.shape, located[:min(c, cap)].cpu().numpy())
        pd.append(a)
        pfa.append(b)
        n_loc.append(c)
    return float(np.mean(pd)), float(np.mean(pfa)), float(np.mean(n_loc))


def timed_plain(R, torch, plan, cubes, stream, frames, count, located, amp):
    """Frames/s of back-to-back rsft_execute_async calls (CUDA events), after 3 warm-up frames."""
    for k in range(3):
        R.rsft_execute_async(plan, cubes[k % len(cubes)], count, stream=stream, located=located, amp=amp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(frames):
        R.rsft_execute_async(plan, cubes[k % len(cubes)], count, stream=stream, located=located, amp=amp)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def paper_design(R, torch, wl, nv, seed, cubes, targets, stream, dev, ws, frames, located, amp, count, cap):
    """The paper's own operating point (eq. (opt) with Claims 2-3's Normal approximations): its
    thresholds, Pd / Pfa and plain frames/s on the same frames."""
    plan = R.rsft_plan_create(workload_desc(R, wl, nv, seed, design=R.RSFT_DESIGN_NORMAL))
    pd, pfa, n_loc = rsft_quality(R, plan, wl, cubes, targets, located, cap)
    ms = max_over_ranks(timed_plain(R, torch, plan, cubes, stream, frames, count, located, amp), ws, dev)
    out = {"mu": int(R.rsft_plan_get(plan, R.RSFT_GET_MU)[0]), "pfa1": float(R.rsft_plan_get(plan, R.RSFT_GET_PFA1)[0]),
           "pd": pd, "pfa": pfa, "located_per_frame": n_loc,
           "plain_frames_per_s": whole_job_rate(ws, frames, ms),
           "note": "thresholds of eq. (opt) with the Normal vote approximations of Claims 2-3 (the paper's design)"}
    plan.close()
    return out


def estimate_mode(R, torch, wl, seed, cubes, targets, stream, dev, ws, frames, located, amp, count, cap):
    """The same workload with the noise level unknown: each loop's threshold from the lower median
    of its bucket powers (np_detect's noise-floor reduction); Pd / Pfa and plain frames/s."""
    plan = R.rsft_plan_create(workload_desc(R, wl, 0.0, seed))
    pd, pfa, n_loc = rsft_quality(R, plan, wl, cubes, targets, located, cap)
    ms = max_over_ranks(timed_plain(R, torch, plan, cubes, stream, frames, count, located, amp), ws, dev)
    out = {"pd": pd, "pfa": pfa, "located_per_frame": n_loc, "plain_frames_per_s": whole_job_rate(ws, frames, ms),
           "ms_per_frame": ms / frames,
           "note": "noise_var unknown: gamma_l = lowermedian(|f-hat_l|^2) / ln 2 * (-ln Pfa1), binomial design"}
    plan.close()
    return out


C5 = "c5_4d"


def c5_frames(R, torch, ri, dev, ws, stream, frames):
    """The 4-D workload (512 x 512 x 64 x 32 complex64, 4.3 GB, B = 32 x 32 x 8 x 4, L = 16,
    Pfa = 1e-7, K = 256 at 0-20 dB): frames/s of plain executes on one resident frame (4.3 GB, far
    beyond L2), its fold roofline, Pd / Pfa, and the dense 4-D Bartlett pass on the same frame."""
    wl = ri.WORKLOADS[C5]
    cube, tg, _, nv = ri.workload_frame(C5, 0)
    x = torch.from_numpy(cube).to(dev)
    del cube
    cap = 1 << 22
    seed = ri.frame_seed(wl, 0)
    plan = R.rsft_plan_create(workload_desc(R, wl, nv, seed, max_located=cap))
    loc = torch.zeros(cap, dtype=torch.int64, device=dev)
    amp = torch.zeros(cap, dtype=torch.complex64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    pd, pfa, n_loc = rsft_quality(R, plan, wl, [x], [tg], loc, cap)
    R.rsft_plan_timing(plan, True)
    ms = max_over_ranks(timed_plain(R, torch, plan, [x], stream, frames, count, loc, amp), ws, dev)
    st = R.rsft_plan_get(plan, R.RSFT_GET_STAGE_MS)
    fold_s = st[0] / max(1.0, st[6]) / 1e3
    fold_bytes = int(R.rsft_plan_get(plan, R.RSFT_GET_FOLD_BYTES)[0])
    peak, peak_kind = measured_peak()
    plan.close()
    dense = dense_comparator(R, torch, wl, nv, [x], [tg], stream, dev, ws, max(2, frames // 2), 2, cap,
                             whole_job_rate(ws, frames, ms), matched_pfa=pfa if pfa > 0 else None)
    return {"workload": workload_name(wl), "value": whole_job_rate(ws, frames, ms), "unit": "frames/s",
            "frames": frames, "ms_per_frame": ms / frames, "fold_us": fold_s * 1e6,
            "fold_frac_of_hbm": fold_bytes / fold_s / 1e9 / peak, "peak_source": peak_kind,
            "pd": pd, "pfa": pfa, "located_per_frame": n_loc, "dense_fft": dense,
            "note": "one resident frame, back-to-back rsft_execute_async; binomial-design thresholds"}


def refinement(R, torch, plan, wl, cubes, targets, stream, cap, steps=20, lr=0.7, max_tones=64):
    """Bucket-domain refinement of the RSFT's located tones on frame 0: the strongest located
    frequencies (at most one per +-2-bin box) start on their grid points with the median
    amplitude estimates; reports the frequency error (bins) of the targets they sit on, before
    and after `steps` Levenberg-Marquardt steps, and the time of rsft_refine."""
    dev = cubes[0].device
    loc = torch.zeros(cap, dtype=torch.int64, device=dev)
    amp = torch.zeros(cap, dtype=torch.complex64, device=dev)
    c = min(R.rsft_execute(plan, cubes[0], located=loc, amp=amp, allow_capacity=True), cap)
    n = np.asarray(wl.shape)
    idx = np.stack(np.unravel_index(loc[:c].cpu().numpy(), wl.shape), axis=1)
    mag = np.abs(amp[:c].cpu().numpy())
    picked = []
    for i in np.argsort(-mag):
        if len(picked) == max_tones:
            break
        if all(np.any(np.minimum(np.abs(idx[i] - idx[j]), n - np.abs(idx[i] - idx[j])) > 2) for j in picked):
            picked.append(i)
    f0 = (idx[picked] / n).astype(np.float32)
    a0 = amp[:c].cpu().numpy()[picked].astype(np.complex64)
    f = torch.from_numpy(f0).to(dev)
    a = torch.from_numpy(a0).to(dev)
    R.rsft_refine(plan, cubes[0], len(picked), f.clone(), a.clone(), 2, lr, stream=stream)  # warm-up
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    R.rsft_refine(plan, cubes[0], len(picked), f, a, steps, lr, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    f1 = f.cpu().numpy().astype(np.float64)
    truth = targets[0].freqs * n
    before, after = [], []
    for t in truth:
        d0 = np.abs(f0 * n - t)
        d0 = np.minimum(d0, n - d0)
        j = int(np.argmin(np.max(d0, axis=1)))
        if np.max(d0[j]) <= 1.0:
            d1 = np.abs(f1[j] * n - t)
            d1 = np.minimum(d1, n - d1)
            before.append(d0[j])
            after.append(d1)
    rms = (lambda v: float(np.sqrt(np.mean(np.square(v)))) if len(v) else None)
    return {"tones": len(picked), "steps": steps, "ms": ev0.elapsed_time(ev1),
            "targets_matched": len(before), "freq_rmse_bins_before": rms(before), "freq_rmse_bins_after": rms(after),
            "note": "rsft_refine on frame 0: fold of the cube + Levenberg-Marquardt steps on the bucket residual"}


def segment_mode(R, torch, plan, wl, cubes, stream, dev, ws, located, amp, count, frames):
    """Segment mode (loop l folds its own data segment): frames of L segments each, the
    segments taken round-robin from the ring of cubes; the fold reads L cubes per frame."""
    F = len(cubes)
    segs = [cubes[l % F] for l in range(wl.loops)]
    for _ in range(2):
        R.rsft_execute_segments_async(plan, segs, count, stream=stream, located=located, amp=amp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(frames):
        segs = [cubes[(k + l) % F] for l in range(wl.loops)]
        R.rsft_execute_segments_async(plan, segs, count, stream=stream, located=located, amp=amp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    cube_bytes = int(np.prod(wl.shape)) * 8
    return {"value": whole_job_rate(ws, frames, ms), "unit": "frames/s", "frames": frames,
            "ms_per_frame": ms / frames, "segments_per_frame": wl.loops,
            "hbm_gbs": wl.loops * cube_bytes * frames / (ms / 1e3) / 1e9,
            "note": "one 1024x256x64 segment per loop, taken round-robin from the ring of frames"}


SRUR_BUCKETS = (64, 16, 8)
SRUR_BURSTS = 8


def srur_frames(R, torch, ri, dev, ws, stream, frames):
    """SRUR radar frames (§VI): 8 bursts of the Table III system (2048 range samples x 64
    elements x 32 repetition intervals, complex64, 268 MB per frame) with the Table IV targets
    at their "mixed" SNRs and Swerling-I amplitudes redrawn per burst, one burst per loop
    (segment mode), B = 64x16x8, 60 dB Chebyshev, P_fa = 1e-6; Pd of the four targets."""
    sy = ri.SrurSystem()
    cubes, freqs, _ = ri.srur_bursts(sy, ri.TABLE_IV["mixed"], SRUR_BURSTS, seed=4001)
    segs = [torch.from_numpy(c).to(dev) for c in cubes]
    del cubes
    cap = 1 << 18
    plan = R.rsft_plan_create(R.make_desc(sy.shape, SRUR_BUCKETS, SRUR_BURSTS, atten_db=60.0, p_fa=1e-6, k_max=4,
                                          noise_var=1.0, seed=4001, max_located=cap))
    loc = torch.zeros(cap, dtype=torch.int64, device=dev)
    amp = torch.zeros(cap, dtype=torch.complex64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    c = min(R.rsft_execute_segments(plan, segs, stream=stream, located=loc, amp=amp, allow_capacity=True), cap)
    n = np.asarray(sy.shape)
    idx = np.stack(np.unravel_index(loc[:c].cpu().numpy(), sy.shape), axis=1)
    hits = 0
    for f in freqs:
        d = np.abs(idx - np.rint(f * n).astype(np.int64) % n)
        hits += int(np.any(np.all(np.minimum(d, n - d) <= 1, axis=1)))
    for _ in range(3):
        R.rsft_execute_segments_async(plan, segs, count, stream=stream, located=loc, amp=amp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(frames):
        R.rsft_execute_segments_async(plan, segs, count, stream=stream, located=loc, amp=amp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    plan.close()
    return {"value": whole_job_rate(ws, frames, ms), "unit": "frames/s", "frames": frames,
            "ms_per_frame": ms / frames, "bursts_per_frame": SRUR_BURSTS,
            "hbm_gbs": SRUR_BURSTS * int(np.prod(sy.shape)) * 8 * frames / (ms / 1e3) / 1e9,
            "pd": hits / len(freqs), "located": int(c),
            "note": "Table III system, Table IV targets (mixed SNRs), one burst per loop, B = 64x16x8"}


MIXED = ("c3_small", "c3_mid", "c3_large")
MIXED_CAP = 1 << 17


def mixed_batch(R, torch, ri, dev, ws, stream, n_frames=512, per_shape=2, lanes=4, chunk=64, group=16):
    """Batched frames of uneven shapes: 512 frames drawn uniformly from the three sizes of the
    mixed-size workload, each shape with its own plan (fold schedule picked by
    rsft_plan_autotune on one of its frames).  Headline form: each shape's frames go 16 at a time
    through one launch per stage (rsft_execute_frames), recorded as CUDA graphs
    (rsft_graph_create_frames) and launched together, so the three shapes' graphs overlap.  Also
    timed: every frame its own recorded execute over 4 lanes per plan, and the same sequence
    through rsft_execute_async on one stream."""
    rng = np.random.default_rng(1610)
    shape_of = [MIXED[i] for i in rng.integers(0, len(MIXED), n_frames)]
    counts_by = {n: sum(1 for x in shape_of if x == n) for n in MIXED}
    plans, rings, graphs, outs, tuned, fgraphs, together = {}, {}, {}, [], {}, {}, {}
    for name in MIXED:
        wl = ri.WORKLOADS[name]
        cubes, nv = [], wl.noise_var
        for f in range(per_shape):
            cube, _, _, nv = ri.workload_frame(name, f)
            cubes.append(torch.from_numpy(cube).to(dev))
        # the paper's design: with K = 8..64 targets in 128-4096 buckets the binomial law admits no mu
        # that meets P_fa = 1e-5 on these shapes (Remark 2 is nearly reached), so the batch keeps eq. (opt)
        plan = R.rsft_plan_create(workload_desc(R, wl, nv, ri.frame_seed(wl, 0), max_located=MIXED_CAP,
                                                design=R.RSFT_DESIGN_NORMAL))
        us, chosen = R.rsft_plan_autotune(plan, cubes[0], candidates=4, reps=5, stream=stream)
        tuned[name] = {"fold_us": us, "candidate": chosen}
        together[name] = R.rsft_plan_frames_together(plan)
        plans[name], rings[name], graphs[name] = plan, cubes, []
        for g in range(lanes):  # graph g: resident frame g % per_shape on lane g
            o = (torch.zeros(MIXED_CAP, dtype=torch.int64, device=dev),
                 torch.zeros(MIXED_CAP, dtype=torch.complex64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
            outs.append(o)
            graphs[name].append(R.rsft_graph_create(plan, cubes[g % per_shape], o[2], located=o[0], amp=o[1], lane=g))
        # frames form: one graph of `group` frames (resident frames in turn) and one of the remainder
        fgraphs[name] = []
        for size in (group, counts_by[name] % group):
            if size == 0:
                continue
            o = (torch.zeros(size * MIXED_CAP, dtype=torch.int64, device=dev),
                 torch.zeros(size * MIXED_CAP, dtype=torch.complex64, device=dev),
                 torch.zeros(size, dtype=torch.int64, device=dev))
            outs.append(o)
            fgraphs[name].append(R.rsft_graph_create_frames(plan, [cubes[k % per_shape] for k in range(size)], o[2],
                                                            located=o[0], amp=o[1]))
    seen = {n: 0 for n in MIXED}
    seq, plain = [], []
    for name in shape_of:
        k = seen[name]
        seen[name] += 1
        seq.append(graphs[name][k % lanes])
        plain.append((plans[name], rings[name][k % lanes % per_shape]))
    # frames form: each shape's full groups then its remainder, the shapes interleaved
    per_shape_seq = {n: [fgraphs[n][0]] * (counts_by[n] // group) + (fgraphs[n][1:] if counts_by[n] % group else [])
                     for n in MIXED}
    fseq = []
    while any(per_shape_seq.values()):
        for n in MIXED:
            if per_shape_seq[n]:
                fseq.append(per_shape_seq[n].pop(0))
    frame_bytes = sum(int(np.prod(ri.WORKLOADS[n].shape)) * 8 for n in shape_of)

    def run_graphs(frames):
        for i in range(0, len(frames), chunk):
            R.rsft_graph_launch_batch(frames[i:i + chunk], stream=stream)

    count = torch.zeros(1, dtype=torch.int64, device=dev)
    loc = torch.zeros(MIXED_CAP, dtype=torch.int64, device=dev)
    amp = torch.zeros(MIXED_CAP, dtype=torch.complex64, device=dev)

    def run_plain(frames):
        for plan, x in frames:
            R.rsft_execute_async(plan, x, count, stream=stream, located=loc, amp=amp)

    run_graphs(seq[:2 * chunk])
    run_graphs(fseq)
    run_plain(plain[:16])
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    R.rsft_graph_launch_batch(fseq, stream=stream)
    ev[1].record(stream)
    run_graphs(seq)
    ev[2].record(stream)
    run_plain(plain)
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev[0].elapsed_time(ev[1]), ws, dev)
    ms_graphs = max_over_ranks(ev[1].elapsed_time(ev[2]), ws, dev)
    ms_plain = max_over_ranks(ev[2].elapsed_time(ev[3]), ws, dev)
    for name in MIXED:
        for g in graphs[name] + fgraphs[name]:
            g.close()
        plans[name].close()
    value = whole_job_rate(ws, n_frames, ms)
    return {"value": value, "unit": "frames/s", "frames": n_frames,
            "shapes": counts_by, "frames_together": together,
            "ms_per_frame": ms / n_frames, "hbm_gbs_cube_reads": frame_bytes / (ms / 1e3) / 1e9,
            "per_frame_graphs": {"value": whole_job_rate(ws, n_frames, ms_graphs), "unit": "frames/s",
                                 "note": f"every frame one recorded execute, over {lanes} lanes per plan"},
            "plain": {"value": whole_job_rate(ws, n_frames, ms_plain), "unit": "frames/s",
                      "note": "the same sequence, one rsft_execute_async per frame on one stream"},
            "speedup_over_plain": ms_plain / ms, "autotune": tuned,
            "note": f"shapes {', '.join('x'.join(map(str, ri.WORKLOADS[n].shape)) for n in MIXED)} (B = N/16 per "
                    f"dim, L = 10, Pfa = 1e-5, the paper's eq. (opt) thresholds), {per_shape} resident frames per "
                    f"shape; {group} frames per launch of each stage (rsft_execute_frames) recorded as CUDA graphs, "
                    f"all {len(fseq)} graphs in one rsft_graph_launch_batch"}


def frames_fold_roofline(R, torch, fplans, cubes, peak, groups=24, group=16, cap=BATCH_CAP):
    """The fold as the frames form launches it (16 frames per launch): CUDA events around every
    fold launch of `groups` rsft_execute_frames calls on the headline's two plans, all on one
    stream, so each fold launch runs alone on the GPU (in the recorded form the two plans' groups
    overlap, which shares the GPU between two folds and makes either launch look longer)."""
    dev = cubes[0].device
    one = torch.cuda.Stream()
    streams = [one, one]
    outs = []
    for s_ in streams:
        with torch.cuda.stream(s_):
            outs.append((torch.zeros(group * cap, dtype=torch.int64, device=dev),
                         torch.zeros(group * cap, dtype=torch.complex64, device=dev),
                         torch.zeros(group, dtype=torch.int64, device=dev)))
    seq = [cubes[k % len(cubes)] for k in range(group)]
    torch.cuda.synchronize()
    for fp in fplans:
        R.rsft_plan_timing(fp, True)
    before = [R.rsft_plan_get(fp, R.RSFT_GET_FRAMES_FOLD) for fp in fplans]
    for g in range(groups):
        i = g % 2
        loc, amp, cnt = outs[i]
        R.rsft_execute_frames(fplans[i], seq, cnt, located=loc, amp=amp, stream=streams[i])
    torch.cuda.synchronize()
    after = [R.rsft_plan_get(fp, R.RSFT_GET_FRAMES_FOLD) for fp in fplans]
    for fp in fplans:
        R.rsft_plan_timing(fp, False)
    ms = sum(a[0] - b[0] for a, b in zip(after, before))
    launches = sum(a[2] - b[2] for a, b in zip(after, before))
    frames = sum(a[1] - b[1] for a, b in zip(after, before))
    per_launch_s = ms / max(1.0, launches) / 1e3
    bytes_per_launch = int(R.rsft_plan_get(fplans[0], R.RSFT_GET_FOLD_BYTES)[0]) * (frames / max(1.0, launches))
    achieved = bytes_per_launch / per_launch_s / 1e9
    return {"achieved": achieved, "frac": achieved / peak, "launch_us": per_launch_s * 1e6,
            "frames_per_launch": frames / max(1.0, launches), "launches_timed": int(launches),
            "algorithmic_bytes_per_launch": int(bytes_per_launch)}


def per_pass_roofline(R, torch, wl, nv, seed, cubes, stream, peak, steps, lpp=4):
    """The fold with `lpp` loops per pass over the cube (ceil(L / lpp) passes, each reading the
    cube): the HBM-bound form of the same step, against the one fused compute-bound pass."""
    plan = R.rsft_plan_create(workload_desc(R, wl, nv, seed))
    R.rsft_plan_set_loops_per_pass(plan, lpp)
    dev = cubes[0].device
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    loc = torch.zeros(1 << 20, dtype=torch.int64, device=dev)
    amp = torch.zeros(1 << 20, dtype=torch.complex64, device=dev)
    for k in range(3):
        R.rsft_execute_async(plan, cubes[k % len(cubes)], count, stream=stream, located=loc, amp=amp)
    torch.cuda.synchronize()
    R.rsft_plan_timing(plan, True)
    for k in range(steps):
        R.rsft_execute_async(plan, cubes[k % len(cubes)], count, stream=stream, located=loc, amp=amp)
    torch.cuda.synchronize()
    st = R.rsft_plan_get(plan, R.RSFT_GET_STAGE_MS)
    n = max(1.0, st[6])
    fold_s = st[0] / n / 1e3
    fold_bytes = int(R.rsft_plan_get(plan, R.RSFT_GET_FOLD_BYTES)[0])
    passes = -(-wl.loops // lpp)
    plan.close()
    achieved = fold_bytes / fold_s / 1e9
    return {"bound": "hbm", "loops_per_pass": lpp, "passes": passes, "fold_us": fold_s * 1e6,
            "us_per_pass": fold_s * 1e6 / passes, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "algorithmic_bytes_per_execute": fold_bytes,
            "note": "same workload and kernel, the cube read once per pass of lpp loops (CUDA events over "
                    f"{steps} executes); frames/s is lower than the fused pass, HBM use per byte higher"}


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    import paper_1610_01050_gb300 as R
    from paper_1610_01050_gb300 import build as B
    import rsft_inputs as ri

    B.build()
    R.load_library()
    wl = ri.WORKLOADS[args.workload]
    F = max(1, args.frames)
    host, targets = [], []
    nv = wl.noise_var
    for fid in shard_frames(rank, F):
        cube, tg, _, nv = ri.workload_frame(args.workload, fid)
        host.append(torch.from_numpy(cube).pin_memory())
        targets.append(tg)
    dev = torch.device("cuda", local)
    cubes = [h.to(dev) for h in host]
    seed = ri.frame_seed(wl, 0)
    plan = R.rsft_plan_create(workload_desc(R, wl, nv, seed))
    cap = 1 << 20
    located = torch.zeros(cap, dtype=torch.int64, device=dev)
    amp = torch.zeros(cap, dtype=torch.complex64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    # detection quality on the ring (also a warm-up)
    pd, pfa, n_loc = rsft_quality(R, plan, wl, cubes, targets, located, cap)
    fps = max(1, args.frames_per_step)
    n_timed = args.steps * fps               # frames in each timed region
    n_warm = max(3, args.warmup) * fps

    for k in range(n_warm):
        R.rsft_execute_async(plan, cubes[k % F], count, stream=stream, located=located, amp=amp)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    # batched form: the same frames over concurrent lanes; the lane count is tuned on a few chunks
    bplan = R.rsft_plan_create(workload_desc(R, wl, nv, seed, max_located=BATCH_CAP))
    ring = [cubes[k % F] for k in range(BATCH_CHUNK)]
    bcounts = torch.zeros(BATCH_CHUNK, dtype=torch.int64, device=dev)
    bloc = torch.zeros(BATCH_CHUNK * BATCH_CAP, dtype=torch.int64, device=dev)
    bamp = torch.zeros(BATCH_CHUNK * BATCH_CAP, dtype=torch.complex64, device=dev)
    tune = {}
    for lanes in (1, 2, 3, 4):
        batched_frames(R, bplan, ring, BATCH_CHUNK, lanes, bcounts, bloc, bamp, stream)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        batched_frames(R, bplan, ring, 4 * BATCH_CHUNK, lanes, bcounts, bloc, bamp, stream)
        t1.record(stream)
        torch.cuda.synchronize()
        tune[lanes] = 4 * BATCH_CHUNK / (t0.elapsed_time(t1) / 1e3)
    best_lanes = max(tune, key=tune.get)
    if ws > 1:
        best_lanes = int(max_over_ranks(best_lanes, ws, dev))
    # the same frames as recorded executes (CUDA graphs), one per lane over 4 lanes
    glanes = 4
    gout = [(torch.zeros(BATCH_CAP, dtype=torch.int64, device=dev), torch.zeros(BATCH_CAP, dtype=torch.complex64, device=dev),
             torch.zeros(1, dtype=torch.int64, device=dev)) for _ in range(glanes)]
    graphs = [R.rsft_graph_create(bplan, cubes[k % F], gout[k][2], located=gout[k][0], amp=gout[k][1], lane=k)
              for k in range(glanes)]
    graph_frames(R, graphs, BATCH_CHUNK, stream)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    graph_frames(R, graphs, 4 * BATCH_CHUNK, stream)
    t1.record(stream)
    torch.cuda.synchronize()
    tune["graphs"] = 4 * BATCH_CHUNK / (t0.elapsed_time(t1) / 1e3)
    # the same frames 16 at a time through one launch per stage (rsft_execute_frames), recorded
    # as CUDA graphs on two plans of the workload so one group's fold overlaps the other's tail
    fplans = [bplan, R.rsft_plan_create(workload_desc(R, wl, nv, seed, max_located=BATCH_CAP))]
    fgroup = 16
    fouts = [(torch.zeros(fgroup * BATCH_CAP, dtype=torch.int64, device=dev),
              torch.zeros(fgroup * BATCH_CAP, dtype=torch.complex64, device=dev),
              torch.zeros(fgroup, dtype=torch.int64, device=dev)) for _ in fplans]
    fgraphs = [R.rsft_graph_create_frames(fp, [cubes[k % F] for k in range(fgroup)], o[2], located=o[0], amp=o[1])
               for fp, o in zip(fplans, fouts)]

    def frames_graphs(nframes):
        seq = [fgraphs[g % 2] for g in range(-(-nframes // fgroup))]
        for i in range(0, len(seq), BATCH_CHUNK):
            R.rsft_graph_launch_batch(seq[i:i + BATCH_CHUNK], stream=stream)

    frames_graphs(4 * fgroup)
    torch.cuda.synchronize()
    t0.record(stream)
    frames_graphs(4 * BATCH_CHUNK)
    t1.record(stream)
    torch.cuda.synchronize()
    tune["frames"] = 4 * BATCH_CHUNK / (t0.elapsed_time(t1) / 1e3)
    form = max(("graphs", "frames", "lanes"), key=lambda k: tune[best_lanes] if k == "lanes" else tune[k])
    if ws > 1:
        # every rank takes the form of rank 0's choice order: the largest code wins
        code = max_over_ranks(float({"lanes": 0, "graphs": 1, "frames": 2}[form]), ws, dev)
        form = {0: "lanes", 1: "graphs", 2: "frames"}[int(code)]
    use_graphs = form == "graphs"
    for k in range(n_warm):
        R.rsft_execute_async(plan, cubes[k % F], count, stream=stream, located=located, amp=amp)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()

    # per-stage device times from a pass with the plan's stage events on (the events themselves
    # add about 2 us a stage, so the plain frames/s below is timed with them off)
    R.rsft_plan_timing(plan, True)
    for k in range(min(n_timed, 200)):
        R.rsft_execute_async(plan, cubes[k % F], count, stream=stream, located=located, amp=amp)
    torch.cuda.synchronize()
    stage = R.rsft_plan_get(plan, R.RSFT_GET_STAGE_MS)
    R.rsft_plan_timing(plan, False)
    sampler = ClockSampler(uuid)
    time.sleep(0.5)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    sampler.mark(True)
    ev0.record(stream)
    for k in range(n_timed):
        R.rsft_execute_async(plan, cubes[k % F], count, stream=stream, located=located, amp=amp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_plain = ev0.elapsed_time(ev1)
    # the headline: the batched form over the same frames
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    if form == "graphs":
        graph_frames(R, graphs, n_timed, stream)
    elif form == "frames":
        frames_graphs(n_timed)
    else:
        batched_frames(R, bplan, ring, n_timed, best_lanes, bcounts, bloc, bamp, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(False)
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, ws, dev)
    ms_plain = max_over_ranks(ms_plain, ws, dev)
    value = whole_job_rate(ws, n_timed, ms)
    plain_value = whole_job_rate(ws, n_timed, ms_plain)

    # the fold as the frames form launches it (when that form is the headline's)
    ffold = frames_fold_roofline(R, torch, fplans, cubes, measured_peak()[0]) if form == "frames" else None
    # roofline of the dominant kernel (the fold): algorithmic bytes / average launch time
    fold_bytes = int(R.rsft_plan_get(plan, R.RSFT_GET_FOLD_BYTES)[0])
    timed = max(1.0, stage[6])
    fold_s = stage[0] / timed / 1e3
    peak, peak_kind = measured_peak()
    achieved = fold_bytes / fold_s / 1e9
    tensor_fold = int(R.rsft_plan_get(plan, R.RSFT_GET_FOLD_COPY)[0]) >= 100
    fold_source = "fold_tc.cu" if tensor_fold else "fold.cu"
    traffic = profile_traffic(args.workload, fold_source)
    stages = {k: stage[i] / timed * 1e3 for i, k in
              enumerate(["fold_us", "fft_detect_us", "vote_scatter_us", "stage2_us", "median_us", "execute_us"])}

    # end to end through the C ABI with host buffers: rsft_execute_host_batch, the copy of
    # frame f + 1 overlapping the RSFT of frame f (H2D of every cube and D2H of every result inside)
    e2e_steps = max(1, args.e2e_steps)
    hchunk = 16
    h_loc = torch.zeros(hchunk * BATCH_CAP, dtype=torch.int64).pin_memory()
    h_amp = torch.zeros(hchunk * BATCH_CAP, dtype=torch.complex64).pin_memory()
    h_cnt = torch.zeros(hchunk, dtype=torch.int64)
    hring = [host[k % F] for k in range(hchunk)]
    R.rsft_execute_host_batch(bplan, hring[:4], h_loc, h_cnt, amp=h_amp, stream=stream, allow_capacity=True)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    d2h, done = 0, 0
    while done < e2e_steps:
        m = min(hchunk, e2e_steps - done)
        R.rsft_execute_host_batch(bplan, hring[:m], h_loc, h_cnt, amp=h_amp, stream=stream, allow_capacity=True)
        d2h += int(8 * m + 16 * torch.clamp(h_cnt[:m], max=BATCH_CAP).sum())
        done += m
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws, dev)
    e2e_val = whole_job_rate(ws, e2e_steps, t_e2e * 1e3)

    for g_ in graphs + fgraphs:
        g_.close()
    fplans[1].close()
    bplan.close()
    def side(fn):
        """A secondary measurement: on one GPU a failure is recorded in its own field and the
        line still prints; with several ranks it propagates (a rank that skipped a collective
        would leave the others waiting)."""
        if ws > 1:
            return fn()
        try:
            return fn()
        except Exception as e:  # recorded, not hidden: the field carries the error
            return {"error": f"{type(e).__name__}: {e}"[:400]}

    side_frames = max(20, min(n_timed // 20, 200))
    refine = side(lambda: refinement(R, torch, plan, wl, cubes, targets, stream, cap))
    seg = side(lambda: segment_mode(R, torch, plan, wl, cubes, stream, dev, ws, located, amp, count,
                                    min(side_frames, 50)))
    dense = side(lambda: dense_comparator(R, torch, wl, nv, cubes, targets, stream, dev, ws, side_frames, 5, cap,
                                          value, matched_pfa=pfa if pfa > 0 else None))
    paper = side(lambda: paper_design(R, torch, wl, nv, seed, cubes, targets, stream, dev, ws, side_frames,
                                      located, amp, count, cap))
    estim = side(lambda: estimate_mode(R, torch, wl, seed, cubes, targets, stream, dev, ws, side_frames,
                                       located, amp, count, cap))
    mixed = side(lambda: mixed_batch(R, torch, ri, dev, ws, stream, n_frames=512))
    srur = side(lambda: srur_frames(R, torch, ri, dev, ws, stream, min(side_frames, 50)))
    per_pass = side(lambda: per_pass_roofline(R, torch, wl, nv, seed, cubes, stream, peak, side_frames))
    del cubes
    torch.cuda.empty_cache()
    c5 = side(lambda: c5_frames(R, torch, ri, dev, ws, stream, 10))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, host[0].numpy(), nv, seed)

    roofline_plain = {"bound": "hbm", "kernel": "permute_window_fold (" + ("fold_tc_kernel: tcgen05 3xTF32"
                      if tensor_fold else "fold_kernel: SIMT FP32") + "), one frame per launch", "achieved": achieved,
                      "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                      "peak_source": f"{peak_kind} (copy bandwidth)", "traffic": traffic,
                      "algorithmic_bytes_per_launch": fold_bytes, "launch_us": fold_s * 1e6,
                      "dram_gbs": traffic / fold_s / 1e9 if traffic else None,
                      "dram_note": "ncu DRAM bytes of one launch (traffic) over the same launch time: the "
                                   "sector-level rate, beside the useful-byte rate (achieved); the launch time "
                                   "from CUDA events of the plain executes"}
    if isinstance(ffold, dict):
        ftraffic = profile_traffic(args.workload + "_frames16", fold_source)
        roofline = {"bound": "hbm", "kernel": "permute_window_fold (fold_kernel: SIMT FP32), "
                    f"{ffold['frames_per_launch']:.0f} frames per launch as the headline's frames form runs it",
                    "achieved": ffold["achieved"], "peak": peak, "unit": "GB/s", "frac": ffold["frac"],
                    "peak_source": f"{peak_kind} (copy bandwidth)",
                    "traffic": ftraffic,
                    "algorithmic_bytes_per_launch": ffold["algorithmic_bytes_per_launch"],
                    "launch_us": ffold["launch_us"], "launches_timed": ffold["launches_timed"],
                    "dram_gbs": ftraffic / (ffold["launch_us"] / 1e6) / 1e9 if ftraffic else None,
                    "dram_note": "traffic: ncu DRAM bytes of one 16-frame fold launch (profiles/, the same source); "
                                 "launch time from CUDA events around each fold launch of rsft_execute_frames calls "
                                 "on the headline's two plans, one stream (each fold launch alone on the GPU)"}
    else:
        roofline = roofline_plain
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "frames_per_step": fps,
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": workload_name(wl),
                "frames_per_rank_ring": F,
                "l2": f"inputs larger than L2: ring of {F} frames, {F * int(np.prod(wl.shape)) * 8 / 1e6:.0f} MB",
                "parallelism": f"frames sharded over {ws} GPU(s), no collective on the data path",
                "form": {"graphs": f"batched: each frame one recorded execute (CUDA graph) on one of {glanes} lanes, "
                                   f"{BATCH_CHUNK} graphs per rsft_graph_launch_batch",
                         "frames": f"batched: {fgroup} frames per launch of each stage (rsft_execute_frames recorded as "
                                   f"a CUDA graph), graphs of two plans alternating",
                         "lanes": f"batched: frames spread over {best_lanes} concurrent lanes, {BATCH_CHUNK} frames "
                                  f"per rsft_execute_batch call"}[form] + " (the fastest form in the tuning)",
                "step": f"{fps} frames, each one whole RSFT",
                "design": "eq. (opt) with the binomial vote laws (RSFT_DESIGN_BINOMIAL)",
                "mu": int(R.rsft_plan_get(plan, R.RSFT_GET_MU)[0]),
                "pfa1": float(R.rsft_plan_get(plan, R.RSFT_GET_PFA1)[0]),
            },
            "detection": {"pd": pd, "pfa": pfa, "located_per_frame": n_loc,
                          "dense_at_same_pfa": dense.get("at_rsft_pfa") if isinstance(dense, dict) else None,
                          "note": "Pd: targets located within +-1 bin per dim; Pfa: located cells outside +-3-bin "
                                  "target boxes; the dense detector is run at the RSFT's measured Pfa"},
            "stages_us_per_frame": stages,
            "roofline": roofline,
            "roofline_one_frame": roofline_plain,
            "roofline_per_pass": per_pass,
            "e2e": {"value": e2e_val, "unit": "frames/s", "h2d_bytes_per_step": int(np.prod(wl.shape)) * 8,
                    "d2h_bytes_per_step": int(d2h / e2e_steps)},
            "plain": {"value": plain_value, "unit": "frames/s", "ms_per_frame": ms_plain / n_timed,
                      "note": "one frame per rsft_execute_async, back to back on one stream",
                      "batched_speedup": value / plain_value, "lanes_tuning_frames_per_s": tune},
            "dense_fft": dense,
            "mixed_batch": mixed,
            "segment_mode": seg,
            "srur": srur,
            "refine": refine,
            "paper_design": paper,
            "estimate_mode": estim,
            "c5_4d": c5,
            # kernels of the timed headline: one execute's launches per frame, or per group of
            # frames for the frames form (each stage launches once per group)
            "gpu_launches": int(stage[7]) * (-(-n_timed // fgroup) if form == "frames" else n_timed),
            "clocks": clocks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """`--profile N`: N back-to-back rsft_execute_async calls over the workload's ring of frames
    (headline plan), then exit.  The ring is the timed one (4 frames, larger than L2)."""
    import torch
    import paper_1610_01050_gb300 as R
    from paper_1610_01050_gb300 import build as B
    import rsft_inputs as ri
    B.build()
    R.load_library()
    wl = ri.WORKLOADS[args.workload]
    cubes, nv = [], wl.noise_var
    for fid in range(max(1, args.frames)):
        cube, _, _, nv = ri.workload_frame(args.workload, fid)
        cubes.append(torch.from_numpy(cube).cuda())
    plan = R.rsft_plan_create(workload_desc(R, wl, nv, ri.frame_seed(wl, 0)))
    cap = 1 << 20
    located = torch.zeros(cap, dtype=torch.int64, device="cuda")
    amp = torch.zeros(cap, dtype=torch.complex64, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    if args.profile_frames > 0:
        nf = args.profile_frames
        seq = [cubes[k % len(cubes)] for k in range(nf)]
        floc = torch.zeros(nf * cap, dtype=torch.int64, device="cuda")
        famp = torch.zeros(nf * cap, dtype=torch.complex64, device="cuda")
        fcnt = torch.zeros(nf, dtype=torch.int64, device="cuda")
        for _ in range(args.profile):
            R.rsft_execute_frames(plan, seq, fcnt, located=floc, amp=famp)
    else:
        for k in range(args.profile):
            R.rsft_execute_async(plan, cubes[k % len(cubes)], count, located=located, amp=amp)
    torch.cuda.synchronize()
    plan.close()


def main():
    args = parse()
    if args.profile > 0:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
