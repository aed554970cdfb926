#!/usr/bin/env python3
"""Benchmark of the Accessibility Field hot path on GB300.

One step = one 10 Hz LiDAR frame of the streaming pine workload (Mid-360-like
rosette, 20,000 returns, v = 2 cm, K = 64 of G = 128 directions): integrate
the scan into the map, then score the frame's voxel-deduplicated surface
points. The headline metric is point x orientation tests per second (a test is
one (confident point, candidate direction) pair decided), next to the
frame latency p50 / p99.

Passes over the same frames, each on a fresh map:
  A  device-resident inputs, per-step CUDA events, L2 flushed between steps
     -> value, latency, clocks;
  B  as A with per-kernel CUDA events inside the library -> roofline;
  C  af_frame_host from pinned host buffers (copies inside the step) -> e2e.
The CPU oracle is timed on a bounded sample of the same workload
(cpu_baseline); `--impl reference` times only the oracle.

Under torchrun with N > 1 every rank runs an independent replica (the path
has no exchange step); value = all ranks' tests / the slowest rank's time.

Other lines, each with the oracle timed beside it on a bounded sample:
  --batched    64 uneven scenes ticked together, against the per-scene path;
  --soft       the differentiable step: 100k points, 20 ascent steps each;
  --points     the stateful layer (triggers, budget, PCA normals, c and a);
  --large      the 40 x 40 m map at 1 cm: 3,000 frames, then every surface point;
  --large --batched  its eight pine orbits as eight scenes ticked together,
               against the per-scene path;
  --large --soft     the differentiable step on it (brick-sparse SDF view);
and variants of the default line: --projective, --clamp-signed, --ring
(the paper's yaw ring; with --points also --c2f), --score-split B.
--noalloc times the allocation-free integration into a dense box of the
pine map beside the map path's integration of the same frames.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point x orientation tests/s (10 Hz frame latency p99 alongside)"
UNIT = "tests/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batched", action="store_true",
                    help="the batched form (many scenes per tick) instead of the pine stream")
    ap.add_argument("--scenes", type=int, default=64)
    ap.add_argument("--soft", action="store_true",
                    help="the differentiable form on the pine map after 300 frames")
    ap.add_argument("--soft-points", type=int, default=100_000)
    ap.add_argument("--points", action="store_true",
                    help="the stateful point layer over the pine stream")
    ap.add_argument("--points-budget", type=int, default=16384)
    ap.add_argument("--points-trigger", choices=("sampled", "all", "brick"), default="sampled",
                    help="--points: changed voxels within r_u drawn 256 per frame (the paper's), "
                         "all of them, or the brick rule")
    ap.add_argument("--large", action="store_true",
                    help="the large map: 3,000 frames at 1 cm, then every surface point, K = 256")
    ap.add_argument("--score-split", type=int, default=None,
                    help="af_set_score_split budget (-1: one warp per point; default: library's)")
    ap.add_argument("--ring", action="store_true",
                    help="the paper's approach set, 180 yaw directions and a 70 degree cone")
    ap.add_argument("--projective", action="store_true",
                    help="projective integration over an octahedral range image (Tab. 3 ablation)")
    ap.add_argument("--c2f", action="store_true",
                    help="--points --ring: coarse-to-fine search (20 degrees, +-24 degrees, 0.3 m)")
    ap.add_argument("--noalloc", action="store_true",
                    help="af_integrate_scan_noalloc into a dense box of the pine map, "
                         "beside the map path's integration")
    ap.add_argument("--clamp-signed", action="store_true",
                    help="the [-tau, tau] clamp ablation (Tab. 4)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _frames(W, start, count):
    from paper_2608_06412_gb300 import workload
    out = []
    for f in range(start, start + count):
        fr, pts, nrm = workload.pine_frame(W, f)
        out.append((fr, pts, nrm))
    return out


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.t0 = self.t1 = None
        # the raw samples go to BENCH_CLOCKS_DIR if set, else the temporary directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}",
                                          f"--query-gpu={self.Q}", "--format=csv,noheader",
                                          "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except OSError:
            self.proc = None

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, p in rows for i in range(4)
                          if p[5 + i].lower() == "active"})
        sm = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# Oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_objs(W, tables: bool = True):
    import oracle
    p = W.map_params()
    cfg = oracle.Config(v=p["v"], tau=p["tau"], r_c=p["r_c"], cube_radius=p["cube_radius"],
                        clear_samples=p["clear_samples"],
                        dom_min=tuple(8 * b for b in W.dom_min),
                        dom_size=tuple(8 * b for b in W.dom_bricks), cone_cos=p["cone_cos"],
                        range_min=p["range_min"], range_max=p["range_max"],
                        clear_lo=p["clear_lo"], clear_hi=p["clear_hi"], w_min=p["w_min"],
                        w_cap=p["w_cap"])
    tool = oracle.Tool(**W.tool())
    # the kernel tables are built once, as the method precomputes them (Sec. 3.6)
    return oracle.Map(cfg), (tool, oracle.ScoreTables(cfg, tool, W.dirs) if tables else None)


def _oracle_frame(om, tool, W, frame, n_sample, rng):
    """Integrate one frame, score a random sample of its points; returns the
    per-frame estimate (tests, seconds) prorated from the sample."""
    fr, pts, nrm = frame
    t0 = time.perf_counter()
    om.integrate(fr.pts, fr.pose)
    t1 = time.perf_counter()
    sel = rng.choice(len(pts), min(n_sample, len(pts)), replace=False)
    lab, best, ds = om.score_tables(tool[1], pts[sel], nrm[sel], dir_scores=True)
    t2 = time.perf_counter()
    tests = int((ds >= 0).sum())
    scale = len(pts) / max(len(sel), 1)
    return tests * scale, (t1 - t0) + (t2 - t1) * scale, t1 - t0, t2 - t1, len(sel)


def cpu_baseline(W, frames, n_frames=6, n_sample=200):
    rng = np.random.default_rng(0)
    om, tool = _oracle_objs(W)
    tests = secs = 0.0
    t_int = t_sc = 0.0
    pts_scored = 0
    for k in range(n_frames):
        last = k == n_frames - 1
        fr = frames[k]
        if not last:
            t0 = time.perf_counter()
            om.integrate(fr[0].pts, fr[0].pose)
            t_int += time.perf_counter() - t0
            continue
        te, se, ti, ts, ns = _oracle_frame(om, tool, W, fr, n_sample, rng)
        tests, secs = te, se
        t_int += ti
        t_sc, pts_scored = ts, ns
    returns = sum(len(frames[k][0].pts) for k in range(n_frames))
    return {"value": tests / secs if secs > 0 else None, "unit": UNIT, "cores": 1,
            "kind": "oracle", "returns_per_s": returns / t_int if t_int > 0 else None,
            "sample": f"single-threaded C oracle: frames 0-{n_frames - 1} integrated "
                      f"({t_int / n_frames:.2f} s/frame), {pts_scored} random points of "
                      f"frame {n_frames - 1} scored in full ({t_sc:.2f} s, kernel tables "
                      f"built once beforehand); per-frame tests and time prorated to all "
                      f"points of that frame"}


def points_cpu_baseline(W, frames, n_frames=6, budget=400):
    """The oracle's stateful layer over the first frames of the stream with a
    per-frame budget: evaluations per second (integration, point set,
    triggers and evaluations all timed)."""
    import oracle
    om, (tool, _) = _oracle_objs(W)
    P = oracle.PointSet(om, oracle.PointsConfig(trig_tsdf=2 * W.params["v"], budget=budget),
                        tool, W.dirs)
    t0 = time.perf_counter()
    evals = 0
    for k in range(n_frames):
        fr = frames[k][0]
        evals += P.frame(fr.pts, fr.pose)
    secs = time.perf_counter() - t0
    return {"value": evals / secs if secs > 0 else None, "unit": "evaluations/s", "cores": 1,
            "kind": "oracle",
            "sample": f"single-threaded C oracle: the stateful layer over frames 0-{n_frames - 1} "
                      f"with {budget} evaluations per frame ({evals} evaluations, {secs:.1f} s)"}


def sample_cpu_baseline(W, frames, n_frames, n_points, seed=0):
    """The plain oracle on one workload: frames integrated, then a random
    sample of the last frame's points scored with kernel tables built once.
    Returns (tests, seconds, returns integrated, integration seconds)."""
    import oracle
    om, (tool, tables) = _oracle_objs(W)
    t0 = time.perf_counter()
    for k in range(n_frames):
        om.integrate(frames[k][0], frames[k][1])
    t1 = time.perf_counter()
    P, N = frames[n_frames - 1][2], frames[n_frames - 1][3]
    sel = np.random.default_rng(seed).choice(len(P), min(n_points, len(P)), replace=False)
    t2 = time.perf_counter()
    _, _, ds = om.score_tables(tables, P[sel], N[sel], dir_scores=True)
    t3 = time.perf_counter()
    returns = sum(len(frames[k][0]) for k in range(n_frames))
    return int((ds >= 0).sum()), t3 - t2, returns, t1 - t0


def large_cpu_baseline(W, frames, n_frames=5, n_points=30, every=16):
    """The plain oracle on the large map: the first frames integrated, then a
    random sample of the last one's points scored against every `every`-th
    direction (kernel tables for all 512 take minutes to build; a test costs
    the same whichever direction it is)."""
    import oracle
    om, _ = _oracle_objs(W, tables=False)
    tool = oracle.Tool(**W.tool())
    dirs = np.ascontiguousarray(W.dirs[::every])
    tables = oracle.ScoreTables(om.cfg, tool, dirs)
    t0 = time.perf_counter()
    for k in range(n_frames):
        om.integrate(frames[k][0], frames[k][1])
    t1 = time.perf_counter()
    P, N = frames[n_frames - 1][3], frames[n_frames - 1][4]
    sel = np.random.default_rng(0).choice(len(P), min(n_points, len(P)), replace=False)
    t2 = time.perf_counter()
    _, _, ds = om.score_tables(tables, P[sel], N[sel], dir_scores=True)
    t3 = time.perf_counter()
    tests = int((ds >= 0).sum())
    returns = sum(len(frames[k][0]) for k in range(n_frames))
    return {"value": tests / (t3 - t2), "unit": "tests/s", "cores": 1, "kind": "oracle",
            "returns_per_s": returns / (t1 - t0),
            "sample": f"single-threaded C oracle: frames 0-{n_frames - 1} integrated "
                      f"({(t1 - t0) / n_frames:.2f} s/frame), {len(sel)} random points of frame "
                      f"{n_frames - 1} scored against {len(dirs)} of the {len(W.dirs)} directions "
                      f"({tests} tests, {t3 - t2:.1f} s)"}


def run_reference(args, W, ws, rank):
    if rank != 0:
        return None
    rng = np.random.default_rng(1)
    om, tool = _oracle_objs(W)
    frames = _frames(W, 0, args.warmup + args.steps)
    for k in range(args.warmup):
        om.integrate(frames[k][0].pts, frames[k][0].pose)
    tests = secs = 0.0
    lat = []
    t_start = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        te, se, _, _, _ = _oracle_frame(om, tool, W, frames[k], 8, rng)
        tests += te
        secs += se
        lat.append(se * 1e3)
    measured = time.perf_counter() - t_start     # the work actually done, per step below
    value = tests / secs if secs > 0 else None
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": measured * 1e3 / max(args.steps, 1),
            "prorated_ms_per_frame": secs * 1e3 / max(args.steps, 1),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": W.name, "returns_per_frame": W.params["n_returns"],
                       "K": W.params["K"], "G": len(W.dirs), "voxel_m": W.params["v"]},
            "prorated_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                    "p99": float(np.percentile(lat, 99))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: the oracle integrates the frame and "
                                       "scores 8 random points of it with kernel tables "
                                       "built once (ms_per_step: the measured time of that "
                                       "work); value: tests and time prorated to all points "
                                       "of the frame (prorated_ms_per_frame)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# Roofline bookkeeping
# ---------------------------------------------------------------------------

def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


_L2_PEAK = None


def l2_peak():
    """The L2 read bandwidth of this GPU measured by the library's own probe
    (af_probe_l2_read: an L2-resident working set read with 16-byte L2-only
    loads, best launch of 20), the best over 24 and 48 MiB working sets."""
    global _L2_PEAK
    if _L2_PEAK is None:
        from paper_2608_06412_gb300 import af
        runs = {mb: af.probe_l2_read(mb << 20, reps=40, launches=20) for mb in (24, 48)}
        best = max(runs, key=runs.get)
        _L2_PEAK = (runs[best], f"measured: af_probe_l2_read, {best} MiB L2-resident working "
                                f"set, 16-byte ld.global.cg, best of 20 launches "
                                f"({', '.join(f'{m} MiB {v:.0f} GB/s' for m, v in runs.items())})")
    return _L2_PEAK


def integration_counts(W, frames, caps, sample, integrate_fn=None):
    """Per frame of `sample` (frame indices): accepted returns N_acc, voxels
    whose (S, w) the scan changed U_vox (the exported map before and after
    the frame, compared brick by brick), and bricks the scan touched B_dirty
    (the library's stats). Untimed; a map of its own."""
    from paper_2608_06412_gb300 import af
    import torch
    g = af.Map(W.af_config(**caps))
    out = []

    def words(e):
        keys = (e["key"].astype(np.int64) * np.array([1, 1 << 21, 1 << 42])).sum(1)
        return keys, (e["S"].astype(np.int64) << 20) | e["w"].astype(np.int64)

    for k in range(max(sample) + 1):
        xyz = torch.from_numpy(frames[k][0].pts).cuda()
        if k in sample:
            kb, wb = words(g.export_blocks())
            s0 = g.stats()
        g.integrate_scan(xyz, frames[k][0].pose)
        if k in sample:
            ka, wa = words(g.export_blocks())
            s1 = g.stats()
            order = np.argsort(kb)
            pos = np.searchsorted(kb[order], ka) if len(kb) else np.zeros(len(ka), np.int64)
            pos = np.minimum(pos, max(len(kb) - 1, 0))
            old = (len(kb) > 0) & (kb[order][pos] == ka) if len(kb) else np.zeros(len(ka), bool)
            prev = np.zeros_like(wa)
            prev[old] = wb[order][pos[old]]
            out.append(dict(n_ret=len(frames[k][0].pts),
                            n_acc=s1["returns_accepted"] - s0["returns_accepted"],
                            u_vox=int((wa != prev).sum()),
                            b_dirty=s1["blocks_dirty_last"]))
    g.close()
    return out


# Single-precision operations of one (return, cube voxel) pair as the method
# states them (Sec. 3.2): voxel centre 3 x (convert, add, multiply); a = x - p
# (3); |a|^2 (5); a . b (5); the cosine (sqrt, multiply, divide) and its test
# (4); x - q (3); |x - q|^2 (5); sqrt (1); d (1); clamp (2); quantisation
# (multiply, convert: 2); the accumulation (1).
INTEGRATION_OPS_PER_PAIR = 41


def fp32_peak_gops(device: int = 0):
    """FP32 operation issue peak: SMs x 128 FP32 lanes x the maximum SM clock
    (MEASURED_PEAKS.json's sm_max_mhz, else 2070 MHz); one op per lane per
    clock, since the path's arithmetic is separately rounded (no FMA)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz, kind = 2070.0, "nominal maximum SM clock"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        if d.get("sm_max_mhz"):
            mhz, kind = float(d["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    return sms * 128 * mhz * 1e6 / 1e9, f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz ({kind})"


# Algorithmic bytes of one integration (the count of the roofline table, with this
# library's 8-byte voxel word): 12 B per return in, a read and a write of the
# 8-byte word of every voxel the scan updates, and per touched brick its 512
# words (4096 B) and cleared marks (64 B) read and its occupied / known view
# (2 x 64 B) written.
def integration_bytes(c):
    return 12 * c["n_ret"] + 16 * c["u_vox"] + (4096 + 64 + 128) * c["b_dirty"]


def score_bytes_per_test(W, tool=None, dirs=None) -> float:
    """Algorithmic bytes of one point x orientation test: the occupied and
    known bits (2 bits per voxel) of every voxel the test's tool kernel,
    corridor kernel and three arm samples cover, with no early exit; the
    mean over the direction table."""
    from paper_2608_06412_gb300 import af
    t = W.af_tool() if tool is None else tool
    v = W.params["v"]
    vox = [len(af.kernel_offsets(t, v, u, af.KERNEL_TOOL)) +
           len(af.kernel_offsets(t, v, u, af.KERNEL_CORRIDOR)) + 3
           for u in (W.dirs if dirs is None else dirs)]
    return 2.0 * float(np.mean(vox)) / 8.0

# per scored point: 24 B of point + normal in, 3 B of label + best out
SCORE_BYTES_PER_POINT = 27.0

# DRAM bytes (read + write) per launch from one ncu capture of the benchmark
# (profiles/), valid only while the kernel's sources hash as recorded.
TRAFFIC = {
    "k_score": (10053760, {"paper_2608_06412_gb300/csrc/af_score.cu": "6a62001b84d4e0b3",
                        "paper_2608_06412_gb300/csrc/af_score.cuh": "c56e18e35201957e",
                        "paper_2608_06412_gb300/csrc/af_internal.cuh": "ee1a297df623f66b"}),
}


# L2 traffic of k_score per launch (lts__t_sectors.sum x 32 B) from the same
# capture (profiles/k_score_pine_stream.md), keyed like TRAFFIC; reported
# against the measured L2 read peak beside the algorithmic fraction.
L2_TRAFFIC = {"k_score": 375335248}


def _l2(kernel: str, avg_ms: float, peak: float):
    if kernel not in L2_TRAFFIC or _traffic(kernel) is None:
        return None
    b = L2_TRAFFIC[kernel]
    rate = b / (avg_ms * 1e-3) / 1e9
    return {"traffic": b, "achieved": rate, "peak": peak, "unit": "GB/s", "frac": rate / peak,
            "what": "L2 sectors moved (32 B each) per launch / launch time"}


def _traffic(kernel: str):
    import hashlib
    if kernel not in TRAFFIC:
        return None
    nbytes, files = TRAFFIC[kernel]
    for path, digest in files.items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != digest:
                return None
    return nbytes


def reduce_over_ranks(tests: float, total_ms: float, ws: int, device=None):
    """Whole-job totals of independent replicas: the tests of all ranks, and
    the slowest rank's timed milliseconds."""
    if ws <= 1:
        return tests, total_ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([tests], dtype=torch.float64, device=device)
    mm = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    dist.all_reduce(mm, op=dist.ReduceOp.MAX)
    return float(tt.item()), float(mm.item())


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_ours(args, W, ws, rank, local):
    import torch
    from paper_2608_06412_gb300 import af

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nfr = args.warmup + args.steps
    frames = _frames(W, 0, nfr)
    from paper_2608_06412_gb300.workload import BENCH_CAPS
    from paper_2608_06412_gb300 import synth
    caps = dict(BENCH_CAPS, clamp_signed=int(args.clamp_signed))
    tool, dirs = W.af_tool(), W.dirs
    if args.ring:   # the paper's approach set: 180 yaw directions, 70 degree cone
        tool.cos_theta_max = synth.COS_70
        dirs = synth.yaw_ring(180)

    def integrate(g, k):
        if args.projective:
            g.integrate_scan_projective(d_xyz[k], frames[k][0].pose, 812)
        else:
            g.integrate_scan(d_xyz[k], frames[k][0].pose)

    d_xyz = [torch.from_numpy(f[0].pts).to(dev) for f in frames]
    d_pts = [torch.from_numpy(f[1]).to(dev) for f in frames]
    d_nrm = [torch.from_numpy(f[2]).to(dev) for f in frames]
    lab = torch.empty(1 << 16, dtype=torch.uint8, device=dev)
    best = torch.empty(1 << 16, dtype=torch.int16, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)   # 256 MiB > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def pass_device(profile: bool, clocks: Clocks | None):
        g = af.Map(W.af_config(**caps))
        g.set_tool(tool, dirs)
        if args.score_split is not None:
            g.set_score_split(args.score_split)
        for k in range(args.warmup):
            integrate(g, k)
            m = len(d_pts[k])
            g.score(d_pts[k], d_nrm[k], lab[:m], best[:m])
        torch.cuda.synchronize()
        st0 = g.stats()
        g.profile(profile)
        if profile:
            g.profile_read(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.mark(True)
        for i, k in enumerate(range(args.warmup, nfr)):
            flush.zero_()
            ev[i][0].record(stream)
            integrate(g, k)
            m = len(d_pts[k])
            g.score(d_pts[k], d_nrm[k], lab[:m], best[:m])
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        if clocks:
            clocks.mark(False)
        st1 = g.stats()
        ms = [a.elapsed_time(b) for a, b in ev]
        prof = g.profile_read(reset=True) if profile else None
        g.close()
        return ms, st0, st1, prof

    clocks = Clocks(local)
    clocks.start()
    ms, st0, st1, _ = pass_device(False, clocks)
    clk = clocks.stop()
    tests = st1["tests"] - st0["tests"]
    total_ms = sum(ms)

    # per-kernel times (pass B)
    msB, sB0, sB1, prof = pass_device(True, None)

    # e2e through af_frame_host with pinned host buffers (pass C)
    e2e = None
    if not args.no_e2e and not args.projective and not args.ring and not args.clamp_signed:
        g = af.Map(W.af_config(**caps))
        g.set_tool(W.af_tool(), W.dirs)
        if args.score_split is not None:
            g.set_score_split(args.score_split)
        pin = []
        for fr, pts, nrm in frames:
            pin.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                             for a in (fr.pts, pts, nrm)))
        hl = torch.empty(1 << 16, dtype=torch.uint8).pin_memory()
        hb = torch.empty(1 << 16, dtype=torch.int16).pin_memory()
        lib = af.load()
        import ctypes as C

        def frame_host(k):
            x, p, n = pin[k]
            pose = np.ascontiguousarray(frames[k][0].pose, np.float32).reshape(16)
            st = lib.af_frame_host(g._h, C.c_void_p(x.data_ptr()), x.shape[0],
                                   pose.ctypes.data_as(C.c_void_p), C.c_void_p(p.data_ptr()),
                                   C.c_void_p(n.data_ptr()), p.shape[0],
                                   C.c_void_p(hl.data_ptr()), C.c_void_p(hb.data_ptr()),
                                   C.c_void_p(stream.cuda_stream))
            if st != 0:
                raise RuntimeError(f"af_frame_host failed: {st}")

        for k in range(args.warmup):
            frame_host(k)
        e0 = g.stats()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.warmup, nfr):
            frame_host(k)
        t1 = time.perf_counter()
        barrier()
        e1 = g.stats()
        h2d = sum(12 * len(frames[k][0].pts) + 24 * len(frames[k][1])
                  for k in range(args.warmup, nfr)) / args.steps
        d2h = sum(3 * len(frames[k][1]) + 4 for k in range(args.warmup, nfr)) / args.steps
        e2e_tests = e1["tests"] - e0["tests"]
        e2e = {"value": e2e_tests / (t1 - t0), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": (t1 - t0) * 1e3 / args.steps}
        g.close()

    tests_all, total_ms_max = reduce_over_ranks(float(tests), total_ms, ws, dev)

    returns = sum(len(frames[k][0].pts) for k in range(args.warmup, nfr))
    hbm, hbm_kind = _peaks()
    l2, l2_kind = l2_peak()
    # dominant kernel and its roofline
    prof = {k: v for k, v in prof.items() if v[0] > 0}
    kt = {k: v[1] for k, v in prof.items()}
    dom = max(kt, key=kt.get)
    # one call per slot and step; a scoring call with work sharing is three kernels
    n_launch = args.steps
    avg_ms = kt[dom] / n_launch
    # the views the scorer reads stay resident in L2 (91.5% L2 hits), so L2 bounds it
    roof = {"kernel": dom, "bound": "l2", "unit": "GB/s", "peak": l2, "peak_kind": l2_kind,
            "traffic": _traffic(dom),
            "kernel_ms": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
            "kernel_share": {k: round(v / max(sum(kt.values()), 1e-9), 4) for k, v in kt.items()}}
    if dom == "k_score":
        bpt = score_bytes_per_test(W, tool, dirs)
        tests_l = (sB1["tests"] - sB0["tests"]) / max(n_launch, 1)
        pts_l = (sB1["points_scored"] - sB0["points_scored"]) / max(n_launch, 1)
        alg = bpt * tests_l + SCORE_BYTES_PER_POINT * pts_l
        roof["algorithmic_bytes_per_launch"] = alg
        roof["bytes_per_test"] = bpt
        roof["achieved"] = alg / (avg_ms * 1e-3) / 1e9
        roof["frac"] = roof["achieved"] / l2
        roof["hbm"] = {"peak": hbm, "peak_kind": hbm_kind, "frac": roof["achieved"] / hbm}
        roof["l2_sectors"] = _l2(dom, avg_ms, l2)
    else:
        roof["achieved"] = None
        roof["frac"] = None
    # integration (k_alloc + k_integrate + k_bitview): its bytes are few and
    # stay in L2, its arithmetic is the bound -- single-precision operations
    # per (return, cube voxel) pair against the FP32 issue rate; the L2 figure
    # beside it, with counts taken on sample frames of the same stream
    integ = None
    if not args.projective and all(k in kt for k in ("k_alloc", "k_integrate", "k_bitview")):
        sample = sorted({args.warmup, (args.warmup + nfr) // 2, nfr - 1})
        counts = integration_counts(W, frames, caps, sample)
        ib = float(np.mean([integration_bytes(c) for c in counts]))
        n_acc = float(np.mean([c["n_acc"] for c in counts]))
        cube = (2 * W.params["cube_radius"] + 1) ** 3
        ops = INTEGRATION_OPS_PER_PAIR * n_acc * cube
        ims = sum(kt[k] for k in ("k_alloc", "k_integrate", "k_bitview")) / args.steps
        alu = fp32_peak_gops(local)
        integ = {"kernels": ["k_alloc", "k_integrate", "k_bitview"], "bound": "alu",
                 "unit": "Gop/s", "peak": alu[0], "peak_kind": alu[1],
                 "algorithmic_ops_per_frame": ops, "ops_per_pair": INTEGRATION_OPS_PER_PAIR,
                 "pairs_per_frame": n_acc * cube, "ms_per_frame": ims,
                 "k_integrate_ms": kt["k_integrate"] / args.steps,
                 "achieved": ops / (ims * 1e-3) / 1e9, "frac": ops / (ims * 1e-3) / 1e9 / alu[0],
                 "l2": {"algorithmic_bytes_per_frame": ib, "peak": l2,
                        "achieved": ib / (ims * 1e-3) / 1e9,
                        "frac": ib / (ims * 1e-3) / 1e9 / l2,
                        "bytes": "12 N_ret + 16 U_vox + (4096 + 64 + 128) B_dirty"},
                 "per_frame_counts": {"frames": sample,
                                      "returns": [c["n_ret"] for c in counts],
                                      "returns_accepted": [c["n_acc"] for c in counts],
                                      "voxels_updated": [c["u_vox"] for c in counts],
                                      "bricks_touched": [c["b_dirty"] for c in counts]}}
    return {
        "metric": METRIC, "value": tests_all / (total_ms_max / 1e3), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
        "config": {"workload": W.name, "returns_per_frame": W.params["n_returns"],
                   "K": W.params["K"], "G": len(dirs), "voxel_m": W.params["v"],
                   "frames": f"{args.warmup}..{nfr - 1}",
                   "score_split": args.score_split if args.score_split is not None else "default",
                   "integration": "projective (812^2 octahedral cells)" if args.projective
                   else "scan-centric",
                   "clamp": "[-tau, tau]" if args.clamp_signed else "[0, tau]",
                   "directions": "yaw ring, 70 deg cone" if args.ring else "Fibonacci sphere",
                   "l2": "flushed between steps (256 MiB write)"},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                       "max": float(max(ms))},
        "returns_per_s": returns / (total_ms / 1e3),
        "tests_per_step": tests / args.steps,
        "roofline": roof,
        "roofline_integration": integ,
        "e2e": e2e,
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
        "_frames": frames,
    }


def run_batched(args, local):
    """Batched form: 64 scenes of uneven size (1-4 pines or clutter, 2k-60k
    returns per frame, three tools, K in {16, 64, 128}) ticked together, one
    graph launch per tick; the same frames then go through the per-scene path
    (af_integrate_scan + af_score per scene) for comparison. Each scene cycles
    through 3 pre-generated frames."""
    import torch
    from paper_2608_06412_gb300 import af, workload
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    S = workload.batch_scenes(args.scenes)
    nfr = 3
    frames = [[workload.pine_frame(W, f) for f in range(nfr)] for W in S]
    d_in = [[(torch.from_numpy(fr.pts).to(dev), fr.pose, torch.from_numpy(p).to(dev),
              torch.from_numpy(n).to(dev)) for fr, p, n in fs] for fs in frames]
    outs = [(torch.empty(max(len(fs[f][1]) for f in range(nfr)), dtype=torch.uint8, device=dev),
             torch.empty(max(len(fs[f][1]) for f in range(nfr)), dtype=torch.int16, device=dev))
            for fs in frames]
    caps = dict(hash_capacity=1 << 18, pool_blocks=1 << 16, max_returns=1 << 16,
                max_points=1 << 16)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    warm, steps = max(args.warmup, 20), (args.steps if args.steps <= 100 else 30)

    def items(t):
        out = []
        for s in range(len(S)):
            xyz, pose, p, n = d_in[s][t % nfr]
            out.append((xyz, pose, p, n, outs[s][0][:len(p)], outs[s][1][:len(p)]))
        return out

    def run(batched: bool):
        maps = [af.Map(W.af_config(**caps)) for W in S]
        for W, m in zip(S, maps):
            m.set_tool(W.af_tool(), W.dirs)
        batch = af.Batch(maps) if batched else None

        def tick(t):
            it = items(t)
            if batched:
                batch.tick(it)
            else:
                for m, (xyz, pose, p, n, lab, best) in zip(maps, it):
                    m.integrate_scan(xyz, pose)
                    m.score(p, n, lab, best)
            return it

        for t in range(warm):
            tick(t)
        torch.cuda.synchronize()
        t0 = sum(m.stats()["tests"] for m in maps)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            it = tick(warm + i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        tests = sum(m.stats()["tests"] for m in maps) - t0
        labels = [np.concatenate([x[4].cpu().numpy(), x[5].cpu().numpy().view(np.uint8)])
                  for x in it]
        tuning = batch.tuning() if batched else None
        if batch:
            batch.close()
        for m in maps:
            m.close()
        return ms, tests, labels, tuning

    msb, testsb, labb, tuning = run(True)
    msp, testsp, labp, _ = run(False)
    agree = float(np.mean([np.array_equal(a, b) for a, b in zip(labb, labp)]))
    returns = sum(len(frames[s][(warm + i) % nfr][0].pts) for s in range(len(S))
                  for i in range(steps))
    return {
        "metric": "batched point x orientation tests/s", "value": testsb / (sum(msb) / 1e3),
        "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": sum(msb) / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
        "config": {"workload": f"batched_{len(S)}_scenes_2k_60k_returns",
                   "tools": "r 3/4/6 cm, L 15/25/40 cm, corridor 0.5/1.0/1.5 m",
                   "K": "16/64/128", "l2": "flushed between steps (256 MiB write)"},
        "latency_ms": {"p50": float(np.percentile(msb, 50)), "p99": float(np.percentile(msb, 99))},
        "returns_per_s": returns / (sum(msb) / 1e3),
        "tuning": tuning,
        "per_scene_path": {"value": testsp / (sum(msp) / 1e3), "ms_per_step": sum(msp) / steps,
                           "latency_ms": {"p50": float(np.percentile(msp, 50)),
                                          "p99": float(np.percentile(msp, 99))}},
        "speedup_vs_per_scene": (sum(msp) / steps) / (sum(msb) / steps),
        "label_agreement": agree,
        "tests_equal": testsb == testsp,
        "cpu_baseline": None if args.no_cpu_baseline else batched_cpu_baseline(S, frames),
    }


def batched_cpu_baseline(S, frames, n_scenes=2, n_points=40):
    """The plain oracle on the first scenes of the batch, each on its own
    three frames and tool, tests/s over the scored samples."""
    tests = secs = 0.0
    for W, fs in zip(S[:n_scenes], frames[:n_scenes]):
        t, sec, _, _ = sample_cpu_baseline(W, [(fr.pts, fr.pose, p, n) for fr, p, n in fs],
                                           len(fs), n_points)
        tests += t
        secs += sec
    return {"value": tests / secs if secs > 0 else None, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"single-threaded C oracle: scenes 0-{n_scenes - 1} of the batch, each "
                      f"integrated from its frames, then {n_points} random points of its last "
                      f"frame scored with its tool (kernel tables built once)"}


SOFT_METRIC = ("soft clearance evaluations/s (plain scoring of 100k points, then 20 ascent "
               "steps from each accessible point's best orientation)")
SOFT_UNIT = "evaluations/s"
SOFT_STEPS = 20
SOFT_LR = dict(lr_dir=0.05, lr_h=0.005, h_max=0.05)


def soft_cpu_baseline(W, frames, P, N, n_points=40, n_frames=6):
    """The oracle's differentiable step on a bounded sample: a map of the
    first frames, then plain scoring, start, soft clearance and refinement
    of n_points points."""
    import oracle
    from paper_2608_06412_gb300 import af
    om, (tool, tables) = _oracle_objs(W)
    for fr, _, _ in frames[:n_frames]:
        om.integrate(fr.pts, fr.pose)
    sel = np.random.default_rng(2).choice(len(P), n_points, replace=False)
    p, nrm = P[sel], N[sel]
    t0 = time.perf_counter()
    lab, best = om.score_tables(tables, p, nrm)
    acc = (lab == 1) & (best >= 0)
    u0 = np.where(acc[:, None], W.dirs[np.maximum(best, 0)], np.nan).astype(np.float32)
    z = np.zeros(n_points, np.float32)
    om.soft_clearance(tool, p[acc], 1, u0[acc], z[acc], z[acc], z[acc], af.TAU_S)
    om.soft_refine(tool, p[acc], 1, u0[acc], z[acc], z[acc], z[acc], SOFT_STEPS,
                   tau_s=af.TAU_S, **SOFT_LR)
    secs = time.perf_counter() - t0
    evals = int(acc.sum()) * (SOFT_STEPS + 2)
    return {"value": evals / secs, "unit": SOFT_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"single-threaded C oracle: map of frames 0-{n_frames - 1}, then plain "
                      f"scoring of {n_points} random points and the soft step of the "
                      f"{int(acc.sum())} accessible ones ({secs:.1f} s)"}


def run_soft(args, local):
    """Differentiable form on the pine map after 300 frames with 100k surface
    points. One step: plain scoring of the points (K = 64 of G = 128), the
    start direction of each accessible point (its best), its soft clearance,
    and 20 ascent steps on (alpha, beta, h) in one launch. Also timed: the
    soft clearance over all K hemisphere orientations of every point (the
    field, 6.4M pairs), the heaviest use of the forward kernel."""
    import torch
    from paper_2608_06412_gb300 import af, synth, workload
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = workload.pine_stream()
    frames = _frames(W, 0, 300)
    P, N = workload.soft_points(frames, W.params["v"], args.soft_points)
    K = W.params["K"]
    m = len(P)
    caps = dict(workload.BENCH_CAPS, max_points=max(m, workload.BENCH_CAPS["max_points"]))
    g = af.Map(W.af_config(**caps))
    g.set_tool(W.af_tool(), W.dirs)
    for fr, _, _ in frames:
        g.integrate_scan(torch.from_numpy(fr.pts).to(dev), fr.pose)
    torch.cuda.synchronize()
    Pd, Nd = torch.from_numpy(P).to(dev), torch.from_numpy(N).to(dev)
    lab = torch.empty(m, dtype=torch.uint8, device=dev)
    best = torch.empty(m, dtype=torch.int16, device=dev)
    u0 = torch.empty((m, 3), dtype=torch.float32, device=dev)
    z = torch.zeros(m, dtype=torch.float32, device=dev)
    al, be, hh, c0, c, cmin = (torch.empty(m, dtype=torch.float32, device=dev) for _ in range(6))
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    steps, warm = max(1, min(args.steps, 50)), max(args.warmup, 3)

    def step(p_d=Pd, n_d=Nd):
        g.score(p_d, n_d, lab, best)
        g.soft_start(lab, best, out=u0)
        g.soft_clearance_raw(p_d, u0, z, z, z, 1, out=c0)
        al.zero_()
        be.zero_()
        hh.zero_()
        g.soft_refine(p_d, u0, al, be, hh, 1, steps=SOFT_STEPS, out=(c, cmin), **SOFT_LR)

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        for i in range(k):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    n_acc = int((lab == af.ACCESSIBLE).sum().item())
    clocks = Clocks(local)
    clocks.start()
    clocks.mark(True)
    ms = timed(step, steps)
    clocks.mark(False)
    clk = clocks.stop()
    evals = n_acc * (SOFT_STEPS + 2)

    g.profile(True)
    g.profile_read(reset=True)
    timed(step, 3)
    prof = g.profile_read(reset=True)
    kt = {k: v for k, v in prof.items() if v[0] > 0}

    # the field: soft clearance of every point at its K hemisphere orientations
    table = synth.fibonacci_hemisphere(K, W.tool()["cos_theta_max"])
    uf = torch.empty((m * K, 3), dtype=torch.float32, device=dev)
    zf = torch.zeros(m * K, dtype=torch.float32, device=dev)
    cf = torch.empty(m * K, dtype=torch.float32, device=dev)

    def field():
        g.soft_seed(Nd, table, out=uf)
        g.soft_clearance_raw(Pd, uf, zf, zf, zf, K, out=cf)

    field()
    g.profile_read(reset=True)
    ms_field = timed(field, max(3, steps // 4))
    prof_f = g.profile_read(reset=True)
    g.profile(False)

    # outcome of one step
    step()
    torch.cuda.synchronize()
    acc = (lab == af.ACCESSIBLE).cpu().numpy()
    gain = (c - c0).cpu().numpy()[acc]
    cmin_h = cmin.cpu().numpy()[acc]

    # end to end: points and normals from pinned host memory; labels, best
    # directions and refined poses back
    hP, hN = torch.from_numpy(P).pin_memory(), torch.from_numpy(N).pin_memory()
    outs = [torch.empty(m, dtype=torch.float32).pin_memory() for _ in range(5)]
    hl = torch.empty(m, dtype=torch.uint8).pin_memory()
    hb = torch.empty(m, dtype=torch.int16).pin_memory()
    dP, dN = torch.empty_like(Pd), torch.empty_like(Nd)

    def e2e_step():
        dP.copy_(hP, non_blocking=True)
        dN.copy_(hN, non_blocking=True)
        step(dP, dN)
        hl.copy_(lab, non_blocking=True)
        hb.copy_(best, non_blocking=True)
        for h_t, d_t in zip(outs, (al, be, hh, c, cmin)):
            h_t.copy_(d_t, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    t_e2e = (time.perf_counter() - t0) / steps

    total = sum(ms)
    share = sum(v[1] for v in kt.values())
    dom = max(kt, key=lambda k: kt[k][1])
    roof = {"kernel": dom, "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in kt.items()},
            "kernel_share": {k: round(v[1] / share, 4) for k, v in kt.items()}}
    n_field = m * K
    out = {
        "metric": SOFT_METRIC, "value": evals / (total / steps / 1e3), "unit": SOFT_UNIT,
        "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": total / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"soft_refine_pine_300_frames_{m}_points_K{K}",
                   "points": m, "K": K, "G": len(W.dirs), "refine_steps": SOFT_STEPS,
                   **SOFT_LR, "tau_s": af.TAU_S, "l2": "flushed between steps (256 MiB write)"},
        "points_per_s": m / (total / steps / 1e3),
        "accessible_points": n_acc,
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "roofline": roof,
        "gpu_launches": int(round(sum(v[0] for v in kt.values()) / 3 * steps)),
        "labels": "the plain path's (exact); refinement changes directions and standoffs only",
        "refine": {"gain_m_mean": float(gain.mean()) if len(gain) else None,
                   "gain_m_p10": float(np.percentile(gain, 10)) if len(gain) else None,
                   "gain_m_p90": float(np.percentile(gain, 90)) if len(gain) else None,
                   "hard_clear_after": float((cmin_h > 0).mean()) if len(cmin_h) else None},
        "field": {"pairs": n_field, "ms": sum(ms_field) / len(ms_field),
                  "evaluations_per_s": n_field / (sum(ms_field) / len(ms_field) / 1e3),
                  "kernel_ms": {k: round(v[1] / v[0], 4) for k, v in prof_f.items() if v[0]}},
        "e2e": {"value": evals / t_e2e, "unit": SOFT_UNIT, "h2d_bytes_per_step": 24 * m,
                "d2h_bytes_per_step": 23 * m, "ms_per_step": t_e2e * 1e3},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = soft_cpu_baseline(W, frames, P, N)
    g.close()
    return out


LARGE_CAPS = dict(hash_capacity=1 << 23, pool_blocks=1 << 22, max_returns=1 << 15,
                  max_points=1 << 20)


def run_large(args, local):
    """The large map (8 pines on a noisy 40 x 40 m ground, 3,000 frames of
    20k returns, v = 1 cm, tau = 4 cm, K = 256 of G = 512, 1.5 m corridor):
    the whole stream integrated frame by frame, then every surface point of
    it (one per voxel hit) scored in chunks of 2^20. The occupancy views are
    several GB, far beyond L2, so no flush is needed between steps."""
    from paper_2608_06412_gb300 import workload
    W = workload.large_map()
    # frames come from spawned workers, before the first CUDA call
    frames = workload.large_frames(W, range(W.params["frames"]))
    import torch
    from paper_2608_06412_gb300 import af
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = af.Map(W.af_config(**LARGE_CAPS))
    g.set_tool(W.af_tool(), W.dirs)
    d_xyz = [torch.from_numpy(f[0]).to(dev) for f in frames]
    stream = torch.cuda.current_stream()
    # integration: every frame, CUDA events around each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in frames]
    clocks = Clocks(local)
    clocks.start()
    clocks.mark(True)
    for k, f in enumerate(frames):
        ev[k][0].record(stream)
        g.integrate_scan(d_xyz[k], f[1])
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ims = [a.elapsed_time(b) for a, b in ev]
    if g.sync_status() != 0:
        raise RuntimeError("large map: capacity exceeded")
    del d_xyz
    # every surface point of the stream, one per voxel (first occurrence)
    P = np.concatenate([f[3] for f in frames])
    N = np.concatenate([f[4] for f in frames])
    v = np.float64(np.float32(W.params["v"]))
    ijk = np.floor(P.astype(np.float64) / v).astype(np.int64) + (1 << 20)
    key = ijk[:, 0] | (ijk[:, 1] << 21) | (ijk[:, 2] << 42)
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)
    P = torch.from_numpy(np.ascontiguousarray(P[first])).to(dev)
    N = torch.from_numpy(np.ascontiguousarray(N[first])).to(dev)
    m = len(first)
    chunk = LARGE_CAPS["max_points"]
    lab = torch.empty(chunk, dtype=torch.uint8, device=dev)
    best = torch.empty(chunk, dtype=torch.int16, device=dev)
    for _ in range(max(args.warmup, 3)):          # warm-up: the first chunk
        g.score(P[:chunk], N[:chunk], lab[:min(chunk, m)], best[:min(chunk, m)])
    torch.cuda.synchronize()
    st0 = g.stats()
    g.profile(True)
    g.profile_read(reset=True)
    sev = []
    for a0 in range(0, m, chunk):
        n = min(chunk, m - a0)
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        e[0].record(stream)
        g.score(P[a0:a0 + n], N[a0:a0 + n], lab[:n], best[:n])
        e[1].record(stream)
        sev.append(e)
    torch.cuda.synchronize()
    clocks.mark(False)
    clk = clocks.stop()
    prof = g.profile_read(reset=True)
    st1 = g.stats()
    sms = [a.elapsed_time(b) for a, b in sev]
    tests = st1["tests"] - st0["tests"]
    scored = st1["points_scored"] - st0["points_scored"]
    score_ms = sum(sms)
    peak, peak_kind = _peaks()
    bpt = score_bytes_per_test(W)
    kms = prof["k_score"][1]
    alg = bpt * tests + SCORE_BYTES_PER_POINT * scored
    returns = sum(len(f[0]) for f in frames)
    out = {
        "metric": "large map: point x orientation tests/s (every surface point after 3,000 frames)",
        "value": tests / (score_ms / 1e3), "unit": "tests/s", "n_gpus": 1,
        "steps": len(sms), "warmup": max(args.warmup, 3), "ms_per_step": score_ms / len(sms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
        "data": "synthetic",
        "config": {"workload": W.name, "frames": len(frames), "voxel_m": W.params["v"],
                   "K": W.params["K"], "G": len(W.dirs), "points": m, "chunk": chunk,
                   "l2": "occupancy views far larger than L2; no flush"},
        "integration": {"returns_per_s": returns / (sum(ims) / 1e3),
                        "frame_ms": {"p50": float(np.percentile(ims, 50)),
                                     "p99": float(np.percentile(ims, 99))}},
        # the early-exit-free count (2 bits per kernel voxel) overstates what the
        # search reads at K = 256 and a 1.5 m corridor: most tests end early,
        # so its rate exceeds the HBM peak and is reported beside, not as, frac
        "roofline": {"kernel": "k_score", "bound": "latency", "unit": "GB/s", "peak": peak,
                     "peak_kind": peak_kind, "traffic": None, "achieved": None, "frac": None,
                     "early_exit_free_bytes_per_test": bpt,
                     "early_exit_free_rate": alg / (kms * 1e-3) / 1e9},
        "tests_per_point": tests / max(scored, 1),
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
        "cpu_baseline": None if args.no_cpu_baseline else large_cpu_baseline(W, frames),
    }
    g.close()
    return out


# the neighbourhood trigger of Sec. 3.5 (ii): 256 changed voxels drawn per
# frame (the paper's), all of them, or the brick rule
POINTS_TRIGGERS = {"sampled": {}, "all": dict(trig_sample=0), "brick": dict(trig_exact=0)}


def run_points(args, local):
    """The stateful point layer (Sec. 3.4, 3.5) over the pine stream: each
    step integrates one frame and updates the point set -- new points,
    viewpoints, triggers, up to `budget` evaluations with PCA normals and the
    observation-side filter."""
    import torch
    from paper_2608_06412_gb300 import af, workload
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2608_06412_gb300 import synth
    W = workload.pine_stream()
    nfr = args.warmup + args.steps
    frames = _frames(W, 0, nfr)
    tool, dirs = W.af_tool(), W.dirs
    if args.ring:
        tool.cos_theta_max = synth.COS_70
        dirs = synth.yaw_ring(180)
    c2f = dict(c2f_stride=10, c2f_half=12, c2f_radius=0.3) if args.c2f else {}
    trig = POINTS_TRIGGERS[args.points_trigger]
    caps = dict(workload.BENCH_CAPS, clamp_signed=int(args.clamp_signed))

    def layer():
        m = af.Map(W.af_config(**caps))
        m.set_tool(tool, dirs)
        m.points_enable(af.PointsConfig(trig_tsdf=2 * W.params["v"], budget=args.points_budget,
                                        capacity=1 << 21, **c2f, **trig))
        return m
    g = layer()
    d_xyz = [torch.from_numpy(f[0].pts).to(dev) for f in frames]
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for k in range(args.warmup):
        g.points_frame(d_xyz[k], frames[k][0].pose)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    evals = 0
    clocks = Clocks(local)
    clocks.start()
    clocks.mark(True)
    for i, k in enumerate(range(args.warmup, nfr)):
        flush.zero_()
        ev[i][0].record(stream)
        g.points_frame(d_xyz[k], frames[k][0].pose)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    # evaluations per frame, counted in a second pass over the same frames
    g2 = layer()
    per = []
    for k in range(nfr):
        g2.points_frame(d_xyz[k], frames[k][0].pose)
        if k >= args.warmup:
            per.append(g2.points_stats()[1])
    evals = sum(per)
    n, _ = g.points_stats()
    e = g.points_export()
    total = sum(ms)
    out = {
        "metric": "stateful point-layer evaluations/s (integration + point set + triggers + budgeted evaluation)",
        "value": evals / (total / 1e3), "unit": "evaluations/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
        "data": "synthetic",
        "config": {"workload": W.name, "budget": args.points_budget,
                   "trigger": args.points_trigger,
                   "directions": "yaw ring, 70 deg cone" if args.ring else "Fibonacci sphere",
                   "G": len(dirs), "search": "coarse-to-fine" if args.c2f else "full",
                   "clamp": "[-tau, tau]" if args.clamp_signed else "[0, tau]",
                   "l2": "flushed between steps (256 MiB write)"},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                       "max": float(max(ms))},
        "evaluations_per_frame": {"mean": float(np.mean(per)), "max": int(max(per))},
        "points": n,
        "labels": {"unscored": int((e["label"] == 0).sum()),
                   "accessible": int((e["label"] == 1).sum()),
                   "blocked": int((e["label"] == 2).sum()),
                   "queued": int(e["queued"].sum())},
        "with_direction": int((e["best"] >= 0).sum()),
        "clocks": clk,
        # the oracle's layer on the default set-up (a variant line reports none)
        "cpu_baseline": None if (args.no_cpu_baseline or args.ring or args.clamp_signed)
        else points_cpu_baseline(W, frames),
    }
    g.close()
    g2.close()
    return out


def run_noalloc(args, local):
    """The allocation-free integration (af_integrate_scan_noalloc) over the
    pine stream into one caller-owned dense box of the whole map box (51 x 51
    x 86 bricks: 115M voxels, 1.0 GB of words and flags), timed per frame
    beside the map path's integration (af_integrate_scan) of the same frames;
    the box's contents are checked against the map path's export at the end."""
    import torch
    from paper_2608_06412_gb300 import af, workload
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = workload.pine_stream()
    nfr = args.warmup + args.steps
    frames = _frames(W, 0, nfr)
    cfg = W.af_config(**workload.BENCH_CAPS, clamp_signed=int(args.clamp_signed))
    box_min = np.array(W.dom_min) * 8
    box_dim = np.array(W.dom_bricks) * 8
    count = int(np.prod(box_dim))
    vox = torch.zeros(count, dtype=torch.int64, device=dev)
    flags = torch.zeros(count, dtype=torch.uint8, device=dev)
    d_xyz = [torch.from_numpy(f[0].pts).to(dev) for f in frames]
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    g = af.Map(cfg)

    def timed(call):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for i, k in enumerate(range(args.warmup, nfr)):
            flush.zero_()
            ev[i][0].record(stream)
            call(k)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for k in range(args.warmup):
        af.integrate_scan_noalloc(cfg, d_xyz[k], frames[k][0].pose, box_min, box_dim, vox, flags)
        g.integrate_scan(d_xyz[k], frames[k][0].pose)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    clocks.mark(True)
    ms = timed(lambda k: af.integrate_scan_noalloc(cfg, d_xyz[k], frames[k][0].pose, box_min,
                                                   box_dim, vox, flags))
    ms_map = timed(lambda k: g.integrate_scan(d_xyz[k], frames[k][0].pose))
    clocks.mark(False)
    clk = clocks.stop()
    # the box against the map path's voxels (both integrated every frame)
    got = vox.cpu().numpy()
    fl = flags.cpu().numpy()
    ref = af.export_voxels(g.export_blocks())
    rel = ref["ijk"] - box_min
    at = (rel[:, 2] * box_dim[1] + rel[:, 1]) * box_dim[0] + rel[:, 0]
    want = (ref["S"].astype(np.int64) << 20) | ref["w"].astype(np.int64)
    want_fl = ref["cleared"] | (ref["occ"] << 1) | (ref["known"] << 2)
    agree = bool((got[at] == want).all() and (fl[at] == want_fl).all() and
                 np.count_nonzero(got) == np.count_nonzero(want))
    returns = sum(int(d_xyz[k].shape[0]) for k in range(args.warmup, nfr))
    total = sum(ms)
    g.close()
    return {
        "metric": "allocation-free integration returns/s (af_integrate_scan_noalloc, dense box)",
        "value": returns / (total / 1e3), "unit": "returns/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
        "data": "synthetic",
        "config": {"workload": W.name, "returns_per_frame": W.params["n_returns"],
                   "box_voxels": count, "box_bytes": count * 9,
                   "clamp": "[-tau, tau]" if args.clamp_signed else "[0, tau]",
                   "l2": "flushed between steps (256 MiB write)"},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                       "max": float(max(ms))},
        "map_path": {"returns_per_s": returns / (sum(ms_map) / 1e3),
                     "latency_ms": {"p50": float(np.percentile(ms_map, 50)),
                                    "p99": float(np.percentile(ms_map, 99))}},
        "box_equals_map_path": agree,
        "clocks": clk,
        "cpu_baseline": None,
    }


def run_soft_large(args, local):
    """The differentiable step on the large map (3,000 frames at 1 cm, K = 256
    of G = 512, 1.5 m corridor): 100k surface points drawn from the stream's
    points, plain scoring, the start direction of each accessible point, its
    soft clearance and 20 ascent steps. The box's dense SDF view would need
    over 2^31 cells, so the brick-sparse view is built (af_soft_set_view 0
    chooses it); its build is timed once, the step after it."""
    from paper_2608_06412_gb300 import workload
    W = workload.large_map()
    frames = workload.large_frames(W, range(W.params["frames"]))   # spawned workers first
    import torch
    from paper_2608_06412_gb300 import af
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m = args.soft_points
    g = af.Map(W.af_config(**dict(LARGE_CAPS, max_points=max(m, LARGE_CAPS["max_points"]))))
    g.set_tool(W.af_tool(), W.dirs)
    for f in frames:
        g.integrate_scan(torch.from_numpy(f[0]).to(dev), f[1])
    torch.cuda.synchronize()
    P = np.concatenate([f[3] for f in frames])
    N = np.concatenate([f[4] for f in frames])
    v = np.float64(np.float32(W.params["v"]))
    ijk = np.floor(P.astype(np.float64) / v).astype(np.int64) + (1 << 20)
    key = ijk[:, 0] | (ijk[:, 1] << 21) | (ijk[:, 2] << 42)
    _, first = np.unique(key, return_index=True)
    sel = np.sort(np.random.default_rng(9).choice(np.sort(first), m, replace=False))
    Pd = torch.from_numpy(np.ascontiguousarray(P[sel])).to(dev)
    Nd = torch.from_numpy(np.ascontiguousarray(N[sel])).to(dev)
    lab = torch.empty(m, dtype=torch.uint8, device=dev)
    best = torch.empty(m, dtype=torch.int16, device=dev)
    u0 = torch.empty((m, 3), dtype=torch.float32, device=dev)
    z = torch.zeros(m, dtype=torch.float32, device=dev)
    al, be, hh, c0, c, cmin = (torch.empty(m, dtype=torch.float32, device=dev) for _ in range(6))
    stream = torch.cuda.current_stream()

    def step():
        g.score(Pd, Nd, lab, best)
        g.soft_start(lab, best, out=u0)
        g.soft_clearance_raw(Pd, u0, z, z, z, 1, out=c0)
        al.zero_()
        be.zero_()
        hh.zero_()
        g.soft_refine(Pd, u0, al, be, hh, 1, steps=SOFT_STEPS, out=(c, cmin), **SOFT_LR)

    g.profile(True)
    g.profile_read(reset=True)
    step()                                   # builds the sparse view
    torch.cuda.synchronize()
    build_ms = g.profile_read(reset=True).get("k_views", (0, 0.0))[1]
    warm, steps = max(args.warmup, 3), max(1, min(args.steps, 20))
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    g.profile_read(reset=True)
    n_acc = int((lab == af.ACCESSIBLE).sum().item())
    clocks = Clocks(local)
    clocks.start()
    clocks.mark(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    prof = g.profile_read(reset=True)
    assert g.sync_status() == 0
    evals = n_acc * (SOFT_STEPS + 2)
    out = {
        "metric": "large map: " + SOFT_METRIC, "value": evals / (sum(ms) / steps / 1e3),
        "unit": SOFT_UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": sum(ms) / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"soft_refine_{W.name}_{m}_points", "points": m,
                   "K": W.params["K"], "G": len(W.dirs), "refine_steps": SOFT_STEPS, **SOFT_LR,
                   "tau_s": af.TAU_S, "sdf_view": "brick-sparse (automatic: the box's dense "
                   "view exceeds 2^31 cells)", "l2": "views far larger than L2; no flush"},
        "accessible_points": n_acc,
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "kernel_ms": {k: round(v[1] / steps, 4) for k, v in prof.items() if v[0]},
        "sparse_view_build_ms": build_ms,
        "bricks": g.block_count(),
        "gpu_launches": int(sum(v[0] for v in prof.values()) / steps),
        "clocks": clk,
    }
    g.close()
    return out


LARGE_SCENE_CAPS = dict(hash_capacity=1 << 21, pool_blocks=1 << 20, max_returns=1 << 15,
                        max_points=1 << 15)


def run_large_batched(args, local):
    """The large map's workload in the batched form: its eight pine orbits
    (375 frames each, v = 1 cm, tau = 4 cm, K = 256 of G = 512, 1.5 m
    corridor) as eight scenes, each a 14 x 14 m map box around its pine (the
    returns whose cubes leave it are dropped, as at any box edge). A tick
    integrates one frame of every scene and scores that frame's surface
    points; the same ticks then run through the per-scene path
    (af_integrate_scan + af_score per scene). Labels and best directions of
    every tick are compared between the two paths."""
    import hashlib
    from paper_2608_06412_gb300 import synth, workload
    W = workload.large_map()
    p = W.params
    frames = workload.large_frames(W, range(p["frames"]))   # spawned workers, before CUDA
    import torch
    from paper_2608_06412_gb300 import af
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    npine, per = p["pines"], p["frames_per_pine"]
    centres = synth.pine_positions(p["seed"], npine, p["ground_half"])
    scenes = []
    for c in centres:
        lo = np.array([c[0] - 7.0, c[1] - 7.0, -0.3])
        hi = np.array([c[0] + 7.0, c[1] + 7.0, 12.6])
        dmin, db = synth.domain_bricks(lo, hi, p["v"], margin=0.0)
        scenes.append(workload.Workload(f"{W.name}_pine", p, W.scene, dmin, db, W.dirs))
    ticks = min(per, args.steps) if args.steps < per else per
    warm = 3
    dx = [[torch.from_numpy(frames[i * per + t][0]).to(dev) for t in range(ticks)]
          for i in range(npine)]
    dp = [[torch.from_numpy(frames[i * per + t][3]).to(dev) for t in range(ticks)]
          for i in range(npine)]
    dn = [[torch.from_numpy(frames[i * per + t][4]).to(dev) for t in range(ticks)]
          for i in range(npine)]
    mmax = max(len(frames[k][3]) for k in range(len(frames)))
    outs = [(torch.empty(mmax, dtype=torch.uint8, device=dev),
             torch.empty(mmax, dtype=torch.int16, device=dev)) for _ in range(npine)]
    stream = torch.cuda.current_stream()

    def run(batched: bool):
        maps = [af.Map(S.af_config(**LARGE_SCENE_CAPS)) for S in scenes]
        for m in maps:
            m.set_tool(W.af_tool(), W.dirs)
        batch = af.Batch(maps) if batched else None
        h = hashlib.sha256()
        ms, t0 = [], None
        for t in range(ticks):
            if t == warm:
                torch.cuda.synchronize()
                t0 = sum(m.stats()["tests"] for m in maps)
            items = []
            for i in range(npine):
                n = len(dp[i][t])
                items.append((dx[i][t], frames[i * per + t][1], dp[i][t], dn[i][t],
                              outs[i][0][:n], outs[i][1][:n]))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if batched:
                batch.tick(items)
            else:
                for m, (xyz, pose, pp, nn, lab, best) in zip(maps, items):
                    m.integrate_scan(xyz, pose)
                    m.score(pp, nn, lab, best)
            b.record(stream)
            torch.cuda.synchronize()
            if t >= warm:
                ms.append(a.elapsed_time(b))
            for it in items:
                h.update(it[4].cpu().numpy().tobytes())
                h.update(it[5].cpu().numpy().tobytes())
        tests = sum(m.stats()["tests"] for m in maps) - t0
        status = [m.sync_status() for m in maps]
        if any(status):
            raise RuntimeError(f"large map scenes: device status {status}")
        tuning = batch.tuning() if batched else None
        if batch:
            batch.close()
        blocks = [m.block_count() for m in maps]
        for m in maps:
            m.close()
        return ms, tests, h.hexdigest(), tuning, blocks

    clocks = Clocks(local)
    clocks.start()
    clocks.mark(True)
    msb, testsb, digb, tuning, blocks = run(True)
    msp, testsp, digp, _, _ = run(False)
    clocks.mark(False)
    clk = clocks.stop()
    steps = len(msb)
    returns = sum(len(frames[i * per + t][0]) for i in range(npine) for t in range(warm, ticks))
    return {
        "metric": "large map, batched: point x orientation tests/s (8 pine scenes per tick)",
        "value": testsb / (sum(msb) / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warm, "ms_per_step": sum(msb) / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
        "config": {"workload": f"{W.name}_8_scenes", "scenes": npine, "ticks": ticks,
                   "scene_box_m": "14 x 14 x 12.9 around each pine", "voxel_m": p["v"],
                   "K": p["K"], "G": len(W.dirs), "per_tick": "one frame of every scene, "
                   "integrated, then its surface points scored",
                   "l2": "scene views far larger than L2; no flush"},
        "latency_ms": {"p50": float(np.percentile(msb, 50)), "p99": float(np.percentile(msb, 99))},
        "returns_per_s": returns / (sum(msb) / 1e3),
        "tuning": tuning,
        "bricks_per_scene": blocks,
        "per_scene_path": {"value": testsp / (sum(msp) / 1e3), "ms_per_step": sum(msp) / steps,
                           "latency_ms": {"p50": float(np.percentile(msp, 50)),
                                          "p99": float(np.percentile(msp, 99))}},
        "speedup_vs_per_scene": (sum(msp) / steps) / (sum(msb) / steps),
        "label_agreement": 1.0 if digb == digp else 0.0,
        "labels_digest": digb[:16],
        "tests_equal": testsb == testsp,
        "gpu_launches": None,
        "clocks": clk,
    }


def main():
    args = _args()
    ws, rank, local = _dist()
    if args.large and args.batched:
        print(json.dumps(run_large_batched(args, local)), flush=True)
        return
    if args.large and args.soft:
        print(json.dumps(run_soft_large(args, local)), flush=True)
        return
    if args.batched:
        out = run_batched(args, local)
        print(json.dumps(out), flush=True)
        return
    if args.soft:
        print(json.dumps(run_soft(args, local)), flush=True)
        return
    if args.points:
        print(json.dumps(run_points(args, local)), flush=True)
        return
    if args.large:
        print(json.dumps(run_large(args, local)), flush=True)
        return
    if args.noalloc:
        print(json.dumps(run_noalloc(args, local)), flush=True)
        return
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    from paper_2608_06412_gb300 import workload
    W = workload.pine_stream()
    if args.impl == "reference":
        out = run_reference(args, W, ws, rank)
    else:
        out = run_ours(args, W, ws, rank, local)
        frames = out.pop("_frames")
        variant = args.projective or args.ring or args.clamp_signed
        if rank == 0 and ws == 1 and not args.no_cpu_baseline and not variant:
            out["cpu_baseline"] = cpu_baseline(W, frames)
        if rank != 0:
            out = None
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
