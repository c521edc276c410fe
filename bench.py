#!/usr/bin/env python
"""Throughput of the per-step metadynamics bias path on one GB300.

Metric: atom-steps/s of one whole step (cell-list neighbour build, per-atom
coordination number and locally averaged Q6, their FP64 means, the
well-tempered Gaussian-hill bias from a 200 x 200 FP64 grid plus 20,000 live
hills, the adjoint and the bias forces; a hill deposited every 500 frames) on
the 1,000,000-atom half-wurtzite / half-liquid workload, frames resident in
HBM.  One JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl metad|reference]

--impl reference times the FP64 CPU oracle (the slow, plain restatement the
tests compare against) on the host cores instead.  Under torchrun each rank
runs an independent replica (weak scaling; the path has no exchange step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "atom-steps/s CV+bias+force at 1M atoms (%HBM roofline); served p50/p99 vs plain"
UNIT = "atom-steps/s"
WORKLOAD = ("1M-atom half-wurtzite/half-RSA-liquid periodic box (228.6 A), 2 CVs (unlike-pair coordination "
            "number + locally averaged Q6, rc 3.5 A), FP64 bias = 200x200 bicubic-Hermite grid (20,000 folded "
            "hills) + 20,000 live well-tempered hills, one deposit per 500 frames")

# Algorithmic work, counted once per unordered neighbour pair or per atom
# (the kernels' own redundant work is not counted): per unordered pair Y_6m
# ~110, accumulate ~50, CN ~40 flop in the forward pass and ~300 for the
# adjoint gradient of w Y.G in the force pass; per atom ~500 for the neighbour
# search and ~800 for the Q6 averaging and adjoint-seed gathers (split
# evenly between those two passes).  Totals about 5e3 FP32 flop per atom.
FLOP_PER_PAIR = {"cv_fwd": 200.0, "force_pairs": 300.0}
FLOP_PER_ATOM = {"cv_fwd": 500.0, "cv_avg": 400.0, "adjoint": 400.0}
# Algorithmic HBM bytes per atom-step with the neighbour list persisted
# between steps: positions in (16 B), forces out (12 B) and the list read
# and written (~2 x 60 B); about 160 B.
STEP_BYTES_PER_ATOM = 160.0


def stage_flops(stage: str, n_atoms: int, pairs: float) -> float:
    """Algorithmic FP32 flops of one launch of a stage at this size."""
    return FLOP_PER_PAIR.get(stage, 0.0) * pairs + FLOP_PER_ATOM.get(stage, 0.0) * n_atoms


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="metad", choices=["metad", "reference"])
    ap.add_argument("--frames", type=int, default=16, help="distinct resident frames, cycled")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--atoms", type=int, default=1_000_000, help="workload size (1M is the reported config)")
    ap.add_argument("--skin", type=float, default=1.0,
                    help="Verlet skin in A (1.0 is the reported config; 0 rebuilds the rows every step)")
    ap.add_argument("--hills", type=int, default=None, help="live hills (default: the workload's 20,000)")
    ap.add_argument("--hills-folded", type=int, default=None, help="hills folded into the grid (default 20,000)")
    ap.add_argument("--max-neighbors", type=int, default=64, help="per-atom neighbour-row capacity")
    ap.add_argument("--drift-step", type=float, default=0.01,
                    help="random-walk step (A per coordinate and frame) of the timed drifting trajectory")
    ap.add_argument("--no-skin0", action="store_true", help="skip the rebuild-every-step (skin 0) measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the served offered-rate sweep")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-system batched comparison")
    ap.add_argument("--no-served", action="store_true", help="skip the served (continuous batching) trace")
    ap.add_argument("--no-small", action="store_true", help="skip the torsion / nearest-distance walker forms")
    ap.add_argument("--no-npt", action="store_true", help="skip the NPT (lattice CVs, box gradient) form")
    ap.add_argument("--batched-steps", type=int, default=10)
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Sources that make up the per-atom kernels; a profile summary records their
# SHA-1 when its counters were taken.
KERNEL_SOURCES = ("paper_2510_06873_gb300/csrc/k_cv.cu", "paper_2510_06873_gb300/csrc/metad_impl.cuh")
# The kernel each timed stage launches (its ncu summary is profiles/<kernel>.md).
STAGE_KERNEL = {"cv_fwd": "k_cv_fwd", "cv_avg": "k_cv_avg", "adjoint": "k_adjoint", "force_pairs": "k_force_pairs",
                "force_gather": "k_force_gather", "neighbors": "k_verlet", "gather": "k_gather_check", "bias": "k_bias"}


def kernel_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic(kernel: str, n_atoms: int):
    """DRAM bytes (read + write) per launch of `kernel` at n_atoms, from the
    ncu capture summarised in profiles/<kernel>.md (bytes per atom of the
    captured case times n_atoms); None when the summary is missing or the
    kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}.md")
    if not os.path.exists(path):
        return None
    per_atom, sha = None, None
    for line in open(path):
        if line.startswith("traffic_bytes_per_atom ="):
            per_atom = float(line.split("=", 1)[1])
        elif line.startswith("sources_sha1 ="):
            sha = line.split("=", 1)[1].strip()
    if per_atom is None or sha != kernel_sources_sha1():
        return None
    return per_atom * n_atoms


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    replica's); x itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size: int, units_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job atom-steps/s: every replica's units over the slowest time."""
    return world_size * units_per_rank * steps / seconds


def device_drift_frames(system, count, step_sigma, sigma, dev, seed):
    """Frames 0 .. count-1 of synth.drift_trajectory's drifting trajectory
    (per-atom random walk of step_sigma per coordinate and frame plus thermal
    N(0, sigma^2), wrapped into the box in FP64 and rounded to float32),
    generated on the device from torch's seeded generator so that a
    1M-atom trajectory of a few hundred frames takes milliseconds, not the
    minutes of the host generator: the same distribution, other draws.
    Returns float32 [count, N, 4]."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    base = torch.from_numpy(system.base).to(dev)
    b64 = base[:, :3].double()
    L = torch.tensor(np.asarray(system.box, dtype=np.float64), device=dev)
    out = torch.empty((count, system.n, 4), dtype=torch.float32, device=dev)
    walk = torch.zeros_like(b64)
    for f in range(count):
        if f > 0:
            walk += step_sigma * torch.randn(walk.shape, generator=g, device=dev, dtype=torch.float64)
        x = b64 + walk + sigma * torch.randn(walk.shape, generator=g, device=dev, dtype=torch.float64)
        w = x - L * torch.floor(x / L)
        w32 = w.float()
        out[f, :, :3] = torch.where(w32.double() >= L, torch.zeros_like(w32), w32)
        out[f, :, 3] = base[:, 3]
    return out


def kbdt(mp):
    return mp.kB * mp.temperature * (mp.biasfactor - 1.0)


def make_system(n):
    if n == 1_000_000:
        return synth.config3_system()
    return synth.wurtzite_system(n, cfg=3)


# ---------------------------------------------------------------- CPU legs
def oracle_sample(n_atoms, frames, nthreads=0):
    """The FP64 oracle on `frames` frames of the workload (hills and grid set up
    by the oracle itself, not timed).  Returns (atom-steps/s, cores, seconds,
    setup) with setup = (frames, oracle results, hill centres, heights of
    the folded and of the live hills, grid range) for the error block."""
    import oracle
    system = make_system(n_atoms)
    mp = synth.method_params(3)
    cfgp = synth.CONFIG_PARAMS[3]
    p = oracle.params_from(mp, system.box)
    s_ref, _, _ = oracle.cv(system.base, p, nthreads)
    K1, K2 = cfgp["hills_folded"], cfgp["hills"]
    cen = synth.hill_centres(3, system.sys, s_ref, mp.sigma, K1 + K2)
    sig = np.asarray(mp.sigma)
    w1 = oracle.deposit_sequence(cen[:K1], mp.sigma, mp.w0, kbdt(mp))
    G = oracle.HillGrid(cfgp["grid_n"], s_ref - 16 * sig, s_ref + 16 * sig)
    G.fold(cen[:K1], w1, mp.sigma, nthreads)
    w2 = oracle.deposit_sequence(cen[K1:], mp.sigma, mp.w0, kbdt(mp), grid=G)
    fr = [synth.perturbed_frame(system, f) for f in range(frames)]
    out = []
    t0 = time.perf_counter()
    for f in fr:
        out.append(oracle.step(f, p, cen[K1:], w2, mp.sigma, grid=G, nthreads=nthreads))
    dt = time.perf_counter() - t0
    cores = nthreads if nthreads > 0 else oracle.max_threads()
    setup = (fr, out, cen, w1, w2, (s_ref - 16 * sig, s_ref + 16 * sig))
    return system.n * frames / dt, cores, dt, setup


def result_errors(metad, dev, stream, system, setup, max_neighbors):
    """Error of every result of the CUDA path against the FP64 oracle on the
    oracle's frames and hill set: a fresh context with the oracle's hills
    (folded into the grid, then live), one step per frame.  CVs and V
    relative; dV/ds_d relative to max(|dV/ds_d|, w0 / sigma_d) (the parity
    floor); forces norm-wise (||dF|| / ||F||) and per atom
    (max_i |dF_i| / max_i |F_i|).  The worst over the frames."""
    import torch
    mp = synth.method_params(3)
    cfgp = synth.CONFIG_PARAMS[3]
    frames, refs, cen, w1, w2, (lo, hi) = setup
    K1 = cfgp["hills_folded"]
    params = metad.params_for(system.n, system.box, n_cv=2, sigma=mp.sigma, grid=(cfgp["grid_n"], lo, hi),
                              hill_capacity=len(w2) + 64, stream=stream.cuda_stream, max_neighbors=max_neighbors)
    ctx = metad.Metad(params)
    ctx.load_hills(cen[:K1], w1)
    ctx.fold_hills()
    ctx.load_hills(cen[K1:], w2)
    F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    err = {"s1": 0.0, "s2": 0.0, "V": 0.0, "dVds1": 0.0, "dVds2": 0.0, "F_normwise": 0.0, "F_per_atom": 0.0}
    for fr, ref in zip(frames, refs):
        ctx.step(torch.from_numpy(fr).to(dev), F)
        cv, V, dV = ctx.read_results()
        Fg = F.cpu().numpy().astype(np.float64)
        dF = Fg - ref["F"]
        e = {"s1": abs(cv[0] - ref["s"][0]) / abs(ref["s"][0]), "s2": abs(cv[1] - ref["s"][1]) / abs(ref["s"][1]),
             "V": abs(V - ref["V"]) / max(abs(ref["V"]), mp.w0),
             "dVds1": abs(dV[0] - ref["dV"][0]) / max(abs(ref["dV"][0]), mp.w0 / mp.sigma[0]),
             "dVds2": abs(dV[1] - ref["dV"][1]) / max(abs(ref["dV"][1]), mp.w0 / mp.sigma[1]),
             "F_normwise": float(np.linalg.norm(dF) / np.linalg.norm(ref["F"])),
             "F_per_atom": float(np.max(np.linalg.norm(dF, axis=1)) / np.max(np.linalg.norm(ref["F"], axis=1)))}
        err = {k: max(err[k], float(e[k])) for k in err}
    ctx.close()
    err["frames"] = len(frames)
    err["tolerance"] = 1e-5
    err["note"] = ("CUDA path (FP32 pairs, FP64 reductions, hills and grid) against the FP64 oracle on the "
                   "same frames and hills; dV/ds relative to max(|dV/ds|, w0/sigma)")
    return err


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    # each step: the oracle on one frame of a 100,000-atom sample built the
    # same way (atom-steps/s of the oracle is flat in N), so K + W steps end
    # within a few minutes on the host cores
    n_sample = 100_000 if (args.steps + args.warmup) <= 300 else 20_000
    system = make_system(n_sample)
    mp = synth.method_params(3)
    cfgp = synth.CONFIG_PARAMS[3]
    p = oracle.params_from(mp, system.box)
    s_ref, _, _ = oracle.cv(system.base, p)
    K1, K2 = cfgp["hills_folded"], cfgp["hills"]
    cen = synth.hill_centres(3, system.sys, s_ref, mp.sigma, K1 + K2)
    sig = np.asarray(mp.sigma)
    w1 = oracle.deposit_sequence(cen[:K1], mp.sigma, mp.w0, kbdt(mp))
    G = oracle.HillGrid(cfgp["grid_n"], s_ref - 16 * sig, s_ref + 16 * sig)
    G.fold(cen[:K1], w1, mp.sigma)
    w2 = oracle.deposit_sequence(cen[K1:], mp.sigma, mp.w0, kbdt(mp), grid=G)
    nfr = 4
    frames = [synth.perturbed_frame(system, f) for f in range(nfr)]
    for k in range(args.warmup):
        oracle.step(frames[k % nfr], p, cen[K1:], w2, mp.sigma, grid=G)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.step(frames[k % nfr], p, cen[K1:], w2, mp.sigma, grid=G)
    dt = time.perf_counter() - t0
    value = system.n * args.steps / dt
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_atoms_sampled": system.n, "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one frame of a {system.n}-atom system built like the 1M workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU leg
def run_metad(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    # a non-default stream shared by torch's copies and the library's kernels
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    from paper_2510_06873_gb300 import build, metad
    if rank == 0 or not os.path.exists(metad.LIB_PATH):
        build.build()
    if ws > 1:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    system = make_system(args.atoms)
    mp = synth.method_params(3)
    cfgp = synth.CONFIG_PARAMS[3]
    n = system.n
    # ---- context, hills and grid, all made by the CUDA path
    base = torch.from_numpy(system.base).to(dev)
    probe = metad.Metad(metad.params_for(n, system.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream))
    probe.build_neighbors(base)
    s_ref = probe.cv_forward()
    probe_launches = probe.launch_count
    probe.close()
    sig = np.asarray(mp.sigma)
    lo, hi = s_ref - 16 * sig, s_ref + 16 * sig
    params = metad.params_for(n, system.box, n_cv=2, sigma=mp.sigma, grid=(cfgp["grid_n"], lo, hi),
                              hill_capacity=cfgp["hills"] + 1024, stream=stream.cuda_stream,
                              max_neighbors=args.max_neighbors, skin=args.skin)
    ctx = metad.Metad(params)
    K1 = cfgp["hills_folded"] if args.hills_folded is None else args.hills_folded
    K2 = cfgp["hills"] if args.hills is None else args.hills
    cen = synth.hill_centres(3, system.sys, s_ref, mp.sigma, K1 + K2)
    ctx.deposit_hills(cen[:K1], want_heights=False)
    ctx.fold_hills()
    ctx.deposit_hills(cen[K1:], want_heights=False)
    ctx.sync()
    # ---- resident frames (16 x 16 MB; each step reads a frame not in L2)
    nfr = max(1, args.frames)
    frames_h = [synth.perturbed_frame(system, f) for f in range(nfr)]
    frames = torch.from_numpy(np.stack(frames_h)).to(dev)
    F = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    every = cfgp["deposit_every"]
    frame_no = 0

    def one_step():
        nonlocal frame_no
        ctx.step(frames[frame_no % nfr], F, deposit=((frame_no + 1) % every == 0))
        frame_no += 1

    for _ in range(max(3, args.warmup)):
        one_step()
    ctx.sync()
    entries, max_nn = ctx.neighbor_stats()
    pairs = entries / 2
    # kernels of this library launched before the timed region (for ncu -s)
    print(f"setup_launches={probe_launches + ctx.launch_count}", file=sys.stderr, flush=True)

    def timed_region(c, step_fn, steps, profile=True):
        """CUDA events on the context stream around `steps` steps, clocks
        sampled during the region, launches and rebuilds, and with `profile`
        the per-stage events (which add their own records to the stream)."""
        clocks = ClockSampler(local)
        launches0, rebuilds0 = c.launch_count, c.rebuild_count
        if profile:
            c.profile_begin(16 * steps + 64)
        clocks.start()
        time.sleep(0.3)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step_fn()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t_ms = ev0.elapsed_time(ev1)
        if ws > 1:
            dist.barrier()
        clk_ = clocks.stop()
        st = c.profile_end() if profile else None
        return max_over_ranks(t_ms, dev), st, c.launch_count - launches0, clk_, c.rebuild_count - rebuilds0

    def stage_table(st, total_ms):
        return {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / max(total_ms, 1e-9)}
                for k, v in st.items() if v[1] > 0}

    # ---- static frames: independent thermal perturbations of one base
    # (their spread stays inside half the skin: no rebuild in the region)
    ms_s, stages_s, launches_s, clk_s, reb_s = timed_region(ctx, one_step, args.steps)
    static_line = {"ms_per_step": ms_s / args.steps, "value": job_throughput(ws, n, args.steps, ms_s / 1e3),
                   "rebuilds": reb_s, "gpu_launches": launches_s, "clocks": clk_s,
                   "stages": stage_table(stages_s, ms_s),
                   "frames": f"{nfr} resident frames base + N(0, 0.05^2), cycled"}
    # ---- drifting trajectory (the headline): a per-atom random walk of
    # args.drift_step A per coordinate and frame on top of the thermal noise,
    # so the Verlet rows are rebuilt inside the region at an MD-like rate
    # (the rebuild cost amortised into ms_per_step)
    drift_count = max(3, args.warmup) + 2 * args.steps
    drift = device_drift_frames(system, drift_count, args.drift_step, 0.05, dev, seed=20251006 + rank)
    drift_no = 0

    def drift_step():
        nonlocal drift_no, frame_no
        ctx.step(drift[drift_no], F, deposit=((frame_no + 1) % every == 0))
        drift_no += 1
        frame_no += 1

    for _ in range(max(3, args.warmup)):
        drift_step()
    # kernels of this library launched before the headline region (for ncu -s)
    print(f"headline_launches_before={probe_launches + ctx.launch_count}", file=sys.stderr, flush=True)
    # the headline: plain CUDA events around the steps, no per-stage events
    ms, _, launches, clk, reb_d = timed_region(ctx, drift_step, args.steps, profile=False)
    # the stage breakdown: the next stretch of the same trajectory with the
    # per-stage events on (their own records cost the step a little)
    ms_prof, stages, _, _, reb_p = timed_region(ctx, drift_step, args.steps)
    drift = None  # release the trajectory's device memory
    value = job_throughput(ws, n, args.steps, ms / 1e3)
    # ---- dominant kernel roofline from the live per-stage events, against
    # the FP32 peak measured on this GPU (multiply-add chains, CUDA events)
    fp32_peak = metad.metad_probe_fp32_peak(local)
    peaks_hbm = 6787.2
    try:
        peaks_hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        pass
    timed = {k: v for k, v in stages.items() if v[1] > 0 and k != "other"}
    dom = max(timed, key=lambda k: timed[k][0])
    dom_ms, dom_cnt = stages[dom]
    avg_s = dom_ms / dom_cnt / 1e3
    flops = stage_flops(dom, n, pairs)
    achieved = flops / avg_s / 1e12
    roof = {"kernel": STAGE_KERNEL.get(dom, dom), "bound": "alu", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": profiled_traffic(STAGE_KERNEL.get(dom, dom), n),
            "peak_source": "measured on this GPU: metad_probe_fp32_peak (fmaf chains, CUDA events)",
            "algorithmic": f"{flops / n:.0f} FP32 flop per atom x {n} atoms (search, per-pair and per-atom "
                           f"counts; {pairs / n:.2f} unordered pairs per atom)"}
    step_ms = ms / args.steps
    step_bytes = STEP_BYTES_PER_ATOM * n
    step_flops = sum(stage_flops(k, n, pairs) for k in ("cv_fwd", "cv_avg", "adjoint", "force_pairs"))
    # every per-atom kernel against both ceilings: algorithmic flops against
    # the measured FP32 peak, profiled DRAM bytes (ncu, per launch) against HBM
    per_kernel = {}
    for k in sorted(timed):
        t = stages[k][0] / stages[k][1] / 1e3
        tf = stage_flops(k, n, pairs) / t / 1e12
        dram = profiled_traffic(STAGE_KERNEL.get(k, k), n)
        per_kernel[k] = {"kernel": STAGE_KERNEL.get(k, k), "us": t * 1e6, "tflops": tf, "frac_fp32": tf / fp32_peak,
                         "dram_bytes": dram, "dram_gbs": dram / t / 1e9 if dram else None,
                         "frac_hbm_dram": dram / t / 1e9 / peaks_hbm if dram else None}
    dram_step = [per_kernel[k]["dram_bytes"] for k in per_kernel]
    # ---- the same steps replayed from captured CUDA graphs (no stage events)
    ctx.set_step_graph(True)
    for _ in range(nfr + 3):  # one capture per resident frame buffer, then replays
        one_step()
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        one_step()
    g1.record(stream)
    torch.cuda.synchronize(dev)
    ctx.set_step_graph(False)
    graph_ms = max_over_ranks(g0.elapsed_time(g1), dev) / args.steps
    graph_line = {"ms_per_step": graph_ms, "value": job_throughput(ws, n, 1, graph_ms / 1e3), "steps": args.steps,
                  "note": "metad_step replayed from captured CUDA graphs, no per-stage events"}
    stage_line = stage_table(stages, ms_prof)
    # ---- skin 0: the rows are rebuilt at every step (Verlet rows = exact
    # rows), the same hills and grid; the full-rebuild cost is its
    # "neighbors" stage
    skin0 = None
    if not args.no_skin0:
        p0 = metad.params_for(n, system.box, n_cv=2, sigma=mp.sigma, grid=(cfgp["grid_n"], lo, hi),
                              hill_capacity=cfgp["hills"] + 1024, stream=stream.cuda_stream,
                              max_neighbors=args.max_neighbors, skin=0.0)
        ctx0 = metad.Metad(p0)
        ctx0.deposit_hills(cen[:K1], want_heights=False)
        ctx0.fold_hills()
        ctx0.deposit_hills(cen[K1:], want_heights=False)
        k0 = [0]

        def step0():
            ctx0.step(frames[k0[0] % nfr], F)
            k0[0] += 1

        for _ in range(3):
            step0()
        steps0 = min(args.steps, 50)
        ms0, st0, launches0, clk0, reb0 = timed_region(ctx0, step0, steps0)
        ctx0.close()
        nb0 = st0.get("neighbors", (0.0, 0))
        skin0 = {"ms_per_step": ms0 / steps0, "value": job_throughput(ws, n, steps0, ms0 / 1e3), "steps": steps0,
                 "rebuilds": reb0, "gpu_launches": launches0, "clocks": clk0, "stages": stage_table(st0, ms0),
                 "ms_full_rebuild": nb0[0] / nb0[1] if nb0[1] else None,
                 "note": "skin 0: cell binning, counting sort and rows rebuilt at every step"}
    # ---- end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if args.e2e_steps > 0:
        pin_pos = [torch.from_numpy(f).pin_memory().numpy() for f in frames_h[: min(nfr, 4)]]
        pin_F = torch.zeros((n, 3), dtype=torch.float32).pin_memory().numpy()
        ctx.step_host(pin_pos[0], pin_F)
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            ctx.step_host(pin_pos[k % len(pin_pos)], pin_F, deposit=((frame_no + 1) % every == 0))
            frame_no += 1
        dt = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": job_throughput(ws, n, args.e2e_steps, dt), "unit": UNIT, "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": 12 * n + 24, "steps": args.e2e_steps,
               "call": "metad_step_host (pinned host positions in, host forces + CVs + bias out)"}
    ctx.sync()
    cpu = None
    errors = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, dt, setup = oracle_sample(n, 2)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"2 frames of the same {n}-atom workload (oracle hills/grid set up untimed), {dt:.1f} s"}
        errors = result_errors(metad, dev, stream, system, setup, args.max_neighbors)
    forms = {}
    if rank == 0 and ws == 1:
        if not args.no_batched:
            forms["batched"] = run_batched(args, dev, stream, metad)
        if not args.no_served:
            forms["served"] = run_served(args, dev, stream, metad)
        if not args.no_small:
            forms["small_cvs"] = run_small_cvs(args, dev, stream, metad)
        if not args.no_npt:
            forms["npt"] = run_npt(args, dev, stream, metad, n)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n_atoms": n, "unordered_pairs": int(pairs),
                           "max_neighbors_per_atom": max_nn, "live_hills_end": ctx.hill_count,
                           "precision": "FP32 pair arithmetic, FP64 CV reductions, hills and grid",
                           "frames": f"drifting trajectory: per-atom random walk N(0, {args.drift_step}^2) A per "
                                     f"coordinate and frame + thermal N(0, 0.05^2), {drift_count} frames resident, "
                                     f"skin {args.skin} A (rebuilds amortised)",
                           "frames_resident": drift_count, "skin": args.skin,
                           "parallelism": f"replica x{ws}" if ws > 1 else "single GPU",
                           "l2": f"inputs larger than L2: each step reads a new {16 * n / 1e6:.0f} MB frame "
                                 f"({16 * n * drift_count / 1e6:.0f} MB resident > 129 MB)"},
                "roofline": roof, "kernel_rooflines": per_kernel,
                "step_roofline": {
                    "algorithmic_bytes": step_bytes, "bytes_per_atom": STEP_BYTES_PER_ATOM,
                    "achieved_gbs": step_bytes / (step_ms / 1e3) / 1e9, "peak_gbs": peaks_hbm,
                    "frac_hbm": step_bytes / (step_ms / 1e3) / 1e9 / peaks_hbm,
                    "algorithmic_flops": step_flops, "achieved_tflops": step_flops / (step_ms / 1e3) / 1e12,
                    "peak_tflops": fp32_peak, "frac_fp32": step_flops / (step_ms / 1e3) / 1e12 / fp32_peak,
                    "measured_dram_bytes": sum(dram_step) if dram_step and all(dram_step) else None,
                    "note": "algorithmic bytes = 160 B per atom-step (positions in, forces out, the "
                            "persisted neighbour list); measured DRAM bytes = the profiled per-kernel ncu "
                            "counters summed over the step's kernels (null unless every kernel has one)"},
                "rebuilds": reb_d, "stages": stage_line,
                "stages_region": {"ms_per_step": ms_prof / args.steps, "rebuilds": reb_p,
                                  "note": "the next stretch of the trajectory, per-stage events on"},
                "static_frames": static_line, "skin0": skin0,
                "graph_replay": graph_line, "gpu_launches": launches, "clocks": clk, "e2e": e2e,
                "cpu_baseline": cpu, "errors_vs_oracle": errors,
                **forms}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batched and served forms
def _seeded_hills(metad, system, mp, cfg, count, stream, dev, params):
    """Hill centres around the CUDA path's own CVs of the base frame and their
    well-tempered heights, deposited by the CUDA path (host copies back)."""
    import torch
    ctx = metad.Metad(params)
    ctx.build_neighbors(torch.from_numpy(system.base).to(dev))
    s_ref = ctx.cv_forward()
    cen = synth.hill_centres(cfg, system.sys, s_ref, mp.sigma, count)
    w = ctx.deposit_hills(cen)
    return ctx, cen, w


def run_batched(args, dev, stream, metad):
    """64 systems (1k-200k atoms, 100-10,000 hills): one batched step per
    frame against 64 plain per-context steps, same contexts and frames."""
    import torch
    from paper_2510_06873_gb300 import tune
    mp = synth.method_params(4)
    cfgp = synth.CONFIG_PARAMS[4]
    nsys = cfgp["systems"]
    n, k, dens = synth.batch_layout(4, n_systems=nsys)
    systems = [synth.wurtzite_system(int(n[s]), cfg=4, sys=s, density_scale=float(dens[s])) for s in range(nsys)]
    ctxs = []
    for s, sysm in enumerate(systems):
        p = metad.params_for(sysm.n, sysm.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream,
                             hill_capacity=int(k[s]) + 64)
        ctx, _, _ = _seeded_hills(metad, sysm, mp, 4, int(k[s]), stream, dev, p)
        ctxs.append(ctx)
    nfr = 4  # 4 resident frames per system: about 150 MB of positions, more than L2
    frames = [[torch.from_numpy(synth.perturbed_frame(sysm, f)).to(dev) for f in range(nfr)] for sysm in systems]
    F = [torch.zeros((sysm.n, 3), dtype=torch.float32, device=dev) for sysm in systems]
    steps = max(1, args.batched_steps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def plain(t):
        for s, ctx in enumerate(ctxs):
            ctx.step(frames[s][t % nfr], F[s])

    batch = metad.Batch(ctxs)

    def batched(t):
        batch.step([fr[t % nfr] for fr in frames], F)

    for t in range(3):
        plain(t)
    torch.cuda.synchronize(dev)
    l0 = sum(c.launch_count for c in ctxs)
    ev0.record(stream)
    for t in range(steps):
        plain(t)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = ev0.elapsed_time(ev1) / steps
    plain_launches = (sum(c.launch_count for c in ctxs) - l0) / steps
    tuned = tune.tune_batch(batch, [fr[0] for fr in frames], F, stream)
    for t in range(3):
        batched(t)
    torch.cuda.synchronize(dev)
    b0 = batch.launch_count
    ev0.record(stream)
    for t in range(steps):
        batched(t)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    batch_ms = ev0.elapsed_time(ev1) / steps
    batch_launches = (batch.launch_count - b0) / steps
    atoms = int(sum(sysm.n for sysm in systems))
    batch.close()
    for c in ctxs:
        c.close()
    return {"systems": nsys, "atoms": atoms, "hills": int(np.sum(k)), "steps": steps,
            "plain_ms_per_step": plain_ms, "batched_ms_per_step": batch_ms,
            "plain_atom_steps_per_s": atoms / (plain_ms / 1e3), "batched_atom_steps_per_s": atoms / (batch_ms / 1e3),
            "speedup": plain_ms / batch_ms, "kernels_per_step": {"plain": plain_launches, "batched": batch_launches},
            "tile": tuned["tile"], "tile_ms": {str(c): v for c, v in tuned["ms_per_step"].items()},
            "inputs": f"{nfr} resident frames per system cycled (positions > L2)"}


def run_small_cvs(args, dev, stream, metad):
    """The torsion and nearest-distance CV families on many small walkers:
    256 chain-molecule walkers (22 atoms, two backbone torsions, 10,000 hills
    each, plain metadynamics, sigma 0.35 rad) and 32 slab + water walkers
    (717 atoms, surface-oxygen to nearest-hydrogen distance, 1,500
    well-tempered hills each): one batched step per frame against plain
    per-walker steps, plus one walker's step latency replayed from a CUDA
    graph.  The hill sums (FP64) are the dominant work; hill evaluations per
    second are reported beside walker-steps per second."""
    import torch
    out = {}
    steps = max(1, args.batched_steps)
    specs = []
    pp = synth.SMALL_PARAMS["peptide"]
    pep = []
    for w in range(256):
        p = metad.params_for(synth.PEPTIDE_ATOMS, synth.peptide_box(), n_cv=2, sigma=pp["sigma"], w0=pp["w0"],
                             biasfactor=pp["biasfactor"], cv_kind="torsion", hill_capacity=pp["hills"] + 64,
                             stream=stream.cuda_stream)
        c = metad.Metad(p)
        c.set_cv_atoms(synth.PEPTIDE_TORSIONS)
        cen = synth.torus_centres(w, pp["hills"])
        c.load_hills(cen, np.full(len(cen), pp["w0"]))
        pep.append((c, [synth.peptide_frame(4 * w + f, sys=w) for f in range(4)]))
    specs.append(("torsion_walkers", pep, pp["hills"]))
    sp = synth.SMALL_PARAMS["surface_water"]
    surf = []
    layouts = [synth.SurfaceWater(sys=k) for k in range(4)]  # 8 walkers per layout, own frames and hills
    for w in range(32):
        sw = layouts[w % 4]
        p = metad.params_for(sw.n, sw.box, n_cv=1, sigma=sp["sigma"], w0=sp["w0"], biasfactor=sp["biasfactor"],
                             cv_kind="nearest", hill_capacity=sp["hills"] + 64, stream=stream.cuda_stream)
        c = metad.Metad(p)
        c.set_cv_atoms(sw.cv_atoms())
        cen = synth.interval_centres(synth.SURFACE_CFG, w, sp["hills"], sp["cv_lo"], sp["cv_hi"])
        c.deposit_hills(cen, want_heights=False)
        surf.append((c, [sw.frame(4 * w + f) for f in range(4)]))
    specs.append(("nearest_distance_walkers", surf, sp["hills"]))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, walkers, hills in specs:
        ctxs = [c for c, _ in walkers]
        frames = [[torch.from_numpy(f).to(dev) for f in fr] for _, fr in walkers]
        F = [torch.zeros((fr[0].shape[0], 3), dtype=torch.float32, device=dev) for fr in frames]
        batch = metad.Batch(ctxs)

        def plain(t):
            for k, c in enumerate(ctxs):
                c.step(frames[k][t % 4], F[k])

        def batched(t):
            batch.step([fr[t % 4] for fr in frames], F)

        res = {}
        for label, fn, count in (("plain", plain, lambda: sum(c.launch_count for c in ctxs)),
                                 ("batched", batched, lambda: batch.launch_count)):
            for t in range(3):
                fn(t)
            torch.cuda.synchronize(dev)
            l0 = count()
            ev0.record(stream)
            for t in range(steps):
                fn(t)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            res[label] = (ev0.elapsed_time(ev1) / steps, (count() - l0) / steps)
        batch.close()
        # one walker alone, its step replayed from a captured CUDA graph
        c0 = ctxs[0]
        c0.set_step_graph(True)
        for t in range(3):
            c0.step(frames[0][0], F[0])
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for t in range(200):
            c0.step(frames[0][0], F[0])
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        alone_us = ev0.elapsed_time(ev1) / 200 * 1e3
        nw = len(ctxs)
        pm, pk = res["plain"]
        bm, bk = res["batched"]
        out[name] = {"walkers": nw, "atoms_per_walker": int(frames[0][0].shape[0]), "hills_per_walker": hills,
                     "steps": steps, "plain_ms_per_step": pm, "batched_ms_per_step": bm,
                     "plain_walker_steps_per_s": nw / (pm / 1e3), "batched_walker_steps_per_s": nw / (bm / 1e3),
                     "batched_hill_evals_per_s": nw * hills / (bm / 1e3), "speedup": pm / bm,
                     "kernels_per_step": {"plain": pk, "batched": bk}, "one_walker_graph_step_us": alone_us}
        for c in ctxs:
            c.close()
    return out


def run_npt(args, dev, stream, metad, n_atoms):
    """The same system under triaxial NPT with the lattice-parameter CVs of
    the GaN runs: CVs (s1, s2, L_x, L_y, L_z), 5-D well-tempered hills
    (20,000, deposited by the CUDA path), a new box every step
    (metad_set_box) and the box gradient (bias virial) beside the forces.
    Timed with CUDA events like the main step."""
    import torch
    system = make_system(n_atoms)
    mp = synth.method_params(3)
    nfr, hills = 4, 20000
    frames = [synth.npt_frame(system, f, strain_sigma=1e-3, period=400) for f in range(nfr)]
    pos = [torch.from_numpy(fr).to(dev) for fr, _ in frames]
    F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    sig_l = (0.05, 0.05, 0.05)
    p = metad.params_for(system.n, system.box, n_cv=2, sigma=mp.sigma, lattice_cvs=True, sigma_lattice=sig_l,
                         hill_capacity=hills + 64, stream=stream.cuda_stream)
    ctx = metad.Metad(p)
    ctx.set_box(frames[0][1])
    ctx.build_neighbors(pos[0])
    s_ref = ctx.cv_forward()
    cen = synth.hill_centres(3, system.sys, s_ref, tuple(mp.sigma) + sig_l, hills, half_width_sigmas=4.0)
    ctx.deposit_hills(cen, want_heights=False)

    def one(t):
        ctx.set_box(frames[t % nfr][1])
        ctx.step(pos[t % nfr], F)

    for t in range(3):
        one(t)
    torch.cuda.synchronize(dev)
    steps = max(1, args.batched_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(steps):
        one(t)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    bg = ctx.box_gradient()
    reb = ctx.rebuild_count
    ctx.close()
    return {"atoms": system.n, "cvs": "s1, s2, L_x, L_y, L_z", "hills": hills, "steps": steps,
            "ms_per_step": ms, "atom_steps_per_s": system.n / (ms / 1e3),
            "box_gradient_last": [float(x) for x in bg], "rebuilds": int(reb),
            "note": "a new box every step (strain 1e-3 sin(2 pi f / 400 + phase) per axis, 4 frames cycled); "
                    "the Verlet rows are rebuilt when the moves and the box change leave the skin; "
                    "the box gradient is the lattice term plus the bias virial"}


def run_served(args, dev, stream, metad):
    """32 walkers (2k-500k atoms, 1,000 hills each), 2,000 Poisson requests at
    5,000/s: continuous batching against sequential plain evaluation."""
    import torch
    from paper_2510_06873_gb300 import serve
    mp = synth.method_params(5)
    cfgp = synth.CONFIG_PARAMS[5]
    n_w, arrivals, walker_of = synth.served_trace(5, n_walkers=cfgp["walkers"], n_requests=cfgp["requests"],
                                                  rate_hz=cfgp["rate_hz"])
    systems = [synth.wurtzite_system(int(n_w[w]), cfg=5, sys=w) for w in range(len(n_w))]

    def make_walkers(runs=1):
        out = []
        for w, sysm in enumerate(systems):
            p = metad.params_for(sysm.n, sysm.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream,
                                 hill_capacity=cfgp["hills"] + runs * cfgp["requests"] // cfgp["deposit_every"] + 64)
            out.append(serve.Walker(params=p, centres=hill_sets[w][0], heights=hill_sets[w][1], frames=frames[w]))
        return out

    hill_sets, frames = [], []
    for w, sysm in enumerate(systems):
        p = metad.params_for(sysm.n, sysm.box, n_cv=2, sigma=mp.sigma, stream=stream.cuda_stream,
                             hill_capacity=cfgp["hills"] + 64)
        ctx, cen, hw = _seeded_hills(metad, sysm, mp, 5, cfgp["hills"], stream, dev, p)
        ctx.close()
        hill_sets.append((cen, hw))
        frames.append([torch.from_numpy(synth.perturbed_frame(sysm, f)).pin_memory() for f in range(3)])
    srv = serve.Server(make_walkers(), stream, budget_bytes=cfgp["budget_bytes"],
                       deposit_every=cfgp["deposit_every"])
    srv.preload()
    served = srv.run(arrivals, walker_of)
    srv.close()
    plain_walkers = make_walkers()
    plain = serve.run_plain(plain_walkers, stream, arrivals, walker_of, deposit_every=cfgp["deposit_every"])
    for wk in plain_walkers:
        wk.ctx.close()
    agree = all(np.array_equal(a.cv, b.cv) and a.V == b.V for a, b in zip(served.requests, plain.requests))
    s, q = served.summary(), plain.summary()
    sweep = None
    if not args.no_sweep:
        sweep = served_sweep(args, stream, serve, cfgp, n_w, make_walkers)
    return {"walkers": len(n_w), "atoms_resident": int(sum(sysm.n for sysm in systems)),
            "requests": len(arrivals), "rate_hz": cfgp["rate_hz"], "budget_bytes": cfgp["budget_bytes"],
            "served": s, "plain": q, "p99_ratio_plain_over_served": q["p99_ms"] / s["p99_ms"],
            "throughput_ratio": s["atom_steps_per_s"] / q["atom_steps_per_s"],
            "results_identical_to_plain": bool(agree), "kernels": served.launches, "sweep": sweep,
            "h2d": "positions from page-locked host memory per request; forces and CVs back per request"}


SWEEP_RATES = (5000.0, 10000.0, 20000.0, float("inf"))
SWEEP_SEEDS = (1, 2, 3)


def served_sweep(args, stream, serve, cfgp, n_w, make_walkers):
    """Offered rate against capacity: the served loop and sequential plain
    evaluation on the same walkers, each rate with three request streams
    (synth.served_arrivals seeds 1-3; an infinite rate is a burst of all
    requests at t = 0, i.e. saturation).  Throughput is requests completed
    over the span from the first arrival to the last completion; p50 / p99
    are per-request latencies.  One server and one plain walker set serve
    every stream in turn (their hills grow by the deposits on the way)."""
    runs = len(SWEEP_RATES) * len(SWEEP_SEEDS)
    srv = serve.Server(make_walkers(runs), stream, budget_bytes=cfgp["budget_bytes"],
                       deposit_every=cfgp["deposit_every"])
    srv.preload()
    plain_walkers = make_walkers(runs)
    points = []
    for rate in SWEEP_RATES:
        per = {"served": [], "plain": []}
        for seed in SWEEP_SEEDS:
            arr, wof = synth.served_arrivals(5, len(n_w), cfgp["requests"], rate, seed)
            per["served"].append(srv.run(arr, wof).summary())
            per["plain"].append(serve.run_plain(plain_walkers, stream, arr, wof,
                                                deposit_every=cfgp["deposit_every"]).summary())
        pt = {"offered_req_s": None if math.isinf(rate) else rate, "saturation": math.isinf(rate)}
        for mode in ("served", "plain"):
            rows = per[mode]
            pt[mode] = {key: {"mean": float(np.mean([r[key] for r in rows])), "min": float(min(r[key] for r in rows)),
                              "max": float(max(r[key] for r in rows))}
                        for key in ("throughput_req_s", "atom_steps_per_s", "p50_ms", "p99_ms")}
            pt[mode]["mean_batch"] = float(np.mean([r["mean_batch"] for r in rows]))
        pt["throughput_ratio"] = pt["served"]["throughput_req_s"]["mean"] / pt["plain"]["throughput_req_s"]["mean"]
        points.append(pt)
    srv.close()
    for wk in plain_walkers:
        if wk.ctx is not None:
            wk.ctx.close()
    return {"requests_per_run": cfgp["requests"], "seeds": list(SWEEP_SEEDS), "points": points,
            "capacity_req_s": {"served": points[-1]["served"]["throughput_req_s"]["mean"],
                               "plain": points[-1]["plain"]["throughput_req_s"]["mean"]}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_metad(args)


if __name__ == "__main__":
    sys.exit(main())
