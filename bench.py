#!/usr/bin/env python3
"""Benchmark of the particle <-> dual-grid coupling step on GB300.

Workload (default): the clustered bed, the largest single-GPU
configuration (1 x 1 x 0.5 m, fine 512 x 512 x 256, ratio 4 -> bulk
128 x 128 x 64, 32,000,000 log-normal spheres in 200 Gaussian clusters,
Di Felice drag, gravity, FP32), seeded synthetic inputs resident in HBM.
One step is one call of cg_step with dt = 1e-4: bin, porosity, fluid
average, drag with the fused reaction deposit and the semi-implicit Euler
advance of the particles, projection of the source and of the porosity
onto the fine grid, and the conservation sums.  The particles move from
step to step, so every timed step rebins a new state.  --workload
packed_bed times the 4M-particle packed bed (no advance) instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (the path does not shard): value is the
total particle-steps of all ranks over the slowest rank's time.

--impl reference times the FP64 CPU oracle on the same workload (rank 0
only, a bounded number of full steps on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled particle-steps/s"
UNIT = "particle-steps/s"

# DRAM traffic per launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel, valid only while the kernel's
# source files are byte-identical to the ones profiled (sha256 prefixes).
NCU_TRAFFIC = {
    # packed bed, one warm launch of k_average<float,4>: 405.5 MB read + 8.1 MB written
    ("packed_bed", "average"): {"files": {"fine.cu": "b5357b772279f4b1"}, "bytes": 413.6e6},
    # clustered-bed recipe at 16M particles, a warm sorted step of k_drag<float,1>:
    # 578.7 MB read + 904.7 MB written, times 2 for the 32M bed (traffic per particle)
    ("clustered_bed", "drag"): {"files": {"drag.cu": "96408310edce01e8", "drag_law.cuh": "e2f8745533c61039"},
                                "bytes": 2.967e9},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="clustered_bed",
                    choices=["packed_bed", "small_packed_bed", "clustered_bed", "medium_clustered_bed",
                             "small_clustered_bed"])
    ap.add_argument("--batch", action="store_true",
                    help="64 uneven instances: batched persistent launches vs one by one")
    ap.add_argument("--learned", action="store_true",
                    help="train the drag closure on the workload family, then compare learned and plain steps")
    ap.add_argument("--activation", choices=("gelu", "relu"), default="relu",
                    help="activation of the closure trained by --learned or timed by --closure-drag")
    ap.add_argument("--closure-drag", action="store_true",
                    help="time the learned drag kernel alone on the workload (a random closure whose feature box "
                         "holds every row): the profiling case of the closure")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=0,
                    help="full oracle steps in the CPU baseline (0: one above 8M particles, else two)")
    ap.add_argument("--no-graph", action="store_true", help="time eager cg_step calls instead of a CUDA graph")
    ap.add_argument("--map", action="store_true",
                    help="time the maps between non-nested grids (bulk 64x64x128, fine 250x250x500 offset)")
    ap.add_argument("--reorder", action="store_true",
                    help="reorder the particles into cell order once before timing (cg_reorder_particles) and "
                         "bin with the per-cell sort")
    ap.add_argument("--particles", type=int, default=0,
                    help="clustered-bed workloads only: this many particles on the workload's grid (profiling "
                         "cases of the same recipe)")
    ap.add_argument("--step", choices=["auto", "sorted", "caller"], default="auto",
                    help="the step timed: cg_step_sorted (particles left in cell order every step; the default "
                         "for an advancing workload) or cg_step (the caller's particle order kept)")
    ap.add_argument("--stencil", choices=("gather", "window"), default="gather",
                    help="the drag's stencil reads: eight loads per particle from L1/L2, or each warp's stencil "
                         "window staged in shared memory (sorted step only)")
    ap.add_argument("--implicit", action="store_true",
                    help="also form the semi-implicit exchange coefficients (bulk and fine) in every step "
                         "(device entry only: no e2e line)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device=None):
    """The largest value of x over all ranks (x itself on one rank): the
    job's time is the slowest replica's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, steps, seconds):
    """Units all replicas processed over the slowest replica's time."""
    return world * units_per_rank * steps / seconds


def file_sha(path):
    """Hash of a source's code with its comments and whitespace removed, so that
    stored counters outlive an edit of the comments alone."""
    with open(path) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


class ClockSampler:
    """nvidia-smi clock / throttle samples, kept with their timestamps."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self._t is not None:
            self._t.join(timeout=2)

    def summary(self, t0, t1):
        rows = []
        for ts, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            rows.append((ts, parts))
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15] or \
            sorted(rows, key=lambda r: abs(r[0] - (t0 + t1) / 2))[:3]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[0]) for _, p in inside if num(p[0]) is not None]
        smax = [num(p[1]) for _, p in inside if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, p in inside for i in range(4) if p[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inside),
                "power_w_max": max((num(p[2]) or 0.0) for _, p in inside)}


CLUSTERED_GRIDS = {"clustered_bed": (512, 512, 256), "medium_clustered_bed": (256, 256, 128),
                   "small_clustered_bed": (128, 128, 64)}


def make_workload(args, seed):
    """The named synthetic workload; --particles re-draws a clustered bed
    with that many particles on the same grid."""
    import synth
    if args.particles > 0:
        if args.workload not in CLUSTERED_GRIDS:
            raise SystemExit("--particles applies to the clustered-bed workloads")
        return synth.clustered_bed(seed=seed, fine_n=CLUSTERED_GRIDS[args.workload], n=args.particles)
    return getattr(synth, args.workload)(seed=seed)


def workload_name(name, w):
    """The workload with its sizes, as the JSON line's config names it."""
    d = w.desc
    box = "x".join(f"{e:g}" for e in d["extent"])
    law = "Di Felice" if d["law"] == 0 else "Ergun/Wen-Yu"
    prec = "FP64" if d.get("fp64") else "FP32"
    return (f"{name}: {box} box, fine {'x'.join(map(str, d['fine_n']))}, ratio {d['ratio']}, "
            f"{w.n} spheres, {law}, {prec}")


def algorithmic_bytes(g, n, eps_fine=True, implicit=False, euler=False, sorted_step=False):
    """Algorithmic bytes of one step (the minimal traffic of the path) and,
    per launch, of each kernel of this implementation (bytes it must move
    to do its part, FP32; L2-resident gathers of the bulk fields and
    histogram / scan scratch are not counted).

    Step: particles read x, y, z, d (16) and u_p (12), write F (12), plus
    the bin key and permutation written and read once (8); fine cells read
    u_f (12) and write S_f (12) and eps_f (4); bulk cells ~40 B.  With the
    Euler advance, particles also write x and u_p back (24)."""
    import paper_1807_11834_gb300 as cg
    nf, nb = g.n_fine, g.n_bulk
    nbx = nb  # bulk cells
    choice = int(g.desc.get("sort_digits", 0))
    cell_sort = choice == cg.CG_SORT_CELLS or (
        choice == cg.CG_SORT_AUTO and n <= cg.CG_SORT_CELLS_AUTO_MAX and n <= cg.CG_SORT_CELLS_AUTO_DENSITY * nb)
    per = {
        "bin_key": n * (16 + 4 + 4 + (4 if cell_sort else 0)),   # pos read; key, volume (, arrival rank) written
        "bin_scatter": n * (12 + 28) // 2,                # pass 1: 4 r + 8 w; pass 2: 12 r + 16 w (mean)
        "bin_hist": n * 4,
        "bin_place": n * (4 + 4 + 4),                     # key, rank read; id written at its slot
        "bin_seg_sort": n * (4 + 4 + 16),                 # placed id, diameter read; perm, key, inverse, diameter written
        "deposit_volume": (nbx * 8 + n * 8 + nbx * 8) // 2,   # fill eps; read sorted volume + key; write eps
        "pack": nbx * (8 + 12 + 16 + 4),
        "drag": n * (16 + 16 + 4 + 12 + 16),              # pos, vel, slot read; F and sorted F written
        "deposit_momentum": n * (16 + 4) + nbx * 12,
        "project": nf * 12 + nbx * 12,                    # S_f written, S_B read
        "project_eps": nf * 4 + nbx * 4,                  # eps_f written, eps_B read
        "average": nf * 12 + nbx * 16,                    # u_f read, u_B and var written
        "deposit_implicit": n * (16 + 4) + nbx * 16,      # sorted (beta, beta u) + key read; A, b written
        "project_implicit": nf * 16 + nbx * 16,           # A_f, b_f written, A, b read
        # incremental rebinning (the movers' placement and the idle fallback not counted)
        "rebin_key": n * (16 + 4 + 4),                    # pos read; key, diameter written
        "rebin_mark": n * ((16 + 4 + 4 + 4) if sorted_step else (4 + 4 + 4 + 8)),
        # sorted input: pos, old cell read; diameter, record written;
        # else old id, old cell, new cell (gathered) read; record, old id written
        "rebin_cells": nbx * 16,                          # old starts, departures, arrivals read; counts written
        "rebin_slots": n * (4 + 4 + 16 + (0 if sorted_step else 4)),
        # stayers (the movers beside them not counted): record, diameter (and
        # in caller order the old id) read; perm, cell, inverse, diameter written
    }
    step = n * 48 + nf * (24 + (4 if eps_fine else 0)) + nb * 40
    if euler:
        per["drag"] += n * 24                             # x and u_p written back
        step += n * 24
    if implicit:
        per["drag"] += n * 16                             # the sorted (beta, beta u) record
        step += n * 16 + nf * 16 + nb * 16                # beta, beta u per particle; A, b on both grids
    return step, per


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_1807_11834_gb300 as cg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = make_workload(args, rank)
    dt = float(w.dt)                # 1e-4 for the clustered bed (advanced every step), 0 for the packed bed
    # the advancing workload steps with cg_step_sorted, which leaves the
    # particles in cell order (as a DEM code keeps them); --step caller times
    # cg_step, which keeps the caller's particle order
    sorted_step = args.step == "sorted" or (args.step == "auto" and dt > 0)
    if args.reorder:
        w.desc["sort_digits"] = cg.CG_SORT_CELLS
    w.desc["stencil"] = cg.CG_STENCIL_WINDOW if args.stencil == "window" else cg.CG_STENCIL_GATHER
    g = cg.Grids(w.desc)
    n = w.n
    dev = torch.device("cuda", local)
    pos = torch.from_numpy(w.pos_d).to(dev)
    vel = torch.from_numpy(w.vel).to(dev)
    if args.reorder:
        # a DEM code keeps its particles in cell order: once, before timing
        pos2, vel2 = torch.empty_like(pos), torch.empty_like(vel)
        g.cg_bin_particles(pos)
        g.cg_reorder_particles(pos, vel, pos2, vel2)
        torch.cuda.synchronize()
        pos, vel = pos2, vel2
    uf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).to(dev)
    out = g.alloc_outputs(n, var=True, eps_fine=True, implicit=args.implicit, implicit_fine=args.implicit,
                          device=dev)
    if args.implicit:
        args.no_e2e = True   # the host-buffer entries do not form the semi-implicit fields
    input_bytes = pos.numel() * 4 + vel.numel() * 4 + uf.numel() * 4
    # an advanced workload is a run of w.steps steps from its initial state
    # (the clustered bed: 100; explicit Euler at dt = 1e-4 is not stable for
    # the smallest spheres in the clamped cluster cores over much longer
    # runs): timed steps come in such runs, each from a copy of the initial
    # state made outside the timed region
    run_len = int(w.steps) if dt > 0 else 0
    pos0, vel0 = pos.clone(), vel.clone()
    # the sorted step reads one pair of particle arrays and writes the other
    bufs = [(pos, vel), (torch.empty_like(pos), torch.empty_like(vel))] if sorted_step else [(pos, vel)]
    par = [0]
    replayed = [0]   # kernels of the graph replays so far

    def reset():
        if run_len:
            pos.copy_(pos0)
            vel.copy_(vel0)
            par[0] = 0

    def step_sorted():
        src, dst = bufs[par[0]], bufs[par[0] ^ 1]
        g.cg_step_sorted(src[0], src[1], dst[0], dst[1], uf, out, dt=dt)
        par[0] ^= 1

    def step_caller():
        g.cg_step(pos, vel, uf, out, dt=dt)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        """Device time of `steps` calls of fn (CUDA events on the launching
        stream), in runs of run_len steps each from the initial state when
        the workload advances; the resets stay outside the events."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total, left = 0.0, steps
        barrier()
        t0 = time.time()
        while left > 0:
            k = min(run_len, left) if run_len else left
            reset()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(k):
                fn()
            e1.record()
            e1.synchronize()
            total += e0.elapsed_time(e1)
            left -= k
        t1 = time.time()
        barrier()
        return total, t0, t1

    def graphed(eager_fn, variants):
        """CUDA graphs of the step, one per particle buffer the step can start
        from, replayed in turn; captured on a side stream after the handle has
        stepped through every variant once (so that each capture sees the
        handle state its replays will meet)."""
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        g.set_stream(cs)
        with torch.cuda.stream(cs):
            for _ in range(2 * variants):
                eager_fn()
        cs.synchronize()
        graphs, counts = [], []
        for _ in range(variants):
            gr = torch.cuda.CUDAGraph()
            c0 = g.cg_launch_count()
            with torch.cuda.graph(gr, stream=cs):
                eager_fn()
            counts.append(g.cg_launch_count() - c0)   # the library's kernels the graph holds
            graphs.append(gr)
        g.set_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()

        def replay():
            graphs[par[0]].replay()
            replayed[0] += counts[par[0]]
            par[0] = (par[0] + 1) % variants
        return replay

    eager_fn = step_sorted if sorted_step else step_caller
    for _ in range(max(3, args.warmup)):
        eager_fn()
    rc, flags, counts = g.cg_sync_status()
    if rc != 0:
        raise RuntimeError(f"warm-up status {rc} flags {flags} counts {counts}")
    reset()

    eager_ms, _, _ = timed(eager_fn, min(args.steps, 200))
    eager_ms_step = eager_ms / min(args.steps, 200)
    step_fn = eager_fn
    if not args.no_graph:
        reset()
        step_fn = graphed(eager_fn, 2 if sorted_step else 1)
        reset()
        for _ in range(max(3, args.warmup)):
            step_fn()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.35)
    replayed[0] = 0
    l0 = g.cg_launch_count()
    ms, t0, t1 = timed(step_fn, args.steps)
    # the library's kernels launched in the timed region: those of the
    # replayed graphs, or counted as launched by the eager steps
    launches = replayed[0] if step_fn is not eager_fn else g.cg_launch_count() - l0
    time.sleep(0.25)
    sampler.stop()
    ms = max_over_ranks(ms, world, dev)
    rc, flags, counts = g.cg_sync_status()
    if rc != 0:
        raise RuntimeError(f"timed status {rc}")

    # the other step of an advancing workload, timed the same way: cg_step
    # keeps the caller's (generated, random) particle order
    caller = None
    if sorted_step and not args.no_graph:
        reset()
        for _ in range(max(3, args.warmup)):
            step_caller()
        reset()
        par[0] = 0   # one graph: its replays take index 0 (reset leaves it alone when nothing advances)
        caller_fn = graphed(step_caller, 1)
        ms_c, _, _ = timed(caller_fn, min(args.steps, 400))
        ms_c /= min(args.steps, 400)
        caller = {"ms_per_step": round(ms_c, 5), "value": n / (ms_c * 1e-3),
                  "entry": "cg_step (particles kept in the caller's order, incremental rebinning from the last step)"}
        par[0] = 0

    # per-kernel device time: a second pass of the same steps with the
    # library's CUDA events around every launch (kept out of the timed pass;
    # the library runs the step on one stream while timing kernels, so each
    # event pair measures one kernel alone)
    prof_steps = min(args.steps, 200)
    g.cg_profile_reset()
    g.cg_profile_enable(True)
    for k in range(prof_steps):
        if k == 0 or (run_len and k % run_len == 0):
            reset()
        eager_fn()
    prof = g.cg_profile_read()
    g.cg_profile_enable(False)

    step_bytes, kern_bytes = algorithmic_bytes(g, n, implicit=args.implicit, euler=dt > 0, sorted_step=sorted_step)
    peak, peak_src = load_peaks()
    kern_ms = {k: v[1] / v[0] for k, v in prof.items() if v[0]}
    kern_total = {k: v[1] for k, v in prof.items()}
    tot = sum(kern_total.values())
    dominant = max((k for k in kern_total if k in kern_bytes), key=kern_total.get)
    kern_launches = {k: v[0] / prof_steps for k, v in prof.items()}
    dom_bytes = kern_bytes.get(dominant)
    roofline = None
    if dom_bytes is not None:
        ach = dom_bytes / (kern_ms[dominant] * 1e-3) / 1e9
        tr = NCU_TRAFFIC.get((args.workload, dominant))
        traffic = None
        # the counters hold only while every source of the kernel is the one they were taken from
        if tr and all(sha == file_sha(os.path.join(ROOT, "paper_1807_11834_gb300", "csrc", f))
                      for f, sha in tr["files"].items()):
            traffic = tr["bytes"]
        roofline = {"bound": "hbm", "kernel": dominant, "achieved": round(ach, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": traffic,
                    "algorithmic_bytes": dom_bytes, "ms_per_launch": round(kern_ms[dominant], 5),
                    "peak_source": peak_src,
                    "timing": "serialized per-kernel CUDA events over a profiled pass of the same steps"}
    ms_step = ms / args.steps
    step_gbs = step_bytes / (ms_step * 1e-3) / 1e9
    value = job_throughput(world, n, args.steps, ms * 1e-3)
    clocks = sampler.summary(t0, t1)

    # end-to-end: host buffers through the host entries (H2D of the inputs and
    # D2H of every output inside the timed region, every step).  The
    # pipelined entry enqueues each step (copies in, step, copies out) and the
    # timed region ends after the wait for the last one; the blocking entry
    # is timed too.  The host entries keep the caller's particle order.
    e2e = None
    if not args.no_e2e:
        hpos = pos0.cpu().pin_memory()
        hvel = vel0.cpu().pin_memory()
        huf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).pin_memory()
        hout = {k: (torch.empty(v.shape, dtype=v.dtype).pin_memory() if v is not None else None)
                for k, v in out.items()}
        for _ in range(2):
            g.cg_step_host(hpos, hvel, huf, hout, dt=dt)
        ke = max(3, min(args.steps, 30))    # within one run of an advanced workload

        def host_run(pipelined):
            barrier()
            ta = time.perf_counter()
            for _ in range(ke):
                if pipelined:
                    g.cg_step_host_async(hpos, hvel, huf, hout, dt=dt)
                else:
                    g.cg_step_host(hpos, hvel, huf, hout, dt=dt)
            if pipelined:
                g.cg_step_host_wait()
            return max_over_ranks(time.perf_counter() - ta, world, dev)

        te_sync = host_run(False)
        te = host_run(True)
        d2h = sum(v.numel() * v.element_size() for v in hout.values() if v is not None)
        if dt > 0:
            d2h += hpos.numel() * 4 + hvel.numel() * 4     # the advanced particles come back too
        e2e = {"value": job_throughput(world, n, ke, te), "unit": UNIT, "h2d_bytes_per_step": int(input_bytes),
               "d2h_bytes_per_step": int(d2h), "steps": ke, "ms_per_step": 1e3 * te / ke,
               "entry": "cg_step_host_async per step + cg_step_host_wait (pinned host buffers)",
               "blocking_entry_ms_per_step": 1e3 * te_sync / ke}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(args, w, dt)

    if world > 1:
        dist.barrier()
    if rank == 0:
        if args.reorder:
            order = "reordered into cell order once before timing, per-cell sort"
        elif sorted_step:
            order = (w.notes.get("order", "as generated") + " at the start of each run; every step writes the "
                     "advanced particles in its own cell order (cg_step_sorted, two particle buffers)")
        else:
            order = w.notes.get("order", "as generated")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w.desc.get("fp64") else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.workload, w),
                       "particles": n, "fine_cells": g.n_fine, "bulk_cells": g.n_bulk,
                       "parallelism": f"replicas x{world}",
                       "l2": (f"inputs {input_bytes / 1e6:.0f} MB {'>' if input_bytes > 126e6 else '<'} L2 (126 MB) "
                              "per step, no flush"),
                       "step": "cg_step_sorted" if sorted_step else "cg_step",
                       "stencil": args.stencil,
                       "timing": ("CUDA graph of one step, replayed K times" if not args.no_graph
                                  else "eager step calls") + (" (one graph per particle buffer, in turn)"
                                                              if sorted_step and not args.no_graph else ""),
                       "eager_ms_per_step": round(eager_ms_step, 5),
                       "launches_per_step": round(launches / args.steps, 3),
                       "step_algorithmic_bytes": step_bytes, "step_gbs": round(step_gbs, 1),
                       "step_frac_of_hbm": round(step_gbs / peak, 4),
                       "semi_implicit": bool(args.implicit),
                       "dt": dt, "euler_advance": dt > 0,
                       "run_length": (f"timed in runs of {run_len} steps, each from the initial state "
                                      "(reset outside the timed region)") if run_len else "one run",
                       "particle_order": order},
            "caller_order_step": caller,
            "roofline": roofline,
            "kernels": {k: {"ms_per_launch": round(kern_ms[k], 5), "share": round(kern_total[k] / tot, 4),
                            "launches_per_step": kern_launches[k]} for k in sorted(kern_total)},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line))
    g.close()
    if world > 1:
        dist.destroy_process_group()


def oracle_rate(w, dt, steps, threads):
    """(particle-steps/s, seconds) of `steps` whole oracle steps of w from its
    initial state, each from the state the last one advanced."""
    import oracle
    oracle.build(threads=threads)
    pos, vel = w.pos_d, w.vel
    ta = time.perf_counter()
    for _ in range(steps):
        r = oracle.step(w.desc, pos, vel, w.u_fine, dt=dt, want_eps_fine=True, threads=threads)
        pos, vel = r["pos_d"], r["vel"]
    tc = time.perf_counter() - ta
    return w.n * steps / tc, tc


def oracle_baseline(args, w, dt):
    """The FP64 oracle on the host cores: the OpenMP build on every core (the
    headline baseline) and the single-thread build, each on a bounded
    sample of whole steps of the same workload."""
    cores = os.cpu_count() or 1
    name = args.workload.replace("_", " ")
    big = w.n > 8_000_000
    k1 = args.cpu_steps if args.cpu_steps > 0 else (1 if big else 2)
    v1, t1 = oracle_rate(w, dt, k1, threads=False)
    single = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"{k1} full oracle step{'s' if k1 > 1 else ''} (dt {dt:g}) of the same {name} from its "
                        f"initial state (FP64 C, single thread), {t1:.1f} s"}
    try:
        kn = max(k1, 2 if big else 4)
        vn, tn = oracle_rate(w, dt, kn, threads=True)
    except Exception as e:   # no OpenMP on this host: the single-thread figure stands alone
        single["all_cores_unavailable"] = str(e)[:200]
        return single
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{kn} full oracle steps (dt {dt:g}) of the same {name} from its initial state (FP64 C, "
                      f"OpenMP build over the independent particle and cell loops, {cores} threads, results "
                      f"bit-identical to the single-thread build), {tn:.1f} s",
            "single_thread": single}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import synth
    import oracle
    w = make_workload(args, 0)
    n = w.n
    dt = float(w.dt)
    cores = os.cpu_count() or 1
    threads = True
    try:
        oracle.build(threads=True)
    except Exception:
        threads, cores = False, 1
        oracle.build()
    # a bounded sample: whole steps of the workload, as many as fit a few minutes
    wu = min(max(0, args.warmup), 1)
    ks = max(1, min(args.steps, 4 if n > 8_000_000 else 8))
    pos, vel = w.pos_d, w.vel
    for _ in range(wu):
        r = oracle.step(w.desc, pos, vel, w.u_fine, dt=dt, want_eps_fine=True, threads=threads)
        pos, vel = r["pos_d"], r["vel"]
    ta = time.perf_counter()
    for _ in range(ks):
        r = oracle.step(w.desc, pos, vel, w.u_fine, dt=dt, want_eps_fine=True, threads=threads)
        pos, vel = r["pos_d"], r["vel"]
    tc = time.perf_counter() - ta
    value = n * ks / tc
    sample = (f"{ks} full oracle steps (warm-up {wu}, dt {dt:g}, each from the state the last one advanced) of the "
              f"{args.workload.replace('_', ' ')}, FP64 C, "
              + (f"OpenMP build on {cores} threads (bit-identical to the single-thread build)" if threads
                 else "single thread"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": ks, "warmup": wu, "ms_per_step": 1e3 * tc / ks, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, w),
                       "particles": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_learned(args):
    """Learned closure against the plain path on one workload family:
    train on seeds 0 and 1 (56-step runs, stale records refreshed every 2,
    5, 10, 20 and 50 steps, fluid relaxed by the coupling source), score the
    drag error on seed 2
    at several refresh intervals K, then time the plain step and the
    learned stale step (CUDA graphs) and report the amortised throughput of
    one refresh plus K - 1 learned steps at the largest K whose learned
    drag error is <= 1%."""
    import numpy as np
    import torch

    import synth
    import paper_1807_11834_gb300 as cg
    from paper_1807_11834_gb300 import closure

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    make = getattr(synth, args.workload)
    dt = 1e-4                      # the clustered bed's step; the packed bed is advanced with the same
    t0 = time.time()
    # runs long enough to cover every refresh interval scored below
    F, T = closure.generate_pairs(make, seeds=(0, 1), refreshes=(2, 5, 10, 20, 50), steps=56,
                                  n_pairs=2_000_000, dt=dt)
    t_gen = time.time() - t0
    m, hist = closure.train(F, T, epochs=20, batch=65536, lr=2e-3, activation=args.activation)
    t_train = time.time() - t0 - t_gen
    n_pairs = int(F.shape[0])
    del F, T
    Ks = (5, 10, 20, 50)
    w = make(seed=2)
    evals = {K: closure.evaluate(m, lambda seed: w, seed=2, refresh=K, steps=K + 2, dt=dt) for K in Ks}
    ok = [K for K in Ks if evals[K]["err_learned"] <= 0.01]
    K_star = max(ok) if ok else None

    # the timed state: the held-out run advanced past a refresh, so that the
    # stale record is `age` steps old and the fluid has evolved as in training
    age = 2
    K_t = K_star or 5
    traj = closure.Trajectory.start(w, K_t, dt=dt)
    for _ in range(K_t + age):
        traj.advance()
    g = traj.grids
    n = w.n
    pos, vel, uf, out = traj.pos, traj.vel, traj.u_fine, traj.out
    out["u_bulk"].copy_(traj.u_stale)
    out["var_bulk"].copy_(traj.var_stale)
    stale_u, stale_var = traj.u_stale.clone(), traj.var_stale.clone()
    torch.cuda.synchronize()
    g.cg_sync_status()

    def graph_of(fn):
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        g.set_stream(cs)
        with torch.cuda.stream(cs):
            fn()
        cs.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=cs):
            fn()
        g.set_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        return gr

    # the plain step overwrites out's bulk record: the learned step is timed
    # on its own output set holding the stale record
    out_l = {k: (v.clone() if v is not None else None) for k, v in out.items()}
    out_l["u_bulk"].copy_(stale_u)
    out_l["var_bulk"].copy_(stale_var)
    plain = graph_of(lambda: g.cg_step(pos, vel, uf, out))
    learned = graph_of(lambda: g.cg_step_learned(pos, vel, uf, out_l, m, age))

    def time_graph(gr, steps):
        for _ in range(max(3, args.warmup)):
            gr.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            gr.replay()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    steps = max(20, min(args.steps, 500))
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ta = time.time()
    ms_plain = time_graph(plain, steps)
    g.cg_sync_status()
    ms_learned = time_graph(learned, steps)
    tb = time.time()
    time.sleep(0.2)
    sampler.stop()
    rc, flags, counts = g.cg_sync_status()
    if rc != 0:
        raise RuntimeError(f"timed status {rc}")
    fallback_timed = counts[4] / (n * (steps + max(3, args.warmup)))

    # per-kernel times of the learned step (serialised events)
    g.cg_profile_reset()
    g.cg_profile_enable(True)
    for _ in range(20):
        g.cg_step_learned(pos, vel, uf, out_l, m, age)
    prof = g.cg_profile_read()
    g.cg_profile_enable(False)
    kern = {k: {"ms_per_launch": round(v[1] / v[0], 5)} for k, v in prof.items() if v[0]}
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    roof = None
    if "drag_learned" in kern:
        # network: 2 (16 x 64 + 64 x 64) flops per row on the tensor cores
        flops = 2.0 * (16 * 64 + 64 * 64) * n
        ach = flops / (kern["drag_learned"]["ms_per_launch"] * 1e-3) / 1e12
        pk = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"kernel": "drag_learned", "bound": "tensor", "achieved": round(ach, 2), "peak": pk,
                "unit": "TFLOP/s", "frac": round(ach / pk, 5),
                "peak_source": "measured" if "bf16_tflops" in peaks else "fallback"}
    amort = None
    if K_star:
        ms_amort = (ms_plain + (K_star - 1) * ms_learned) / K_star
        amort = n / (ms_amort * 1e-3)
    line = {"metric": "learned coupled particle-steps/s at <=1% relative drag error",
            "value": amort, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup),
            "higher_is_better": True, "dtype": "f32 (closure bf16 x bf16 -> f32)", "data": "synthetic",
            "config": {"workload": args.workload, "particles": n, "fine_cells": g.n_fine, "bulk_cells": g.n_bulk,
                       "dt": dt, "activation": args.activation, "training_pairs": n_pairs, "train_seeds": [0, 1],
                       "eval_seed": 2,
                       "generate_s": round(t_gen, 1), "train_s": round(t_train, 1)},
            "refresh_K": K_star,
            "plain": {"ms_per_step": round(ms_plain, 5), "value": n / (ms_plain * 1e-3)},
            "learned_step": {"ms_per_step": round(ms_learned, 5), "value": n / (ms_learned * 1e-3),
                             "age": age, "fallback_share": fallback_timed,
                             "state": f"held-out run after {K_t + age} steps, record refreshed {age} steps before"},
            "drag_error": {str(K): evals[K] for K in Ks},
            "loss_standardised": [round(h, 5) for h in (hist[0], hist[-1])],
            "kernels_learned_step": kern, "roofline_closure": roof,
            "clocks": sampler.summary(ta, tb)}
    print(json.dumps(line))
    m.close()
    traj.close()


def run_closure_drag(args):
    """The learned drag kernel alone, for profiling: one plain step of the
    workload (its record is the closure's stale record), a random closure
    (He-style initial weights) whose feature box holds every row, so no row
    falls back, bound with record age 2; then `warmup` untimed and `steps`
    timed launches of cg_drag with the closure, timed with CUDA events on
    the handle's stream (inputs larger than L2).  One JSON line."""
    import numpy as np
    import torch

    import paper_1807_11834_gb300 as cg
    from paper_1807_11834_gb300 import closure

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    w = make_workload(args, 0)
    g = cg.Grids(w.desc)
    n = w.n
    pos = torch.from_numpy(w.pos_d).cuda()
    vel = torch.from_numpy(w.vel).cuda()
    uf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).cuda()
    out = g.alloc_outputs(n, var=True, eps_fine=True)
    g.cg_step(pos, vel, uf, out)
    feat = torch.empty(n, 8, device="cuda")
    tg = torch.empty(n, device="cuda")
    g.cg_mlp_features(pos, vel, out["eps_bulk"], out["u_bulk"], out["var_bulk"], out["u_bulk"], feat, tg)
    lo, hi = closure.feature_box(feat)
    m = cg.Mlp(cg.mlp_pack(closure.init_params(0)), lo - 1, hi + 1, activation=args.activation)
    m.bind(out["var_bulk"], uf, 2)
    F = torch.empty(3, n, device="cuda")
    for _ in range(max(3, args.warmup)):
        g.cg_drag(pos, vel, out["eps_bulk"], out["u_bulk"], F, mlp=m)
    torch.cuda.synchronize()
    steps = max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.cg_drag(pos, vel, out["eps_bulk"], out["u_bulk"], F, mlp=m)
    e1.record()
    e1.synchronize()
    rc, flags, counts = g.cg_sync_status()
    if rc != 0 or m.sync_status()[0] != 0:
        raise RuntimeError(f"learned drag status {rc}")
    ms = e0.elapsed_time(e1) / steps
    print(json.dumps({"metric": "learned drag launches", "ms_per_launch": round(ms, 5), "rows": n,
                      "ns_per_1000_rows": round(ms * 1e6 / n * 1000, 2), "activation": args.activation,
                      "fallbacks": int(counts[4]), "launches": steps + max(3, args.warmup),
                      "config": {"workload": workload_name(args.workload, w)}}))
    m.close()
    g.close()


def run_map(args):
    """Maps between non-nested grids on the packed bed's bulk grid and a fine
    grid of 250 x 250 x 500 cells (3.9 fine cells per bulk cell per axis,
    offset so it covers the bulk grid): the volume-weighted average of three
    components and the conservative projection of three, each timed with
    CUDA events over repeated launches (inputs > L2)."""
    import numpy as np
    import torch
    import paper_1807_11834_gb300 as cg

    bulk = ((0.0, 0.0, 0.0), (1.0, 1.0, 2.0), (64, 64, 128))
    fine = ((-0.004, -0.004, -0.008), (1.008, 1.008, 2.016), (250, 250, 500))
    m = cg.Map(bulk, fine)
    nb_, nf_ = m.n_bulk, m.n_fine
    g = torch.Generator(device="cuda").manual_seed(0)
    u = torch.rand(3, nf_, device="cuda", generator=g)
    ub = torch.empty(3, nb_, device="cuda")
    sb = torch.rand(3, nb_, device="cuda", generator=g)
    sf = torch.empty(3, nf_, device="cuda")
    reps = max(5, min(args.steps, 200))

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_avg = timed(lambda: m.average(u, ub))
    t_prj = timed(lambda: m.project(sb, sf))
    peak, src = load_peaks()
    b_avg = 3 * 4 * nf_ + 3 * 4 * nb_
    b_prj = 3 * 4 * nf_ + 3 * 4 * nb_
    line = {"metric": "non-nested map bytes/s", "unit": "GB/s",
            "config": {"bulk": bulk, "fine": fine, "components": 3, "repetitions": reps,
                       "l2": f"fine fields {3 * 4 * nf_ / 1e6:.0f} MB > L2"},
            "average": {"ms": round(t_avg, 5), "algorithmic_bytes": b_avg,
                        "gbs": round(b_avg / (t_avg * 1e-3) / 1e9, 1),
                        "frac": round(b_avg / (t_avg * 1e-3) / 1e9 / peak, 4)},
            "project": {"ms": round(t_prj, 5), "algorithmic_bytes": b_prj,
                        "gbs": round(b_prj / (t_prj * 1e-3) / 1e9, 1),
                        "frac": round(b_prj / (t_prj * 1e-3) / 1e9 / peak, 4)},
            "peak": peak, "peak_source": src}
    m.close()
    print(json.dumps(line))


def run_batch(args):
    """64 independent uneven instances (fine edge 32..128, ratio 2/4/8, 10^4
    to 2 10^6 particles each, Taylor-Green fluid, Di Felice, FP32): one by
    one (eager, and as one CUDA graph of the 64 cg_step calls) against the
    batched step (default decomposition, then autotuned, eager and as a
    replayed graph).  Value: batched, tuned, graph particle-steps/s."""
    import numpy as np
    import torch

    import synth
    import paper_1807_11834_gb300 as cg

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    ws = synth.uneven_batch(seed=0, count=64)
    n_tot = sum(w.n for w in ws)
    inst = []
    for w in ws:
        g = cg.Grids(w.desc)
        out = g.alloc_outputs(w.n, var=True, eps_fine=True)
        g.close()
        inst.append((w.desc, torch.from_numpy(w.pos_d).cuda(), torch.from_numpy(w.vel).cuda(),
                     torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).cuda(), out))
    b = cg.Batch(inst)
    steps = max(10, min(args.steps, 200))

    def timed(fn, k):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    l0 = sum(b.instance_launch_count(i) for i in range(len(ws)))
    b.step_each()
    launches_each = sum(b.instance_launch_count(i) for i in range(len(ws))) - l0
    res = {}
    res["one_by_one_eager"] = timed(lambda: b.step_each(), max(3, steps // 4))
    b.use_graph(True)
    res["one_by_one_graph"] = timed(lambda: b.step_each(), max(3, steps // 4))
    b.use_graph(False)
    res["batched_default_eager"] = timed(lambda: b.step(), steps)
    cfg, tune_ms = b.tune(reps=5)
    res["batched_tuned_eager"] = timed(lambda: b.step(), steps)
    b.use_graph(True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ta = time.time()
    res["batched_tuned_graph"] = timed(lambda: b.step(), steps)
    tb = time.time()
    time.sleep(0.2)
    sampler.stop()
    rc, flags, counts = b.sync_status()
    if rc != 0:
        raise RuntimeError(f"batched status {rc} {counts}")
    ms = res["batched_tuned_graph"]
    fine = sum(w.u_fine[0].size for w in ws)
    line = {"metric": "batched coupled particle-steps/s (64 uneven instances)", "value": n_tot / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 uneven instances, seed 0", "particles": n_tot, "fine_cells": fine,
                       "tuned": cfg, "tune_median_ms": tune_ms,
                       "launches_per_batched_step": b.launches_per_step(),
                       "launches_one_by_one_per_step": launches_each},
            "ms_per_step_variants": {k: round(v, 4) for k, v in res.items()},
            "speedup_vs_one_by_one_eager": res["one_by_one_eager"] / ms,
            "speedup_vs_one_by_one_graph": res["one_by_one_graph"] / ms,
            "clocks": sampler.summary(ta, tb)}
    print(json.dumps(line))
    b.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.map:
        run_map(args)
    elif args.batch:
        run_batch(args)
    elif args.learned:
        run_learned(args)
    elif args.closure_drag:
        run_closure_drag(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
