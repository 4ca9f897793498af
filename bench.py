#!/usr/bin/env python
"""Benchmark of the sharp-interface VOF phase-change hot path on GB300.

One step = reconstruct (interface cells, vertex field, isovalue root search, interface
geometry) + phase-change source (interface-modified least-squares gradient on the band, per-side
gradients, q_l, q_v, mdot, Q, totals) over one synthetic input, through the library's C ABI.

Default workload: the large annular case, learned and batched. An extruded jittered 2D Voronoi
disk of radius 1, 600 layers over length 6 (7,903,200 cells), with a wall liquid film
r > 0.9 - 0.04 sin(2 pi (z - t)/0.5) that moves one layer per step; T falls linearly from
T_sat + 8 K at the wall to T_sat at the interface. 100 consecutive steps' alpha and T are
resident on the device, and step k reads pair k mod 100.

Prints one JSON line. `--impl reference` times the FP64 CPU oracle instead (host cores).
Multi-GPU (torchrun, N > 1): every rank processes its own replica of the workload (replicas;
the units of all ranks are summed and divided by the slowest rank's time).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth.workloads import NAMES as WORKLOADS, workload  # noqa: E402

METRIC = "interface cells/s (recon+LSQ∇T+mdot), learned vs bisection, at |Δα|≤1e-10"
UNIT = "interface cells/s"
FP64_NOMINAL_TFLOPS = 152 * 2.07e9 * 4 / 1e12  # 152 SMs x 2070 MHz x 2 FP64 FMA (4 flops) per clock per SM
L2_FLUSH_BYTES = 256 << 20
RESIDENT_STEPS = 100  # device-resident input pairs of the moving-film workload (default)
# A clipping-based estimate, kept as a secondary basis: about 2 kFLOP per FP64 cut-volume
# evaluation of a Voronoi cell of about 14 faces (36 straddle tests, ~15 cut points, ~90 fan
# tetrahedra at ~20 flops). The roofline's own basis is the FP64-equivalent work the kernel counts
# on the device (pieces prepared and expanded, per-pass scaling).
CLIP_FLOPS_PER_EVAL = 2000
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per root-search launch record (one per
# populated bin and step, as in the roofline's launch count), from ncu captures of the workload
# (and layers), path and lanes per cell given; null for anything else. The pipe's root search was
# captured with the 9-24 tetrahedra bin on the thread-per-cell kernel (k_root_cell and its
# hand-over launch) and 4, 8, 16 or 32 lanes per cell in the 5-8 bin (3 launches per step). At
# 8 lanes: 48.16 and 99.10 MB per step on 100- and 200-layer cuts (48,384 and 96,768 interface
# cells), in proportion to within 3 %; on the 200-layer cut 4, 16 and 32 lanes move 99.16, 99.05
# and 99.08 MB (the 5-8 bin reads 6.75 MB whatever its lanes). The 600-layer case has three times
# the 200-layer cut's interface cells (290,304) and is taken to move three times its bytes.
_PIPE200_STEP_BYTES = {4: 99.16e6, 8: 99.10e6, 16: 99.05e6, 32: 99.08e6}
ROOT_TRAFFIC: dict = {("pipe8m", 100, "learned", (0, 8, 1, 0, 0)): 48.16e6 / 2}
for _g, _b in _PIPE200_STEP_BYTES.items():
    ROOT_TRAFFIC[("pipe8m", 200, "learned", (0, _g, 1, 0, 0))] = _b / 2
    ROOT_TRAFFIC[("pipe8m", 600, "learned", (0, _g, 1, 0, 0))] = 3 * _b / 2
# path name -> (root mode, pseudo-time extrapolation, guess option)
PATHS = {"bisect": (0, 0, 0), "learned": (1, 0, 0), "learned_nomlp": (1, 0, 1), "cubic": (2, 0, 1),
         "learned_extrap": (1, 1, 0)}


class Clocks:
    """nvidia-smi sampling (every 50 ms) kept only inside the marked timed window."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # the sampler is up before the timed window opens
        except OSError:
            self.proc = None
        return self

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _ts(field):
        try:
            return time.mktime(time.strptime(field.split(".")[0], "%Y/%m/%d %H:%M:%S")) + \
                float("0." + field.split(".")[1]) if "." in field else 0.0
        except (ValueError, IndexError):
            return None

    def summary(self):
        rows = [r.split(", ") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        t0, t1 = (self.t0 or 0.0) - 0.05, (self.t1 or 1e30) + 0.05
        inside = [r for r in rows if (lambda t: t is not None and t0 <= t <= t1)(self._ts(r[0]))]
        use = inside or rows
        sm = [float(r[1]) for r in use if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": float(use[0][2]),
                "reasons": reasons, "samples": len(inside),
                "window_s": round((self.t1 or 0) - (self.t0 or 0), 3)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def hbm_peak_gbs(path=os.path.join(ROOT, "MEASURED_PEAKS.json")) -> tuple[float, str]:
    """(HBM copy rate in GB/s, where it comes from): the measured copy rate of the GB300s
    when the peaks file is present, else an earlier GB300 measurement of 6.8 TB/s."""
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, f"measured copy rate (read + write bytes) on this GPU type: {v:.1f} GB/s of measured"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "6800 GB/s of fallback (an earlier GB300 copy measurement)"


def n_interface(a) -> int:
    return int(np.count_nonzero((a > 1e-12) & (a < 1 - 1e-12)))


def bench_config(args, desc, n_cells, a, extra) -> dict:
    """The workload as both arms report it (same dict for the GPU path and the oracle arm)."""
    return {"workload": args.workload, "description": desc, "n_cells": int(n_cells), "n_iface": n_interface(a),
            "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write outside the events)",
            "parallelism": "replicas" if args.gpus > 1 else "single", **extra,
            **({"resident_steps": args.resident} if args.workload == "pipe8m" else {})}


def path_options(vof, name):
    mode, extrap, guess = PATHS[name]
    return vof.default_options(root_mode=mode, extrap=extrap, guess=guess)


def run_ours(args, rank, world, dev):
    import torch
    import paper_2604_14938_gb300 as vof
    import synth

    meshes, a, T, Tb, desc, extra = workload(args.workload, layers=args.layers)
    batch = isinstance(meshes, list)
    if batch:
        B = vof.Batch(meshes)
        M = B.mesh
    else:
        B, M = None, vof.Mesh(meshes)
    nc = M.n_cells
    pipe = args.workload == "pipe8m"
    stream = torch.cuda.Stream(device=dev)
    results = {}
    with torch.cuda.stream(stream):
        d = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
        if pipe:
            # device-resident steps: the film translates one layer (n2d cells) per step
            n2d = nc // extra["layers"]
            ta_k = [d(np.roll(a, k * n2d)) for k in range(args.resident)]
            tT_k = [d(np.roll(T, k * n2d)) for k in range(args.resident)]
            tTb = None
        else:
            ta_k, tT_k, tTb = [d(a)], [d(T)], d(Tb)
        mdot = torch.empty(nc, dtype=torch.float64, device=dev)
        Q = torch.empty_like(mdot)
        tot = torch.empty(2, dtype=torch.float64, device=dev)
        btot = torch.empty((B.n, 2), dtype=torch.float64, device=dev) if batch else None
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        have_mlp = vof.load_default_mlp(M)
        if args.root == "auto":
            modes = ["bisect"] + (["learned", "learned_nomlp"] if have_mlp else []) + ["cubic"] + \
                    (["learned_extrap"] if have_mlp and not args.no_extrap else [])
        else:
            modes = [args.root]
            if args.root in ("learned", "learned_extrap") and not have_mlp:
                raise RuntimeError("the learned path needs the shipped MLP weights (mlp_iso.npy)")
        fp64 = vof.fp64_peak(stream=stream)  # the FP64 roofline's denominator, measured in this run
        tuned = {}
        for mode in modes:
            opt = path_options(vof, mode)

            def one(k):
                ta, tT = ta_k[k % len(ta_k)], tT_k[k % len(tT_k)]
                if pipe:  # a different input pair every step: eager launches
                    M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt, stream=stream)
                else:
                    M.step_graph(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt, stream=stream)
                if batch:
                    B.totals(btot, stream=stream)

            if mode == "learned_extrap" and "learned" in tuned:  # the same root search as the learned path
                tuned[mode] = tuned["learned"]
                M.set_group_sizes(tuned[mode])
            elif args.group_sizes:  # a fixed choice, e.g. one tuned without a profiler's serialised launches
                tuned[mode] = [int(x) for x in args.group_sizes.split(",")]
                M.set_group_sizes(tuned[mode])
            else:
                G0 = M.autotune(ta_k[0], opt, reps=10)  # lanes per cell of each bin, for this mode
                tuned[mode] = step_tune(M, G0, one, flush, stream)

            for k in range(args.warmup):
                one(k)
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            iface = []
            with Clocks(torch.cuda.current_device()) as clk:
                clk.start()
                for k, (s0, e0) in enumerate(ev):
                    flush.fill_(k & 0xFF)  # write > L2 between steps (outside the events)
                    s0.record(stream)
                    one(k)
                    e0.record(stream)
                    if pipe:
                        iface.append(M.counts(stream=stream)["n_iface"])  # after the step's events
                stream.synchronize()
                clk.stop()
            if world > 1:
                torch.distributed.barrier()
            ms = sum(s0.elapsed_time(e0) for s0, e0 in ev)
            cnt = M.counts(stream=stream)
            units = sum(iface) if pipe else cnt["n_iface"] * args.steps
            # one more pass, eager with per-kernel events, for the kernel times of the roofline; the
            # device counters are read after every step (they are reset by the next one)
            M.timing_enable(True)
            ksum = {}
            for k in range(min(args.steps, 5)):
                ta, tT = ta_k[k % len(ta_k)], tT_k[k % len(tT_k)]
                flush.fill_(k & 0xFF)
                M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt, stream=stream)
                c = M.counts(stream=stream)
                for key in ("n_iface", "evals_total", "tet_evals", "tets_prepared", "evals32_total"):
                    ksum[key] = ksum.get(key, 0) + c[key]
            kt = M.timing_read(stream=stream)
            M.timing_enable(False)
            results[mode] = dict(ms=ms, units=units, counts=cnt, ksum=ksum, ktime=kt, clocks=clk.summary(),
                                 mean_iface=units / args.steps)
        # end to end: host buffers through vof_step_host, copies inside the timed region, in the
        # headline mode with its own tuned lanes per cell
        best_mode = headline_mode(results)
        M.set_group_sizes(tuned[best_mode])
        opt_best = path_options(vof, best_mode)
        pin = lambda x: torch.as_tensor(np.ascontiguousarray(x)).pin_memory()
        ha, hT = pin(a), pin(T)
        hTb = None if pipe else pin(Tb)
        hm = torch.empty(nc, dtype=torch.float64).pin_memory()
        ht = torch.empty(2, dtype=torch.float64).pin_memory()
        for _ in range(args.warmup):
            M.step_host(ha, hT, hTb, synth.PROPS, hm, ht, opt_best, stream=stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            M.step_host(ha, hT, hTb, synth.PROPS, hm, ht, opt_best, stream=stream)
        e2e_s = time.perf_counter() - t0
        e2e_units = M.counts(stream=stream)["n_iface"] * args.steps
    # bytes in: alpha and T, and T_bnd at the boundary faces (pinned: the library gathers only
    # those entries from host memory); out: mdot and the totals
    n_bnd = sum(int((np.asarray(mm.face_neigh) < 0).sum()) for mm in (meshes if isinstance(meshes, list) else [meshes]))
    info = dict(n_cells=nc, batch=batch, pipe=pipe, tuned=tuned, extra=extra, e2e_units=e2e_units, fp64=fp64,
                h2d=8 * (2 * nc + (0 if pipe else n_bnd)), d2h=8 * (nc + 2))
    return M, (meshes, a, T, Tb), desc, results, e2e_s, info


def step_tune(M, G0, one, flush, stream, steps=8) -> list:
    """The library's autotuner times reconstructions alone; in the step the crossing-face list and
    the zeroing of mdot and Q run beside them, which can change a small bin's best lanes per cell.
    Starting from its choice, coordinate descent over the populated bins with `steps` whole timed
    steps per candidate (L2 flushed between steps, outside the events) keeps the fastest."""
    import torch

    def cost(G):
        M.set_group_sizes(G)
        one(0)  # a graph path captures its graph here
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k, (s0, e0) in enumerate(ev):
            flush.fill_(k & 0xFF)
            s0.record(stream)
            one(k)
            e0.record(stream)
        stream.synchronize()
        return sum(s0.elapsed_time(e0) for s0, e0 in ev)

    best = coordinate_descent(G0, cost)
    M.set_group_sizes(best)
    return best


def coordinate_descent(G0, cost) -> list:
    """Lanes per cell of the populated bins (G0[b] != 0), one bin at a time in bin order: each of
    1, 2, 4, 8, 16, 32 is tried with the other bins at their current best, and the cheapest kept.
    Empty bins stay 0."""
    best, best_t = list(G0), cost(list(G0))
    for b in [b for b in range(len(G0)) if G0[b]]:
        g_start = best[b]  # measured already, with the other bins as they are now
        for G in (1, 2, 4, 8, 16, 32):
            if G == g_start:
                continue
            cand = list(best)
            cand[b] = G
            t = cost(cand)
            if t < best_t:
                best, best_t = cand, t
    return best


def headline_mode(results) -> str:
    """The path the headline value reports: learned when it ran, else bisection, the interval
    cubic, the learned path without its network, or the learned path with the pseudo-time
    extrapolation."""
    return next(k for k in ("learned", "bisect", "cubic", "learned_nomlp", "learned_extrap") if k in results)


def job_rate(units: float, seconds: float, device=None) -> tuple[float, float]:
    """(whole-job rate, slowest rank's seconds): the units of every rank summed and divided by the
    largest time over the ranks; one process without a process group is its own job."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / seconds, seconds
    t = torch.tensor([float(units), float(seconds)], dtype=torch.float64, device=device)
    u = t[:1].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    s = t[1:].clone()
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(s.item()), float(s.item())


def _oracle_step(O, a, T, Tb, cells):
    """One oracle pass: (seconds of the whole-mesh parts, seconds of the sampled reconstruction).
    The whole-mesh parts are the vertex field and the downstream steps (selection, band, crossing
    faces, least squares and source for every interface cell); the reconstruction (FP64
    bisection and geometry, OpenMP over cells) runs on `cells`."""
    import synth
    t0 = time.perf_counter()
    phi = O.vertex_field(a)
    t1 = time.perf_counter()
    rec = O.reconstruct(a, phi, cells=cells)
    t2 = time.perf_counter()
    O.phase_change(a, rec, T, Tb, synth.PROPS)
    t3 = time.perf_counter()
    return (t1 - t0) + (t3 - t2), t2 - t1


def _sample_note(tf, tr, n, n_all, reps, cores):
    return (f"vertex field and downstream steps over the whole mesh, one thread ({tf:.2f} s per pass); FP64 "
            f"bisection reconstruction (OpenMP, {cores} threads) of {n} of {n_all} interface cells (index-order "
            f"prefix, {tr:.2f} s per pass) scaled to all of them; {reps} passes")


def _oracle_sample(O, a, T, Tb, I, step_budget_s):
    """Index-order prefix of the interface cells whose reconstruction takes about step_budget_s
    minus the whole-mesh parts (at least 256 cells). Returns (n, whole-mesh seconds, seconds of
    the sampled reconstruction) of the last sizing pass."""
    n = min(len(I), 256)
    while True:
        fixed, rec = _oracle_step(O, a, T, Tb, I[:n])
        want = max(step_budget_s - fixed, 0.25)
        if n >= len(I) or rec > 0.6 * want:
            return n, fixed, rec
        n = min(len(I), int(n * min(8.0, max(1.5, want / max(rec, 1e-3)))))


def cpu_baseline(m, a, T, Tb, budget_s=12.0):
    """The oracle as it stands on the host cores, timed with perf_counter to about budget_s
    seconds of work: the whole-mesh parts in full, the reconstruction on an index-order prefix
    sample of the interface cells, scaled to all of them."""
    import oracle

    O = oracle.Oracle(m)
    O.geometry()  # mesh geometry is set-up work, as on the GPU
    I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0]
    n, fixed, rec = _oracle_sample(O, a, T, Tb, I, budget_s / 3)
    reps = max(1, int(budget_s / max(fixed + rec, 1e-3)) - 1)
    tf = tr = 0.0
    for _ in range(reps):
        f, r = _oracle_step(O, a, T, Tb, I[:n])
        tf += f / reps
        tr += r / reps
    whole = tf + tr * len(I) / max(n, 1)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(value=len(I) / whole, unit=UNIT, cores=cores, kind="oracle", cpu=cpu_model(),
                sample=_sample_note(tf, tr, n, len(I), reps, cores))


def reference_arm(args):
    """The oracle on the host cores as the reference arm: each step one oracle pass over a
    bounded sample of the workload (whole-mesh parts in full, the reconstruction on a prefix of
    the interface cells, scaled to all of them), sized so that warm-up and timed steps together
    take about three minutes."""
    m, a, T, Tb, desc, extra = workload(args.workload, layers=args.layers)
    if isinstance(m, list):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline covers single-mesh workloads"}))
        return
    import oracle
    if args.workload == "pipe8m":
        Tb = None  # the moving-film steps leave the boundary faces out of the stencil, as the GPU arm does
    O = oracle.Oracle(m)
    O.geometry()
    I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0]
    n, _, _ = _oracle_sample(O, a, T, Tb, I, 180.0 / (args.warmup + args.steps))
    tf, tr = [], []
    for k in range(args.warmup + args.steps):
        f, r = _oracle_step(O, a, T, Tb, I[:n])
        if k >= args.warmup:
            tf.append(f)
            tr.append(r)
    # one step = the whole workload: the sampled reconstruction scaled to every interface cell
    step_s = (sum(tf) + sum(tr) * len(I) / max(n, 1)) / len(tf)
    v = len(I) / step_s
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cb = dict(value=v, unit=UNIT, cores=cores, kind="oracle", cpu=cpu_model(),
              sample=_sample_note(sum(tf) / len(tf), sum(tr) / len(tr), n, len(I), len(tf), cores))
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": bench_config(args, desc, m.n_cells, a, extra),
                      "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                  "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pipe8m", choices=list(WORKLOADS))
    ap.add_argument("--layers", type=int, default=600,
                    help="layers of the pipe workload (600: the full case; fewer: a smaller case for profiling)")
    ap.add_argument("--resident", type=int, default=RESIDENT_STEPS,
                    help="device-resident input pairs of the pipe workload (fewer: a smaller device footprint for "
                         "profiling)")
    ap.add_argument("--root", default="auto", choices=["auto"] + list(PATHS),
                    help="auto: every path, the learned one as the headline; otherwise that path alone")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extrap", action="store_true", help="auto without the pseudo-time extrapolation path")
    ap.add_argument("--group-sizes", default="",
                    help="lanes per cell of the five tetrahedron-count bins, comma-separated (skips the autotuner)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    M, fields, desc, res, e2e_s, info = run_ours(args, rank, world, dev)
    best = headline_mode(res)
    r = res[best]
    value, s_max = job_rate(r["units"], r["ms"] / 1e3, dev)
    ms_max = s_max * 1e3
    paths = {k: job_rate(v["units"], v["ms"] / 1e3, dev) for k, v in res.items()}
    e2e_value, _ = job_rate(info["e2e_units"], e2e_s, dev)
    # roofline of the root search: the FP64 work the kernel counts on the device over the eager
    # timing pass, over the summed durations of its launches (one per non-empty bin and step; the
    # bins run as parallel branches), against the FP64 rate measured in this run
    kt, ks = r["ktime"], r["ksum"]
    nst = max(kt["select"][1], 1)
    root_ms, root_launches = kt["root"]
    counted = M.root_flops(ks)
    clip = CLIP_FLOPS_PER_EVAL * ks["evals_total"]
    peak = info["fp64"]["tflops"]
    achieved = counted / (root_ms / 1e3) / 1e12 if root_ms and counted else None
    clip_tf = clip / (root_ms / 1e3) / 1e12 if root_ms and clip else None
    ktot = sum(v[0] for v in kt.values())
    share = {k: round(v[0] / max(ktot, 1e-30), 4) for k, v in kt.items() if v[1]}
    # the root search launches once per non-empty bin; a bin of at most 24 tetrahedra per cell
    # with one lane per cell (learned or cubic mode) launches the thread-per-cell kernel and then
    # the lane-group kernel on the cells it handed over
    cell_kernel = PATHS[best][0] != 0
    nbins = sum((2 if (cell_kernel and b <= 2 and info["tuned"][best][b] == 1) else 1)
                for b, c in enumerate(M.bin_cells) if c)
    mlp_used = best in ("learned", "learned_extrap")
    # selection, crossing list, crossing points, least squares, source, geometry; root search per
    # bin; MLP features and forward; the pseudo-time extrapolation; batch totals
    per_step = (6 + nbins + (2 if mlp_used else 0) + (1 if best == "learned_extrap" else 0)
                + (1 if info["batch"] else 0))
    traffic = ROOT_TRAFFIC.get((args.workload, args.layers, best, tuple(info["tuned"][best])))
    hbm_peak, hbm_src = hbm_peak_gbs()
    root_gbs = traffic / (root_ms / max(root_launches, 1) / 1e3) / 1e9 if traffic and root_ms else None
    config = bench_config(args, desc, info["n_cells"], fields[1], info["extra"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": config,
        "path": {"root": best, "group_sizes_by_bin": info["tuned"][best], "n_iface_mean": r["mean_iface"],
                 "step": ("eager launches per step (a different resident input pair every step)" if info["pipe"]
                          else "CUDA graph replay")},
        "paths": {k: {"value": paths[k][0], "ms_per_step": paths[k][1] * 1e3 / args.steps,
                      "evals_per_cell": v["counts"]["evals_total"] / max(v["counts"]["n_iface"], 1),
                      "fp32_evals_per_cell": v["counts"]["evals32_total"] / max(v["counts"]["n_iface"], 1),
                      "fallbacks": v["counts"]["n_fallback"], "not_converged": v["counts"]["n_not_converged"],
                      "mlp_skipped": v["counts"]["n_mlp_skipped"], "group_sizes_by_bin": info["tuned"][k],
                      "kernel_ms_per_step": {kk: vv[0] / max(v["ktime"]["select"][1], 1)
                                             for kk, vv in v["ktime"].items() if vv[1]},
                      **({"extrap_iters": v["counts"]["extrap_iters"]} if k == "learned_extrap" else {})}
                  for k, v in res.items()},
        "kernel_ms_per_step": {k: v[0] / nst for k, v in kt.items() if v[1]},
        "kernel_share": share,
        "roofline": {"kernel": "k_root (isovalue root search)", "bound": "alu",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the root-search "
                                        "launches per launch record, captured on 100- and 200-layer cuts of the pipe "
                                        "in this lane choice and scaled by interface cells" if traffic else
                                        "no ncu capture of this workload, path and lane choice"),
                     "flops_per_launch": counted / max(root_launches, 1),
                     "flops_per_iface_cell": counted / max(ks["n_iface"], 1),
                     "launches": root_launches, "ms_per_launch": root_ms / max(root_launches, 1),
                     "flops_basis": "FP64-equivalent work counted on the device: 8 flops per tetrahedron row "
                                    "evaluation or piece expanded, 24 per row or piece prepared, 2 per pass (summed "
                                    "over the eager timing pass); the thread-per-cell kernel does this work in "
                                    "FP32-pair arithmetic, and its FP32 refinement is not counted",
                     "peak_source": (f"FP64 FMA-chain probe in this run (vof_probe_fp64_fma: 8 independent chains per "
                                     f"thread, every SM at full occupancy, best of 3): {peak:.4f} TFLOP/s of measured; "
                                     f"nominal 152 SMs x 2070 MHz x 4 flop/clk = {FP64_NOMINAL_TFLOPS:.4f}"),
                     "hbm": {"achieved": root_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": root_gbs / hbm_peak if root_gbs else None, "peak_source": hbm_src,
                             "note": "the root search's DRAM bytes per launch record over its mean launch time: "
                                     "context beside the binding FP64 figure"},
                     "clip_estimate": {"flops_per_eval": CLIP_FLOPS_PER_EVAL, "achieved": clip_tf,
                                       "frac": clip_tf / peak if clip_tf else None,
                                       "note": "a clipping-based 2 kFLOP per FP64 cut-volume evaluation of a ~14-face "
                                               "cell x the evaluations made; it credits the interval pass's saving, "
                                               "so it can exceed the peak on small cells"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": info["h2d"],
                "d2h_bytes_per_step": info["d2h"]},
        "gpu_launches": args.steps * per_step,
        "clocks": r["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not info["batch"]:
        line["cpu_baseline"] = cpu_baseline(fields[0], fields[1], fields[2], None if info["pipe"] else fields[3])
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
