#!/usr/bin/env python
"""Benchmark of the sharp-interface VOF phase-change hot path on GB300.

One step = reconstruct (interface cells, vertex field, isovalue root search, interface
geometry) + phase-change source (interface-modified least-squares gradient on the band, per-side
gradients, q_l, q_v, mdot, Q, totals) over one synthetic input, through the library's C ABI.

Default workload: jittered-BCC Voronoi mesh, 2 * 50^3 = 250,000 cells on the unit cube (seed 1,
jitter +-h/4), wavy liquid film z < 0.3 + 0.03 sin(2 pi x) sin(2 pi y), T linear across the film
from T_sat + 10 K at the wall to T_sat at the interface, water/steam properties.

Prints one JSON line. `--impl reference` times the FP64 CPU oracle instead (host cores).
Multi-GPU (torchrun, N > 1): every rank processes its own replica of the workload (replicas;
the units of all ranks are summed and divided by the slowest rank's time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "interface cells/s (recon+LSQ∇T+mdot), learned vs bisection, at |Δα|≤1e-10"
UNIT = "interface cells/s"
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12  # 152 SMs x 2070 MHz x 2 FP64 FMA (4 flops) per clock per SM
L2_FLUSH_BYTES = 256 << 20
# library kernels per step: begin, 3 interface selection, 3 band/vertex lists, vertex field,
# root search, least squares, source, totals
KERNELS_PER_STEP = 12


def workload(name: str):
    import synth
    if name == "film250k":
        m = synth.voronoi_bcc(50, jitter=0.25, seed=1)
        reg = dict(type="film", z0=0.3, a=0.03)
        a = synth.alpha(m, reg, mode="subtet", level=3)
        T, Tb = synth.temperature(m, reg, dict(kind="film", dT=10.0))
        desc = "jittered-BCC Voronoi 2x50^3=250k cells (seed 1, +-h/4), wavy film z<0.3+0.03sin(2pi x)sin(2pi y)"
    elif name == "sphere32":
        m = synth.hex_box(32)
        reg = dict(type="spheres", spheres=[(0.5, 0.5, 0.5, 0.25)])
        a = synth.alpha(m, reg, mode="hexgrid", level=3)
        T, Tb = synth.temperature(m, reg, dict(kind="radial", dT=5.0))
        desc = "hex 32^3 unit cube, vapour sphere R=0.25 at the centre, alpha from 8^3 samples"
    else:
        raise SystemExit(f"unknown workload {name}")
    return m, a, T, Tb, desc


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [r.split(", ") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def run_ours(args, rank, world, dev):
    import torch
    import paper_2604_14938_gb300 as vof
    import synth

    m, a, T, Tb, desc = workload(args.workload)
    M = vof.Mesh(m)
    d = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    ta, tT, tTb = d(a), d(T), d(Tb)
    mdot = torch.empty(m.n_cells, dtype=torch.float64, device=dev)
    Q = torch.empty_like(mdot)
    tot = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    learned_ok = False
    if args.root in ("auto", "learned"):
        learned_ok = hasattr(vof, "load_default_mlp") and vof.load_default_mlp(M)
    modes = ["bisect"] + (["learned"] if learned_ok else [])
    results = {}
    for mode in modes:
        opt = vof.default_options(root_mode=vof.ROOT_LEARNED if mode == "learned" else vof.ROOT_BISECT)
        for _ in range(args.warmup):
            M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        M.timing_enable(True)
        with Clocks(torch.cuda.current_device()) as clk:
            for s, e in ev:
                flush.fill_(s.__hash__() & 0xFF)  # write > L2 between steps (outside the events)
                s.record(stream)
                M.step(ta, tT, tTb, synth.PROPS, mdot, Q, tot, opt)
                e.record(stream)
            torch.cuda.synchronize()
        kt = M.timing_read()
        M.timing_enable(False)
        if world > 1:
            torch.distributed.barrier()
        ms = sum(s.elapsed_time(e) for s, e in ev)
        cnt = M.counts()
        results[mode] = dict(ms=ms, counts=cnt, ktime=kt, clocks=clk.summary())
    # end to end: host buffers through the host-buffer ABI call, copies inside the timed region
    opt_best = vof.default_options(root_mode=vof.ROOT_LEARNED if "learned" in results else vof.ROOT_BISECT)
    pin = lambda x: torch.as_tensor(np.ascontiguousarray(x)).pin_memory()
    ha, hT, hTb = pin(a), pin(T), pin(Tb)
    hm = torch.empty(m.n_cells, dtype=torch.float64).pin_memory()
    ht = torch.empty(2, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        M.step_host(ha, hT, hTb, synth.PROPS, hm, ht, opt_best)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        M.step_host(ha, hT, hTb, synth.PROPS, hm, ht, opt_best)
    e2e_s = time.perf_counter() - t0
    return m, (a, T, Tb), desc, results, e2e_s, M


def cpu_baseline(m, a, T, Tb, budget_s=12.0):
    """The oracle as it stands on the host cores: vertex field + bisection reconstruction on a
    prefix sample of the interface cells + the downstream steps, timed with perf_counter."""
    import oracle
    import synth

    O = oracle.Oracle(m)
    O.geometry()  # mesh geometry is set-up work, as on the GPU
    I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0]
    n = min(len(I), 256)
    while True:
        t0 = time.perf_counter()
        phi = O.vertex_field(a)
        rec = O.reconstruct(a, phi, cells=I[:n])
        O.phase_change(a, rec, T, Tb, synth.PROPS)
        dt = time.perf_counter() - t0
        if n >= len(I) or dt > budget_s / 3:
            break
        n = min(len(I), int(n * max(2.0, budget_s / 3 / max(dt, 1e-3))))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(value=n / dt, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{n} of {len(I)} interface cells (index-order prefix) reconstructed by FP64 bisection, "
                       f"vertex field and downstream steps over the whole mesh; {dt:.2f} s"), n, dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="film250k")
    ap.add_argument("--root", default="auto", choices=["auto", "bisect", "learned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        if rank != 0:
            return
        m, a, T, Tb, desc = workload(args.workload)
        times, units = [], []
        base, n, dt = cpu_baseline(m, a, T, Tb, budget_s=6.0)
        import oracle
        import synth
        O = oracle.Oracle(m)
        I = np.where((a > 1e-12) & (a < 1 - 1e-12))[0][:n]
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            phi = O.vertex_field(a)
            rec = O.reconstruct(a, phi, cells=I)
            O.phase_change(a, rec, T, Tb, synth.PROPS)
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
        v = n * len(times) / sum(times)
        cb = dict(base, value=v)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": args.workload, "description": desc},
                          "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                      "d2h_bytes_per_step": 0}}))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, fields, desc, res, e2e_s, M = run_ours(args, rank, world, dev)
    best = "learned" if "learned" in res else "bisect"
    r = res[best]
    n_iface = r["counts"]["n_iface"]
    ms = r["ms"]
    ms_max = ms
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(t.item())
    value = world * n_iface * args.steps / (ms_max / 1e3)
    # roofline of the dominant kernel (root search + geometry): algorithmic FP64 flops per launch
    root_ms, root_n = r["ktime"]["root"]
    c = r["counts"]
    flops = M.root_flops(c)  # counters hold the last step, i.e. one launch of the root kernel
    achieved = flops / (root_ms / root_n / 1e3) / 1e12 if root_n and flops else None
    share = {k: round(v[0] / max(sum(x[0] for x in r["ktime"].values()), 1e-30), 4) for k, v in r["ktime"].items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n_cells": m.n_cells, "n_iface": n_iface,
                   "root": best, "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "paths": {k: {"value": world * v["counts"]["n_iface"] * args.steps / (v["ms"] / 1e3),
                      "ms_per_step": v["ms"] / args.steps,
                      "evals_per_cell": v["counts"]["evals_total"] / max(v["counts"]["n_iface"], 1),
                      "fallbacks": v["counts"]["n_fallback"], "not_converged": v["counts"]["n_not_converged"]}
                  for k, v in res.items()},
        "kernel_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in r["ktime"].items() if v[1]},
        "kernel_share": share,
        "roofline": {"kernel": "k_root (isovalue root search + interface geometry)", "bound": "alu",
                     "flops_per_launch": flops, "flops_per_iface_cell": flops / max(n_iface, 1),
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                     "peak_source": "FP64: 152 SMs x 2070 MHz x 4 flop/clk/SM (2 FMA), no FP64 figure in the measured peaks"},
        "e2e": {"value": world * n_iface * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 8 * (2 * m.n_cells + m.n_faces), "d2h_bytes_per_step": 8 * (m.n_cells + 2)},
        "gpu_launches": args.steps * (KERNELS_PER_STEP + (1 if best == "learned" else 0)),
        "clocks": r["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, _, _ = cpu_baseline(m, *fields)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
