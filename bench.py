"""Benchmark: C^H solves/s at relative residual 1e-5 on 128^3 lattice cells.

One step = the whole hot path over one batch: for each of 16 seeded 128^3 cells (TPMS
network and plate lattices, BCC / octet trusses, volume fractions 0.1-0.4), build the sparse
hierarchy, build the Galerkin operators and the coarsest inverse for E = 1, nu = 0.3, solve
the six elasticity cell problems to max_m r_m <= 1e-5 (mixed-precision V-cycle CG) and
reduce C^H. `value` = cells / second with the voxels already on the device; `e2e` repeats
the step through the same public API from pinned host voxels (host->device copy inside the
timed region) and reads each C^H back to the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmt|reference]
                    [--workload c128|c32|c512] [--physics elastic|heat] [--precision fp32|fp64]

Multi-GPU: one process per GPU (torchrun); every rank solves its own 16 cells (weak scaling,
no data-path collective); the timing is the max over ranks. `--impl reference` times the CPU
FP64 oracle (assembled FE system, Jacobi-preconditioned CG, energy-average C^H) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_26518_b300 import lattices  # noqa: E402

C2_FAMILIES = ("gyroid", "schwarz_p", "diamond", "plate_gyroid", "plate_schwarz_p",
               "plate_diamond", "bcc", "octet")
METRIC = "C^H solves/s at rel. residual 1e-5 (128^3, 512^3); V-cycle HBM GB/s vs peak"
TOL = 1e-5
# ncu DRAM bytes (read + write) per active node of the timed level-0 sweep of the current
# kernel: with the default one level-0 sweep per visit that is the V-cycle's last sweep
# (u, f and K p read, u' written, Krylov partials): 197.3 MB over the 651,308 active nodes
# of the first 128^3 bench cell (profiles/k_stencil_smoother_c128_elastic.md); scaled by
# the nodes of each sweep
NCU_DRAM_BYTES_PER_NODE = 302.9


def workload(name: str, rank: int):
    if name == "c128":
        cells = [lattices.mixed_cell(2000 + 16 * rank + i, 128, families=C2_FAMILIES)
                 for i in range(16)]
        desc = "16 seeded 128^3 cells: TPMS network/plate (gyroid, Schwarz-P, diamond), " \
               "BCC/octet trusses, phi 0.1-0.4"
    elif name == "c32":
        cells = [(lattices.tpms_network("gyroid", 32, 0.30), {"family": "gyroid", "n": 32})]
        desc = "gyroid 32^3, phi 0.30"
    elif name == "batch64":
        cells = [lattices.batch_cell(3000 + 64 * rank + i) for i in range(64)]
        desc = "64 seeded cells, N uniform in {32,48,64,96,128}: TPMS network/plate, " \
               "BCC/octet trusses, spinodal; phi 0.1-0.4"
    elif name == "c256":
        cells = [lattices.mixed_cell(2600 + 4 * rank + i, 256, families=C2_FAMILIES)
                 for i in range(4)]
        desc = "4 seeded 256^3 cells: TPMS network/plate (gyroid, Schwarz-P, diamond), " \
               "BCC/octet trusses, phi 0.1-0.4"
    elif name == "c512":
        cells = [(lattices.tpms_network("gyroid", 512, 0.20), {"family": "gyroid", "n": 512})]
        desc = "gyroid 512^3, phi 0.20"
    else:
        raise ValueError(name)
    return cells, desc


# ---------------------------------------------------------------- clocks sampling
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


# ---------------------------------------------------------------- CPU oracle sample
def cpu_sample(n_cells: int = 1, timeout: float = 600.0):
    """Time the oracle on a bounded sample: the batch's first cells regenerated at 32^3
    (same generator and seeds), full solve to r <= 1e-5 and C^H, single thread."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from paper_2604_26518_b300 import lattices\n"
        "from oracle import solve\n"
        "fams = %r\n"
        "cells = [lattices.mixed_cell(2000 + i, 32, families=fams)[0] for i in range(%d)]\n"
        "t = time.perf_counter()\n"
        "for v in cells: solve.solve_cell(v, 'elastic', 1.0, 0.3, tol=%g)\n"
        "print(json.dumps({'seconds': time.perf_counter() - t, 'cells': len(cells)}))\n"
    ) % (ROOT, C2_FAMILIES, n_cells, TOL)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=timeout, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["cells"] / out["seconds"], out


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_sample(1)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, _ = cpu_sample(1)
        rates.append(rate)
    elapsed = time.perf_counter() - t0
    value = float(np.mean(rates))
    sample = ("per step: the batch's first cell (seed 2000) regenerated at 32^3 by the same "
              "generator, CPU FP64 oracle: assembled K, Jacobi-PCG to max_m r_m <= 1e-5, "
              "energy-average C^H (the 128^3 cells exceed the oracle's assembled-matrix memory)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "C^H solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c128 batch, bounded 32^3 sample (see cpu_baseline.sample)",
                   "physics": "elastic", "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "C^H solves/s", "cores": 1,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "C^H solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gmt(args, rank: int, world: int):
    import torch
    import torch.distributed as dist
    from paper_2604_26518_b300 import gmt

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    gmt.lib()
    cells, desc = workload(args.workload, rank)
    ph = gmt.ELASTIC if args.physics == "elastic" else gmt.HEAT
    prec = gmt.FP32 if args.precision == "fp32" else gmt.FP64
    opts = gmt.default_options(precision=prec, coarsest_max=args.coarsest)
    if args.nu:
        opts.nu_pre = opts.nu_post = args.nu
    elif args.workload == "c512":
        # at 512^3 two level-0 sweeps win (2.62 vs 2.49 solves/s: 7 instead of 9 cycles)
        opts.nu_pre = opts.nu_post = 2
    elif ph == gmt.HEAT:
        # scalar conduction: two level-0 sweeps win on the 128^3 batch (522 vs 481 solves/s
        # over 30 steps: 72 instead of 99 cycles)
        opts.nu_pre = opts.nu_post = 2
    if args.nu_post >= 0:
        opts.nu_post = args.nu_post
    if args.inner_tol > 0:
        opts.inner_tol = args.inner_tol
    if args.nu_coarse > 0:
        opts.nu_coarse = args.nu_coarse
    if args.omega > 0:
        opts.omega = args.omega
    if args.smoother:
        opts.smoother = gmt.JACOBI if args.smoother == "jacobi" else gmt.CHEBYSHEV
    if args.cells:
        cells = cells[:args.cells]
    vox_dev = [torch.from_numpy(v).to(dev) for v, _ in cells]
    vox_host = [torch.from_numpy(v).pin_memory() for v, _ in cells]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    cycles_seen = []
    unconverged, fallbacks = [], []   # cell indices, appended by every step
    # Cells are independent: with --streams S > 1, S host threads each solve every S-th cell
    # on a stream of their own, so that one cell's host synchronisations and small coarse-
    # level kernels overlap another cell's work. The step starts and ends on `stream`.
    nstreams = max(1, args.streams)
    wstreams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)] if nstreams > 1 else [stream]
    pool = ThreadPoolExecutor(max_workers=nstreams) if nstreams > 1 else None

    net, learned = None, None
    if args.learned:
        net, learned = train_initializer(args, ph, opts)

    def run_cells(src, idx, s, trace):
        tot, CH, cyc = {}, {}, []
        for i in idx:
            if trace:   # the hierarchy build precedes the library's tracer: events around it
                b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                b0.record(s)
            h = gmt.Hierarchy(src[i], opts, s)
            if trace:
                b1.record(s)
                b1.synchronize()
                a = tot.setdefault("setup_hierarchy", [0, 0.0, 0.0])
                a[0] += 1
                a[1] += b0.elapsed_time(b1)
                h.trace(True)
            u0 = None
            if net is not None:       # the network's field as the warm start (Alg. 2)
                g = gmt.NetGraph(h)
                u0 = net.forward(g, LEARNED_SCALE * h.level_res(0))
                g.free()
            st, _, info = h.solve(ph, E=1.0, nu=0.3, k=1.0, tol=TOL, u0=u0, want_field=False,
                                  allow_not_converged=True)
            if st == gmt.NOT_CONVERGED:
                unconverged.append(i)          # reported; the cell's time stays in the step
            elif st != gmt.OK:
                raise RuntimeError(f"solve status {st}: {info.as_dict()}")
            if info.fp64_fallback:
                fallbacks.append(i)
            CH[i] = h.homogenize(ph, E=1.0, nu=0.3, k=1.0)
            cyc.append((i, info.inner_total))
            if trace:
                tt = h.trace_totals()
                a = tot.setdefault("_smooth_node_launches", [0, 0.0, 0.0])
                a[2] += float(h.num_nodes(0)) * tt["smooth_l0"][0]   # nodes x sweeps
                for k, (n, ms, b) in tt.items():
                    if k == "setup_hierarchy":
                        continue
                    a = tot.setdefault(k, [0, 0.0, 0.0])
                    a[0] += n
                    a[1] += ms
                    a[2] += b
            h.free()
        return tot, CH, cyc

    def one_step(src, trace, serial=False):
        if pool is None or serial:
            parts = [run_cells(src, range(len(src)), stream, trace)]
        else:
            start = torch.cuda.Event()
            start.record(stream)
            for s in wstreams:
                s.wait_event(start)
            futs = [pool.submit(run_cells, src, range(w, len(src), nstreams), wstreams[w], trace)
                    for w in range(nstreams)]
            parts = [f.result() for f in futs]
            for s in wstreams:
                done = torch.cuda.Event()
                done.record(s)
                stream.wait_event(done)
        tot, CH, cyc = {}, {}, []
        for t_, c_, y_ in parts:
            for k, a in t_.items():
                b = tot.setdefault(k, [0, 0.0, 0.0])
                for j in range(3):
                    b[j] += a[j]
            CH.update(c_)
            cyc.extend(y_)
        cycles_seen.extend(c for _, c in sorted(cyc))
        return tot, [CH[i] for i in range(len(src))]

    for _ in range(args.warmup):
        one_step(vox_dev, False)
    # ---- device-resident timed region
    flush.zero_()
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(dev.index) if rank == 0 else None
    launches0 = gmt.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    totals = {}
    step_ms = []
    for s in range(args.steps):
        flush.zero_()                       # L2 flush between timed iterations (not timed)
        torch.cuda.synchronize()
        e0.record(stream)
        one_step(vox_dev, False)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    launches = gmt.launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    # ---- one traced step for the phase split and the roofline: the library brackets every
    # launch with CUDA events on its stream, which would perturb concurrent streams, so this
    # step runs the cells one after another on `stream` (not part of `value`)
    flush.zero_()
    torch.cuda.synchronize()
    tot, _ = one_step(vox_dev, True, serial=True)
    torch.cuda.synchronize()
    for k, a in tot.items():
        t = totals.setdefault(k, [0, 0.0, 0.0])
        for i in range(3):
            t[i] += a[i]
    trace_steps = 1
    barrier()
    elapsed_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    cells_total = len(cells) * world * args.steps
    value = cells_total / (elapsed_ms / 1000.0)
    # ---- e2e through the public API from pinned host voxels
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        one_step(vox_host, False)
    torch.cuda.synchronize()
    e2e_ms = 1000.0 * (time.perf_counter() - t0)
    if world > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = cells_total / (e2e_ms / 1000.0)
    if rank != 0:
        return
    # ---- roofline of the dominant kernel: the level-0 smoother sweep
    n_sm, ms_sm, b_sm = totals.get("smooth_l0", [0, 0.0, 0.0])
    peak, peak_src = measured_peak_gbs()
    achieved = (b_sm / (ms_sm / 1000.0)) / 1e9 if ms_sm > 0 else None
    avg_nodes = totals.pop("_smooth_node_launches", [0, 0.0, 0.0])[2] / max(n_sm, 1)
    # the ncu figure was taken on the FP32 elasticity sweep; other forms report no traffic
    ncu_matches = (ph == gmt.ELASTIC and prec == gmt.FP32)
    traffic = (NCU_DRAM_BYTES_PER_NODE * avg_nodes) \
        if (NCU_DRAM_BYTES_PER_NODE and ncu_matches) else None
    vals = (18 if ph == gmt.ELASTIC else 3)
    esz = 4 if prec == gmt.FP32 else 8
    total_dev_ms = sum(v[1] for v in totals.values())
    line = {
        "metric": METRIC, "value": value, "unit": "C^H solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == gmt.FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "cells_per_step_per_gpu": len(cells),
                   "n": (cells[0][1]["n"] if len({c[1]["n"] for c in cells}) == 1
                         else sorted({c[1]["n"] for c in cells})),
                   "physics": args.physics, "tol": TOL,
                   "precision": ("fp32 V-cycle CG, float-float outer residual, fp64 coarsest "
                                 "solve and C^H accumulation") if prec == gmt.FP32 else "fp64",
                   "step": "hierarchy + operators + solve + C^H per cell",
                   "coarsest_max": args.coarsest,
                   "smoother": "%s, nu_pre %d, nu_post %d" % (
                       {gmt.JACOBI: "jacobi", gmt.CHEBYSHEV: "chebyshev", gmt.GS8: "gs8"}
                       [opts.smoother], opts.nu_pre, opts.nu_post),
                   "inner_tol": opts.inner_tol, "nu_coarse": opts.nu_coarse,
                   "omega": opts.omega,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}",
                   "concurrent_cells": nstreams},
        "e2e": {"value": e2e_value, "unit": "C^H solves/s",
                "h2d_bytes_per_step": int(sum(v.numel() for v in vox_host)),
                "d2h_bytes_per_step": int(len(cells) * (36 if ph == gmt.ELASTIC else 9) * 8)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm",
                     "kernel": "level-0 smoother sweeps (k_stencil JACOBI; with the default one "
                               "sweep per level-0 visit, the V-cycle's last sweep, which also "
                               "writes the Krylov partials)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read + write of the V-cycle's "
                                        "last level-0 sweep on the first 128^3 cell, per "
                                        "active node, times this workload's nodes per sweep")
                                       if traffic is not None else
                                       "not captured for this physics / precision",
                     "peak_source": peak_src,
                     "algorithmic_bytes": "%d values x %d B per active node for each "
                                          "vector: u and f read, u' written, plus K p read "
                                          "in the V-cycle's last sweep (4 vectors, %d B)"
                                          % (vals, esz, 4 * vals * esz),
                     "avg_nodes_per_launch": avg_nodes,
                     "launches": n_sm, "avg_launch_us": 1000.0 * ms_sm / max(n_sm, 1)},
        "phases_ms_per_step": {k: v[1] / trace_steps for k, v in sorted(totals.items())},
        "traced_device_ms_per_step": total_dev_ms / trace_steps,
        "phases_note": "one extra step, cells one after another, every launch bracketed by "
                       "CUDA events on its stream (not part of value)",
        "vcycles_per_cell": cycles_seen[-len(cells):],
        "unconverged_cells": sorted(set(unconverged)),
        "fp64_fallback_cells": sorted(set(fallbacks)),
        "clocks": clocks,
    }
    if learned is not None:
        line["config"]["learned_initializer"] = learned
        line["config"]["step"] = ("hierarchy + network tables + inference + solve from the "
                                  "prediction + C^H per cell")
    if world == 1 and not args.no_cpu:
        try:
            rate, out = cpu_sample(1)
            line["cpu_baseline"] = {
                "value": rate, "unit": "C^H solves/s", "cores": 1, "kind": "oracle",
                "sample": "first cell of the batch (seed 2000) regenerated at 32^3 by the same "
                          "generator; CPU FP64 oracle to r <= 1e-5 + C^H; %.1f s" % out["seconds"]}
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "error": str(exc)[-300:]}
    print(json.dumps(line), flush=True)


LEARNED_SCALE = 0.04   # network output x 0.04 N = field (u / N has a spread of about 0.04)


def train_initializer(args, ph, opts):
    """Train the initializer network (untimed): solve seeded 32^3 cells to r <= 1e-6 with
    this library, then AdamW on the relative energy-norm loss, one cell per step, cosine
    learning rate from 1e-3."""
    import torch

    from paper_2604_26518_b300 import gmt
    t0 = time.perf_counter()
    data = []
    for i in range(args.learned_cells):
        vox, _ = lattices.mixed_cell(100 + i, 32, families=C2_FAMILIES)
        h = gmt.Hierarchy(vox, opts)
        _, u, _ = h.solve(ph, E=1.0, nu=0.3, k=1.0, tol=1e-6)
        data.append((h, gmt.NetGraph(h), u.reshape(h.num_nodes(0), -1).contiguous()))
    cout = data[0][2].shape[1]
    net = gmt.UNet(cout, torch.from_numpy(lattices.unet_init(gmt.unet_layers(cout), seed=0)))
    t1 = time.perf_counter()
    steps = args.learned_epochs * len(data)
    losses, k = [], 0
    for ep in range(args.learned_epochs):
        for i in np.random.default_rng(ep).permutation(len(data)):
            h, g, u = data[i]
            lr = 1e-3 * 0.5 * (1.0 + np.cos(np.pi * k / steps))
            losses.append(net.train_step(g, u, LEARNED_SCALE * 32, lr=lr, weight_decay=1e-4,
                                         loss=gmt.LOSS_ENERGY, hier=h))
            k += 1
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for h, g, _ in data:
        g.free()
        h.free()
    last = losses[-len(data):]
    return net, {"params": net.num_params, "train_cells": len(data), "train_n": 32,
                 "steps": steps, "loss": "relative energy norm of the error, (e^T K e)/(u^T K u)",
                 "first_epoch_loss": float(np.mean(losses[:len(data)])),
                 "last_epoch_loss": float(np.mean(last)),
                 "data_s": t1 - t0, "train_s": t2 - t1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmt", choices=["gmt", "reference"])
    ap.add_argument("--workload", default="c128", choices=["c128", "c32", "c256", "c512", "batch64"])
    ap.add_argument("--physics", default="elastic", choices=["elastic", "heat"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--coarsest", type=int, default=8, help="coarsest grid side bound")
    ap.add_argument("--nu", type=int, default=0, help="pre/post smoothing sweeps (0: default)")
    ap.add_argument("--nu-post", type=int, default=-1, help="post-smoothing sweeps (-1: as --nu)")
    ap.add_argument("--omega", type=float, default=0.0, help="Jacobi damping (0: default)")
    ap.add_argument("--nu-coarse", type=int, default=0,
                    help="smoothing sweeps on levels >= 1 (0: as on level 0)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed precision: true-residual replacement factor (0: default)")
    ap.add_argument("--streams", type=int, default=4,
                    help="cells solved concurrently, one host thread and CUDA stream each")
    ap.add_argument("--smoother", default="", choices=["", "jacobi", "chebyshev"])
    ap.add_argument("--cells", type=int, default=0, help="use only the first K cells (profiling)")
    ap.add_argument("--learned", action="store_true",
                    help="warm-start every solve from the learned initializer, trained first "
                         "(untimed) on seeded 32^3 cells")
    ap.add_argument("--learned-epochs", type=int, default=20)
    ap.add_argument("--learned-cells", type=int, default=64)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (torch.cuda.is_available() and args.impl == "gmt") else "gloo"
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gmt(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
