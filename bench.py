"""Benchmark: C^H solves/s at relative residual 1e-5 on 128^3 lattice cells.

One step = the whole hot path over one batch: for each of 16 seeded 128^3 cells (TPMS
network and plate lattices, BCC / octet trusses, volume fractions 0.1-0.4), build the sparse
hierarchy, build the Galerkin operators and the coarsest inverse for E = 1, nu = 0.3, solve
the six elasticity cell problems to max_m r_m <= 1e-5 (mixed-precision V-cycle CG) and
reduce C^H. `value` = cells / second with the voxels already on the device; `e2e` repeats
the step through the same public API from pinned host voxels (host->device copy inside the
timed region) and reads each C^H back to the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmt|reference]
                    [--workload c128|c32|c256|c512|batch64] [--physics elastic|heat]
                    [--precision fp32|fp64] [--smoother jacobi|chebyshev|gs8] [--cycle V|W|F]

Before the warm-up the smoothing schedule (nu_pre = nu_post, nu_coarse, coarse_fp16) is
tuned on the workload itself (--no-autotune keeps the fixed one): one timed step per
candidate for a batch of cells, gmt_autotune (one solve per candidate) for a single cell;
the choice and every candidate's time are in config.autotune.

The default (c128) line also carries the 512^3 gyroid as a keyed sub-result (value_512,
ms_per_solve_512, vcycles_512), the V-cycle roofline (roofline.vcycle: algorithmic bytes of
every V-cycle over the traced V-cycle kernel time) and per-kernel rooflines.

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
import threading
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
# ncu DRAM bytes (read + write) per active node and launch, from one capture of each
# kernel on the first 128^3 bench cell (FP32 elasticity). A
# kernel whose source changed after its capture has no entry (its traffic is reported as
# null until it is captured again).
NCU_DRAM_BYTES_PER_NODE = {
    # level-1 damped-Jacobi sweep over the 88,670 level-1 nodes of the first bench cell,
    # keyed by (category, coarse_fp16): stored FP32 per-node stencils (k_stencil KIND 1):
    # 116.9 MB read + 3.1 MB written; their FP16 copy (KIND 2): 69.0 MB + 1.6 MB
    ("stencil_l1", 0): (116.924672e6 + 3.106304e6) / 88670,
    ("stencil_l1", 1): (68.956672e6 + 1.588480e6) / 88670,
}


class _CellQueue:
    """Cell indices handed out one at a time to the worker threads."""

    def __init__(self, items):
        self._it = iter(items)
        self._lock = threading.Lock()

    def __iter__(self):
        return self

    def __next__(self):
        with self._lock:
            return next(self._it)


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
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_ORACLE_CHILD = (
    "import sys, time, json; sys.path.insert(0, %r)\n"
    "from paper_2604_26518_b300 import lattices\n"
    "from oracle import solve\n"
    "cells = [lattices.mixed_cell(s, %d, families=%r)[0] for s in %r]\n"
    "t = time.perf_counter()\n"
    "nodes = 0\n"
    "for v in cells:\n"
    "    r = solve.solve_cell(v, 'elastic', 1.0, 0.3, tol=%g)\n"
    "    nodes += r['level'].num_nodes\n"
    "print(json.dumps({'seconds': time.perf_counter() - t, 'cells': len(cells), 'nodes': nodes}))\n"
)


def cpu_sample(seeds, n: int = 32, procs: int = 1, timeout: float = 900.0):
    """Time the FP64 oracle (assembled K, Jacobi-PCG to max_m r_m <= tol, energy-average
    C^H) on the bench generator's cells `seeds` regenerated at n^3. The cells are split
    over `procs` single-threaded processes that run at the same time (cells are
    independent); the rate is cells over the wall time of the slowest process (cell
    generation excluded)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    seeds = list(seeds)
    groups = [seeds[p::procs] for p in range(procs) if seeds[p::procs]]
    ps = [subprocess.Popen([sys.executable, "-c", _ORACLE_CHILD % (ROOT, n, C2_FAMILIES, g, TOL)],
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
          for g in groups]
    outs = []
    for p in ps:
        o, e = p.communicate(timeout=timeout)
        if p.returncode != 0:
            raise RuntimeError(e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    wall = max(o["seconds"] for o in outs)
    cells = sum(o["cells"] for o in outs)
    return cells / wall, {"seconds": wall, "cells": cells, "procs": len(groups),
                          "nodes": sum(o["nodes"] for o in outs)}


# ---------------------------------------------------------------- reference arm
def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def from_rank0(obj, world: int):
    """Rank 0's obj on every rank (a choice all ranks must share)."""
    if world <= 1:
        return obj
    import torch.distributed as dist
    box = [obj]
    dist.broadcast_object_list(box, src=0)
    return box[0]


def run_reference(args, rank: int, world: int):
    """The CPU FP64 oracle on the bench's 16 cells, regenerated at 32^3 (the 128^3 cells
    need an assembled matrix of ~8 GB and hours of Jacobi-PCG per cell), spread over the
    host's cores (one single-threaded process per cell, at most one per core)."""
    if rank != 0:
        return
    cores = host_cores()
    procs = max(1, min(cores, 16))
    seeds = range(2000, 2016)
    for _ in range(args.warmup):
        cpu_sample(seeds[:procs], 32, procs)
    rates, nodes = [], 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, out = cpu_sample(seeds, 32, procs)
        rates.append(rate)
        nodes = out["nodes"]
    elapsed = time.perf_counter() - t0
    value = float(np.mean(rates))
    sample = ("per step: the c128 batch's 16 cells (seeds 2000-2015) regenerated at 32^3 by the "
              "same generator, %d single-threaded processes on %d host cores; CPU FP64 oracle: "
              "assembled K, Jacobi-PCG to max_m r_m <= 1e-5, energy-average C^H; %d active "
              "nodes over the 16 cells (a 128^3 cell of the batch has about 50x more)" % (procs, cores, nodes))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "C^H solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c128 batch regenerated at 32^3 (bounded sample, see "
                               "cpu_baseline.sample)", "physics": "elastic", "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "C^H solves/s", "cores": procs,
                         "host_cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "C^H solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_block():
    """The oracle as it stands on bounded samples of the bench workload: 1 thread and all
    host cores on 32^3 regenerations of the batch's cells, and 1 thread on the batch's first
    cell at 64^3."""
    cores = host_cores()
    procs = max(1, min(cores, 16))
    r1, o1 = cpu_sample([2000], 32, 1)
    ra, oa = cpu_sample(range(2000, 2000 + procs), 32, procs)
    r64, o64 = cpu_sample([2000], 64, 1)
    return {
        "value": ra, "unit": "C^H solves/s", "cores": procs, "host_cores": cores,
        "kind": "oracle",
        "sample": ("batch cells 2000-%d regenerated at 32^3, one single-threaded process per "
                   "cell on %d cores, CPU FP64 oracle to r <= 1e-5 + C^H; %.1f s wall"
                   % (2000 + procs - 1, procs, oa["seconds"])),
        "one_thread": {"value": r1, "unit": "C^H solves/s", "cores": 1,
                       "sample": "batch cell 2000 at 32^3; %.1f s; %d active nodes"
                                 % (o1["seconds"], o1["nodes"])},
        "c64": {"value": r64, "unit": "C^H solves/s", "cores": 1,
                "sample": "batch cell 2000 (Schwarz-P network) at 64^3, 1 thread; %.1f s; %d "
                          "active nodes" % (o64["seconds"], o64["nodes"])},
    }


def vcycle_bytes(nodes, C: int, b: int, nu_pre: int, nu_post: int, nu_coarse: int) -> float:
    """Algorithmic HBM bytes of one V-cycle with the damped-Jacobi smoother, vectors only,
    each read or written once: on level l (n_l active nodes, C values of b bytes), the first
    pre-smoothing step from zero reads f and writes u (2), every further sweep reads u and f
    and writes u (3), the residual + restriction reads u and f and writes f_{l+1}
    (2 n_l + n_{l+1}), the prolongation + correction reads u_{l+1} and reads and writes u
    (2 n_l + n_{l+1}); the coarsest solve gathers f and scatters u (2 n_L)."""
    tot = 0.0
    L = len(nodes)
    for l in range(L - 1):
        pre = nu_pre if (l == 0 or nu_coarse == 0) else nu_coarse
        post = nu_post if (l == 0 or nu_coarse == 0) else nu_coarse
        n, nc = nodes[l], nodes[l + 1]
        tot += C * b * (n * (2 + 3 * max(pre - 1, 0) + 2 + 2 + 3 * post) + 2 * nc)
    tot += C * b * 2 * nodes[L - 1]
    return tot


VCYCLE_CATS = ("diag_l0", "smooth_l0", "resid_l0", "stencil_l1", "stencil_l2up", "restrict",
               "prolong", "coarse_solve")


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
    prec = {"fp32": gmt.FP32, "fp64": gmt.FP64, "bf16": gmt.BF16}[args.precision]
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
        opts.smoother = {"jacobi": gmt.JACOBI, "chebyshev": gmt.CHEBYSHEV,
                         "gs8": gmt.GS8}[args.smoother]
    if args.cycle:
        opts.cycle = {"V": gmt.CYCLE_V, "W": gmt.CYCLE_W, "F": gmt.CYCLE_F}[args.cycle]
    if args.coarse_fp16:
        opts.coarse_fp16 = 1
    opts.warm_sweeps = args.warm_sweeps
    tuned = None
    if args.autotune and len(cells) == 1:
        # one cell fills the GPU alone: gmt_autotune's solve time is the throughput (untimed)
        h = gmt.Hierarchy(cells[0][0], opts)
        best, times = h.autotune(ph, tol=TOL)
        h.free()
        choice = from_rank0({f: getattr(best, f) for f in TUNED}, world)   # rank 0's choice
        for f in TUNED:
            setattr(opts, f, choice[f])
        tuned = {"by": "gmt_autotune on the cell (one solve per candidate)",
                 "times_ms": [round(float(t), 3) for t in times],
                 "chosen": {f: getattr(best, f) for f in TUNED}}
    if args.cells:
        cells = cells[:args.cells]
    vals = 18 if ph == gmt.ELASTIC else 3        # values per node (components x cases)
    esz = {gmt.FP32: 4, gmt.FP64: 8, gmt.BF16: 2}[prec]   # bytes per V-cycle vector value
    vox_dev = [torch.from_numpy(v).to(dev) for v, _ in cells]
    vox_host = [torch.from_numpy(v).pin_memory() for v, _ in cells]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    cycles_seen = []
    unconverged, fallbacks = [], []   # cell indices, appended by every step
    # Cells are independent: with --streams S > 1, S host threads take cells from a shared
    # queue (largest first) and solve each on the thread's own stream, so that one cell's
    # host synchronisations and small coarse-level kernels overlap another cell's work. The
    # step starts and ends on `stream`.
    nstreams = max(1, args.streams)
    wstreams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)] if nstreams > 1 else [stream]
    pool = ThreadPoolExecutor(max_workers=nstreams) if nstreams > 1 else None

    net, learned = None, None
    if args.learned:
        if args.batched:
            raise SystemExit("--learned runs per-cell solves (no --batched)")
        net, learned = train_initializer(args, ph, opts)
        if args.learned_tc:
            net.tensor_cores(True)
            learned["inference"] = "tcgen05, FP16 operands, FP32 accumulation in tensor memory"

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
                if trace == 1:
                    a = tot.setdefault("setup_hierarchy", [0, 0.0, 0.0])
                    a[0] += 1
                    a[1] += b0.elapsed_time(b1)
                h.trace(True, brackets_only=(trace == 2))
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
                nodes = [h.num_nodes(l) for l in range(h.levels)]
                a = tot.setdefault("_vcycle", [0, 0.0, 0.0])
                a[0] += info.inner_total
                a[2] += info.inner_total * vcycle_bytes(nodes, vals, esz, opts.nu_pre,
                                                        opts.nu_post, opts.nu_coarse)
                for l in range(len(nodes)):
                    a = tot.setdefault("_nodes_l%d" % l, [0, 0.0, 0.0])
                    a[0] += 1
                    a[2] += nodes[l]
                for k, (n, ms, b) in tt.items():
                    if k == "setup_hierarchy" or (trace == 2 and k != "vcycle"):
                        continue
                    a = tot.setdefault(k, [0, 0.0, 0.0])
                    a[0] += n
                    a[1] += ms
                    a[2] += b
            h.free()
        return tot, CH, cyc

    # --batched: the cells of a step are split into `nstreams` groups, each solved by one
    # gmt_solve_batch call from a worker thread (the V-cycles of a group's cells as shared
    # batched launches; the groups overlap like the per-cell streams do); every cell has a
    # stream of its own for its hierarchy and the per-cell solver work
    cstreams = [torch.cuda.Stream(device=dev) for _ in cells] if args.batched else []

    def run_group(src, idx):
        hs = [gmt.Hierarchy(src[i], opts, cstreams[i]) for i in idx]
        CH, cyc = {}, []
        for j0 in range(0, len(hs), gmt.BATCH_MAX):
            res = gmt.solve_batch(hs[j0:j0 + gmt.BATCH_MAX], ph, E=1.0, nu=0.3, k=1.0, tol=TOL,
                                  want_fields=False, allow_not_converged=True)
            for j, (st, _, info) in enumerate(res):
                i = idx[j0 + j]
                if st == gmt.NOT_CONVERGED:
                    unconverged.append(i)
                elif st != gmt.OK:
                    raise RuntimeError(f"solve status {st}: {info.as_dict()}")
                if info.fp64_fallback:
                    fallbacks.append(i)
                cyc.append((i, info.inner_total))
        for i, h in zip(idx, hs):
            CH[i] = h.homogenize(ph, E=1.0, nu=0.3, k=1.0)
            h.free()
        return CH, cyc

    def batched_step(src):
        start = torch.cuda.Event()
        start.record(stream)
        for s in cstreams:
            s.wait_event(start)
        groups = [list(range(w, len(src), nstreams)) for w in range(nstreams)]
        parts = (list(pool.map(lambda g: run_group(src, g), groups)) if pool
                 else [run_group(src, groups[0])])
        for s in cstreams:
            done = torch.cuda.Event()
            done.record(s)
            stream.wait_event(done)
        CH, cyc = {}, []
        for c_, y_ in parts:
            CH.update(c_)
            cyc.extend(y_)
        cycles_seen.extend(c for _, c in sorted(cyc))
        return {}, [CH[i] for i in range(len(src))]

    def one_step(src, trace, serial=False):
        if args.batched and not trace:
            return batched_step(src)
        if pool is None or serial:
            parts = [run_cells(src, range(len(src)), stream, trace)]
        else:
            start = torch.cuda.Event()
            start.record(stream)
            for s in wstreams:
                s.wait_event(start)
            # a shared queue, largest cells first: a worker held up by a slow cell leaves
            # the remaining cells to the others
            q = _CellQueue(sorted(range(len(src)), key=lambda i: -src[i].numel()))
            futs = [pool.submit(run_cells, src, q, wstreams[w], trace) for w in range(nstreams)]
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

    if args.autotune and len(cells) > 1:
        # several cells in flight: a schedule's solve time alone is not the batch's
        # throughput (a second sweep that saves V-cycles on one cell can cost the batch),
        # so every candidate times one whole step (after an untimed one); untimed region
        cands = [(a, b, c) for a in (1, 2) for b in (1, 2, 3) for c in (0, 1)]
        times = []

        def timed_step():
            # one untimed step, then the faster of two timed ones (a single step's time
            # scatters by a few percent, as much as the candidates differ)
            one_step(vox_dev, False)
            best = float("inf")
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                one_step(vox_dev, False)
                torch.cuda.synchronize()
                best = min(best, 1000.0 * (time.perf_counter() - t0))
            return best
        for a, b, c in cands:
            opts.nu_pre = opts.nu_post = a
            opts.nu_coarse = b
            opts.coarse_fp16 = c
            times.append(timed_step())
        a, b, c = cands[min(range(len(cands)), key=lambda i: times[i])]
        opts.nu_pre = opts.nu_post = a
        opts.nu_coarse = b
        opts.coarse_fp16 = c
        # then the chosen schedule with the finer replacement threshold (fewer true-residual
        # replacements: faster on cells that converge in a few cycles, slower on slow ones)
        itol = opts.inner_tol
        if prec != gmt.FP64 and itol > FINE_INNER_TOL:
            opts.inner_tol = FINE_INNER_TOL
            times.append(timed_step())
            if times[-1] < min(times[:-1]):
                itol = FINE_INNER_TOL
        a, b, c, itol = from_rank0((a, b, c, itol), world)   # every rank runs rank 0's choice
        opts.nu_pre = opts.nu_post = a
        opts.nu_coarse = b
        opts.coarse_fp16 = c
        opts.inner_tol = itol
        tuned = {"by": "the faster of two timed steps of the workload per candidate "
                       "(nu_pre = nu_post in {1, 2} x nu_coarse in {1, 2, 3} x coarse_fp16 in "
                       "{0, 1}, then the fastest of those with inner_tol %g)" % FINE_INNER_TOL,
                 "times_ms": [round(t, 2) for t in times],
                 "chosen": {f: getattr(opts, f) for f in TUNED}}
        cycles_seen.clear()
        unconverged.clear()
        fallbacks.clear()
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
    tot, _ = one_step(vox_dev, 1, serial=True)
    torch.cuda.synchronize()
    for k, a in tot.items():
        t = totals.setdefault(k, [0, 0.0, 0.0])
        for i in range(3):
            t[i] += a[i]
    trace_steps = 1
    # ---- and one with only an event pair around each whole V-cycle (no per-launch events
    # inside the cycles): the V-cycle time the roofline divides by
    flush.zero_()
    torch.cuda.synchronize()
    brk, _ = one_step(vox_dev, 2, serial=True)
    torch.cuda.synchronize()
    barrier()
    elapsed_ms = max_over_ranks(sum(step_ms), world, dev)
    cells_total = len(cells) * world * args.steps
    value = cells_total / (elapsed_ms / 1000.0)
    # ---- e2e through the public API from pinned host voxels
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        one_step(vox_host, False)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1000.0 * (time.perf_counter() - t0), world, dev)
    e2e_value = cells_total / (e2e_ms / 1000.0)
    if rank != 0:
        return
    # ---- rooflines from the traced step: per kernel category, the whole V-cycle, and the
    # dominant V-cycle kernel (the category with the most device time)
    peak, peak_src = measured_peak_gbs()
    avg_nodes = totals.pop("_smooth_node_launches", [0, 0.0, 0.0])[2] / \
        max(totals.get("smooth_l0", [1])[0], 1)
    vc = totals.pop("_vcycle", [0, 0.0, 0.0])
    level_nodes = {}
    for k in [k for k in totals if k.startswith("_nodes_l")]:
        a = totals.pop(k)
        level_nodes[int(k[len("_nodes_l"):])] = a[2] / max(a[0], 1)
    kernels = {}
    for k, (n, ms, b) in totals.items():
        if ms > 0 and b > 0 and k in VCYCLE_CATS + ("apply_l0", "outer_resid", "vector"):
            gbs = b / (ms / 1000.0) / 1e9
            kernels[k] = {"launches": n, "ms": ms, "avg_launch_us": 1000.0 * ms / max(n, 1),
                          "achieved_gbs": gbs, "frac": gbs / peak}
    vc_ms_kernels = sum(totals.get(k, [0, 0.0, 0.0])[1] for k in VCYCLE_CATS)
    vbr = brk.get("vcycle", [0, 0.0, 0.0])
    vc_b = brk.get("_vcycle", [0, 0.0, 0.0])
    vc_ms = vbr[1]
    vc_gbs = (vc_b[2] / (vc_ms / 1000.0) / 1e9) if vc_ms > 0 else None
    totals.pop("vcycle", None)
    dom = max((k for k in VCYCLE_CATS if k in kernels), key=lambda k: kernels[k]["ms"],
              default=None)
    dom_n, dom_ms, dom_b = totals.get(dom, [0, 0.0, 0.0]) if dom else (0, 0.0, 0.0)
    dom_gbs = (dom_b / (dom_ms / 1000.0) / 1e9) if dom_ms > 0 else None
    ncu = NCU_DRAM_BYTES_PER_NODE.get((dom, opts.coarse_fp16)) \
        if (ph == gmt.ELASTIC and prec == gmt.FP32) else None
    dom_nodes = avg_nodes if dom in ("smooth_l0", "resid_l0", "diag_l0") else \
        level_nodes.get(1) if dom == "stencil_l1" else None
    traffic = ncu * dom_nodes if (ncu is not None and dom_nodes) else None
    total_dev_ms = sum(v[1] for v in totals.values())
    vcycle_line = {
        "achieved": vc_gbs, "peak": peak, "unit": "GB/s",
        "frac": (vc_gbs / peak) if vc_gbs else None,
        "vcycles": vc_b[0], "vcycle_ms": vc_ms, "algorithmic_bytes": vc_b[2],
        "timing": "one CUDA event pair around each whole V-cycle (cells one after another on "
                  "one stream, no per-launch events inside); the per-launch traced sum of the "
                  "V-cycle kernels is kernels_ms",
        "kernels_ms": vc_ms_kernels,
        "kernels_achieved": (vc[2] / (vc_ms_kernels / 1000.0) / 1e9) if vc_ms_kernels > 0 else None,
        "formula": ("sum over cells of V-cycles x sum over levels l < L-1 of C b [n_l (2 + "
                    "3 (nu_pre_l - 1) + 2 + 2 + 3 nu_post_l) + 2 n_(l+1)] + C b 2 n_(L-1) "
                    "(vectors only, each read/written once: first smoothing step from zero, "
                    "further sweeps, residual + restriction, prolongation + correction, "
                    "coarsest gather/scatter), C = %d values, b = %d B, nu = %d/%d on level 0 "
                    "and %d on coarser levels; divided by the summed device time of the "
                    "V-cycles (kernels: %s)" % (vals, esz, opts.nu_pre, opts.nu_post,
                                                opts.nu_coarse, ", ".join(VCYCLE_CATS))),
        "level_nodes_mean": level_nodes,
    }
    line = {
        "metric": METRIC, "value": value, "unit": "C^H solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == gmt.FP64 else "f32",     # arithmetic (BF16 is storage)
        "data": "synthetic",
        "config": {"workload": desc, "cells_per_step_per_gpu": len(cells),
                   "n": (cells[0][1]["n"] if len({c[1]["n"] for c in cells}) == 1
                         else sorted({c[1]["n"] for c in cells})),
                   "physics": args.physics, "tol": TOL,
                   "precision": {gmt.FP32: "fp32 V-cycle CG, float-float outer residual, fp64 "
                                           "coarsest solve and C^H accumulation",
                                 gmt.BF16: "bf16 V-cycle vectors (fp32 arithmetic), fp32 CG, "
                                           "float-float outer residual, fp64 coarsest solve "
                                           "and C^H accumulation",
                                 gmt.FP64: "fp64"}[prec],
                   "step": "hierarchy + operators + solve + C^H per cell",
                   "coarsest_max": args.coarsest,
                   "smoother": "%s, nu_pre %d, nu_post %d" % (
                       {gmt.JACOBI: "jacobi", gmt.CHEBYSHEV: "chebyshev", gmt.GS8: "gs8"}
                       [opts.smoother], opts.nu_pre, opts.nu_post),
                   "cycle": "VWF"[opts.cycle],
                   "inner_tol": opts.inner_tol, "nu_coarse": opts.nu_coarse,
                   "omega": opts.omega, "coarse_fp16": opts.coarse_fp16,
                   "warm_sweeps": opts.warm_sweeps,
                   "autotune": tuned,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}",
                   "concurrent_cells": nstreams,
                   "solve": ("gmt_solve_batch: the cells' V-cycles as shared batched launches"
                             if args.batched else "gmt_solve per cell")},
        "e2e": {"value": e2e_value, "unit": "C^H solves/s",
                "h2d_bytes_per_step": int(sum(v.numel() for v in vox_host)),
                "d2h_bytes_per_step": int(len(cells) * (36 if ph == gmt.ELASTIC else 9) * 8)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": dom,
                     "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                     "frac": (dom_gbs / peak) if dom_gbs else None, "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read + write per active node of "
                                        "this category's Jacobi-sweep launch on the first "
                                        "128^3 bench cell, times this workload's mean nodes "
                                        "of the level") if traffic else
                                       "no ncu capture of the current kernel for this physics "
                                       "/ precision",
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes": "per launch: the vectors the kernel must read and "
                                          "write, %d values x %d B per active node each, "
                                          "counted once" % (vals, esz),
                     "launches": dom_n, "avg_launch_us": 1000.0 * dom_ms / max(dom_n, 1),
                     "vcycle": vcycle_line, "kernels": kernels},
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
    if world == 1 and args.with_512 and args.workload == "c128":
        line.update(run_512(args, gmt, ph, prec))
    if world == 1 and not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline_block()
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "error": str(exc)[-300:]}
    print(json.dumps(line), flush=True)


def run_512(args, gmt, ph, prec):
    """The 512^3 gyroid (phi 0.20) as a keyed sub-result of the default line: hierarchy +
    operators + solve to r <= 1e-5 + C^H per solve, voxels resident on the device, CUDA
    events around each solve, L2 flushed before each."""
    import torch
    vox = torch.from_numpy(lattices.tpms_network("gyroid", 512, 0.20)).cuda()
    opts = gmt.default_options(precision=prec, coarsest_max=args.coarsest)
    opts.nu_pre = opts.nu_post = 2       # the fixed schedule (--no-autotune)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    tuned = None
    if args.autotune:   # untimed: one solve of the cell per candidate schedule
        h = gmt.Hierarchy(vox, opts, stream)
        best, times = h.autotune(ph, tol=TOL)
        h.free()
        for f in TUNED:
            setattr(opts, f, getattr(best, f))
        tuned = {"by": "gmt_autotune on the cell (one solve per candidate)",
                 "times_ms": [round(float(t), 3) for t in times],
                 "chosen": {f: getattr(best, f) for f in TUNED}}

    def once():
        h = gmt.Hierarchy(vox, opts, stream)
        st, _, info = h.solve(ph, E=1.0, nu=0.3, k=1.0, tol=TOL, want_field=False,
                              allow_not_converged=True)
        C = h.homogenize(ph, E=1.0, nu=0.3, k=1.0)
        h.free()
        return st, info, C

    for _ in range(max(1, min(args.warmup, 2))):
        once()
    ms, cyc, sts = [], [], []
    for _ in range(args.steps_512):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info, C = once()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        cyc.append(info.inner_total)
        sts.append(int(st))
    mean = float(np.mean(ms))
    del vox, flush
    torch.cuda.empty_cache()
    gmt.release_cached_memory()
    return {"value_512": 1000.0 / mean, "ms_per_solve_512": mean, "vcycles_512": cyc[-1],
            "config_512": {"workload": "gyroid 512^3, phi 0.20, elasticity" if ph == gmt.ELASTIC
                           else "gyroid 512^3, phi 0.20, heat conduction",
                           "solves": len(ms), "nu_pre": opts.nu_pre, "nu_post": opts.nu_post,
                           "nu_coarse": opts.nu_coarse, "coarse_fp16": opts.coarse_fp16,
                           "autotune": tuned, "status": sts, "ms_each": ms,
                           "step": "hierarchy + operators + solve + C^H"}}


TUNED = ("nu_pre", "nu_post", "nu_coarse", "coarse_fp16", "inner_tol")   # --autotune picks
FINE_INNER_TOL = 0.003   # the finer true-residual replacement threshold the tuners try last
LEARNED_SCALE = 0.04   # network output x 0.04 N = field (u / N has a spread of about 0.04)


def train_initializer(args, ph, opts):
    """Train the initializer network (untimed): solve seeded cells of side --learned-n
    (32^3 by default) to r <= 1e-6 with this library, then AdamW on the relative energy-norm
    loss, one cell per step, cosine learning rate from 1e-3."""
    import torch

    from paper_2604_26518_b300 import gmt
    t0 = time.perf_counter()
    data = []
    for i in range(args.learned_cells):
        vox, _ = lattices.mixed_cell(100 + i, args.learned_n, families=C2_FAMILIES)
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
            losses.append(net.train_step(g, u, LEARNED_SCALE * args.learned_n, lr=lr,
                                         weight_decay=1e-4,
                                         loss=gmt.LOSS_ENERGY, hier=h))
            k += 1
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for h, g, _ in data:
        g.free()
        h.free()
    last = losses[-len(data):]
    return net, {"params": net.num_params, "train_cells": len(data), "train_n": args.learned_n,
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
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"],
                    help="inner V-cycle precision (bf16: BF16 vectors, FP32 arithmetic)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-512", dest="with_512", action="store_false",
                    help="skip the 512^3 gyroid sub-result of the c128 line")
    ap.add_argument("--steps-512", type=int, default=3, help="timed 512^3 solves")
    ap.add_argument("--coarsest", type=int, default=8, help="coarsest grid side bound")
    ap.add_argument("--nu", type=int, default=0, help="pre/post smoothing sweeps (0: default)")
    ap.add_argument("--nu-post", type=int, default=-1, help="post-smoothing sweeps (-1: as --nu)")
    ap.add_argument("--omega", type=float, default=0.0, help="Jacobi damping (0: default)")
    ap.add_argument("--nu-coarse", type=int, default=0,
                    help="smoothing sweeps on levels >= 1 (0: as on level 0)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed precision: true-residual replacement factor (0: default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the fixed smoothing schedule (by default it is tuned on the "
                         "workload before the warm-up: one timed step per candidate for a "
                         "batch, gmt_autotune for a single cell and for the 512^3 sub-result)")
    ap.add_argument("--coarse-fp16", action="store_true",
                    help="FP16 copies of the coarse levels' stored stencils")
    ap.add_argument("--batched", action="store_true",
                    help="solve the cells of a step together (gmt_solve_batch)")
    ap.add_argument("--streams", type=int, default=8,
                    help="cells solved concurrently, one host thread and CUDA stream each "
                         "(with the tuned schedule, C^H solves/s on the 128^3 batch: 4: 99.0, "
                         "6: 100.5 / 101.7, 8: 101.7 / 101.9, 12: 97.9)")
    ap.add_argument("--smoother", default="", choices=["", "jacobi", "chebyshev", "gs8"])
    ap.add_argument("--cycle", default="", choices=["", "V", "W", "F"])
    ap.add_argument("--cells", type=int, default=0, help="use only the first K cells (profiling)")
    ap.add_argument("--learned", action="store_true",
                    help="warm-start every solve from the learned initializer, trained first "
                         "(untimed) on seeded 32^3 cells")
    ap.add_argument("--warm-sweeps", type=int, default=0,
                    help="damped-Jacobi sweeps on a warm start before the iteration")
    ap.add_argument("--learned-tc", action="store_true",
                    help="network inference on the tensor cores (FP16 operands, tcgen05)")
    ap.add_argument("--learned-epochs", type=int, default=20)
    ap.add_argument("--learned-cells", type=int, default=64)
    ap.add_argument("--learned-n", type=int, default=32, choices=[32, 64],
                    help="side of the training cells")
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
