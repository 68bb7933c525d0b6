#!/usr/bin/env python
"""Throughput of the WLS-ENO hot path: cell-stage updates per second.

Workload: 2-D Burgers u_t + (u^2/2)_x + (u^2/2)_y = 0 on the periodic unit
square, 256 x 256 squares split into 131,072 jittered triangles (vertex
jitter U(-0.2h, 0.2h), seed 1), cubic WLS-ENO reconstruction (p = 4, m = 10)
on the 2-ring stencil (37 cells), Lax-Friedrichs flux with 2 Gauss points per
edge, TVD-RK3 at CFL 0.3 with the time step recomputed every step on the
device, initial data 0.5 + sin(2 pi (x + y)).  One step = one TVD-RK3 step
(three stages) over all cells; value = cells x 3 x steps / device time.
The headline is the FP32-bulk path; the plain FP64 GPU path runs the same
steps from the same state for the speedup and the accuracy comparison.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(N > 1 under torch.distributed.run: independent replicas, one per GPU).
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

from paper_1602_02694_gb300 import synth  # noqa: E402
from paper_1602_02694_gb300.replicas import max_over_ranks, sum_over_ranks  # noqa: E402

METRIC = "cell-stage updates/sec (WLS-ENO recon+flux) vs plain FP64 GPU, equal accuracy"
UNIT = "cell-stage updates/s"
WORKLOAD = ("2-D Burgers, periodic 256x256 jittered triangulated grid (131,072 cells), "
            "p=4 (m=10), 2-ring stencil (37 cells), LF flux, TVD-RK3 CFL 0.3")
N_SIDE, P_ORDER, RING, CFL, JITTER, SEED = 256, 4, 2.0, 0.3, 0.2, 1
FP32_PEAK_LANES_PER_SM = 128   # FP32 FMA lanes per SM (Blackwell)
N_SMS = 152
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (nominal)
# DRAM bytes (read + write) of one launch of the main reconstruction kernel
# on this workload, by (precision, moments mode), from an ncu capture of the
# same kernel (profiles/recon_tpc_*_burgers256_p4.md); None where no capture
# of the current kernel exists.
TRAFFIC_PER_LAUNCH = {("fp32_bulk", 0): 244.78e6 + 4.41e6, ("fp32_bulk", 1): 93.38e6 + 2.62e6,
                      ("fp64", 0): None}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000,
                    help="timed steps (default 1000: ~0.3 s, so that the 200 ms clock samples fall inside)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="wlseno", choices=["wlseno", "reference"])
    ap.add_argument("--n", type=int, default=N_SIDE, help="squares per side (default 256)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU work of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", default="auto",
                    help="reconstruction kernel shape 'lanes,rows' (1,0 = thread per cell); "
                         "default: the autotuner picks the shape and the moments mode")
    ap.add_argument("--moments", type=int, default=0, choices=[0, 1],
                    help="with a fixed --shape 1,0: FP32 moment rows stored (0) or formed on the fly (1)")
    return ap.parse_args()


def algorithmic_flops_per_cell(n, m, npts):
    """Floating-point work one cell's reconstruction needs by the algorithm
    (weights, W A, column scaling, m Householder steps with recomputed
    trailing norms on the n x (m+1) system, triangular solve, evaluation at
    the facet points); padding lanes are not counted."""
    f = 6 * n                       # differences, squares, eps h^2, divide
    f += n * m + 3 * n * m          # W A; column norms and scaling
    for k in range(m):
        rows = n - k
        cols = m - k
        f += 2 * rows * cols        # trailing column norms
        f += 4 * rows * cols        # reflector applied to the other columns and rhs
        f += 3 * rows               # reflector
    f += m * m                      # back substitution
    f += npts * (2 * m + 8)         # monomials and dot product per facet point
    return f


def algorithmic_bytes_per_cell(n, m, npts, dim, a_bytes, on_the_fly=False):
    """Bytes one cell's reconstruction must move at least once: its stencil
    rows of A (formed on the fly: each row's offset instead, and the cell's
    own central moments of degree >= 2), its stencil indices, its own state,
    h, facet neighbours and points, and its facet values."""
    rows = n * dim * 4 + (m - 1 - dim) * 4 if on_the_fly else n * m * a_bytes
    return rows + 4 * n + 8 + 8 + 4 * (dim + 1) + npts * dim * a_bytes + 8 * npts


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None, cmd=None):
        self.rows = []
        self.times = []
        self.proc = None
        self.gpu_id = gpu_id
        self.cmd = cmd
        self.window = None

    def start(self):
        cmd = self.cmd or ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                           "-lms", "200"]
        if self.gpu_id and not self.cmd:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)
                self.times.append(time.time())

    def mark(self, t_begin, t_end):
        """The wall-clock span of the timed region: stop() keeps the samples
        read within it (plus one sampling interval), when there are any."""
        self.window = (t_begin, t_end + 0.2)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        rows = self.rows
        inside = rows
        if self.window:
            inside = [r for r, t in zip(self.rows, self.times) if self.window[0] <= t <= self.window[1]]
            if inside:
                rows = inside
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "samples_in_timed_region": len(inside) if self.window else None}


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample
# ----------------------------------------------------------------------------

PATCH, PATCH_PAD = 20, 6  # timed squares per side; margin beyond the stencils' reach


def patch_submesh(mesh, i0, j0, patch=PATCH, pad=PATCH_PAD):
    """The squares [i0 - pad, i0 + patch + pad) x [j0 - pad, j0 + patch + pad)
    of the "/"-split grid as a mesh of their own (same vertices, renumbered;
    transmissive).  The patch cells' stencils (2-ring), their facet
    neighbours' stencils and all their moments and facet fluxes lie inside the
    margin, so the oracle computes for them exactly what it computes on the
    whole mesh.  Returns (submesh, local indices of the patch cells, local
    cell -> global cell)."""
    n = mesh.n
    cells, glob = [], []
    for j in range(j0 - pad, j0 + patch + pad):
        for i in range(i0 - pad, i0 + patch + pad):
            for t in (0, 1):
                g = 2 * ((j % n) * n + (i % n)) + t
                glob.append(g)
                cells.append(mesh.cells[g])
    cells = np.array(cells)
    verts, inv = np.unique(cells.ravel(), return_inverse=True)
    # unwrap the sub-mesh's vertices into one copy (the patch is away from the
    # periodic seam in the bench mesh, but keep it general)
    coords = mesh.cell_coords[glob]  # [c][v][d]
    vx = np.empty((len(verts), 2))
    vx[inv] = coords.reshape(-1, 2)
    sub = synth.Mesh(vx, inv.reshape(cells.shape).astype(np.int64), np.zeros(2), coords, n=0)
    local = [((j - j0 + pad) * (patch + 2 * pad) + (i - i0 + pad)) * 2 + t
             for j in range(j0, j0 + patch) for i in range(i0, i0 + patch) for t in (0, 1)]
    return sub, local, np.array(glob)


class _PatchSweep:
    """RK stages of the oracle on one patch, advanced a given number of
    cell-stages at a time.  A sweep is one stage: the facet neighbours outside
    the patch are reconstructed when it begins, then the patch cells in
    order; each facet's LF flux is integrated as soon as both of its cells
    are reconstructed, and the patch is updated when the sweep ends, so any
    split of a sweep into steps does exactly one stage's work.  The moment
    matrices are built before any timing (the GPU path precomputes them
    too)."""

    def __init__(self, mesh, u0, i0, j0, patch=None, pad=None):
        from oracle import wlseno_oracle as O
        self.O = O
        sub, cells, glob = patch_submesh(mesh, i0, j0, patch=PATCH if patch is None else patch,
                                         pad=PATCH_PAD if pad is None else pad)
        self.prob = prob = O.Problem(sub.vertices, sub.cells, sub.period, p=P_ORDER, ring=RING, pde=O.BURGERS)
        self.cells = list(cells)
        cellset = set(cells)
        need = set(cells)
        for c in cells:
            need.update(prob.face_nbrs[c])
        self.halo = sorted(need - cellset)
        self.facets_of = {}
        for c in cells:
            fs = []
            for f in range(3):
                c2, f2 = prob.sib[c, f]
                fs.append((c, f, int(c2)) if (c2 < 0 or c < c2) else (int(c2), int(f2), c))
            self.facets_of[c] = fs
        self.cellset = cellset
        for c in need:
            prob.A(c)
        self.u = np.array(u0, dtype=np.float64)[glob]
        self.dt = 1e-5
        self.cursor = 0

    def advance(self, k):
        """k cell-stages (reconstruction, flux share and update of k patch
        cells, continuing the current sweep and starting new ones)."""
        prob, O = self.prob, self.O
        for _ in range(k):
            if self.cursor == 0:
                self.coeffs = {h: prob.reconstruct_cell(self.u, h)[0] for h in self.halo}
                self.acc = {c: 0.0 for c in self.cells}
            c = self.cells[self.cursor]
            self.coeffs[c] = prob.reconstruct_cell(self.u, c)[0]
            for L, fL, R in self.facets_of[c]:
                other = R if L == c else L
                if other >= 0 and other not in self.coeffs:
                    continue
                g = O.facet_flux(prob, self.coeffs, L, fL, R)
                if L in self.cellset:
                    self.acc[L] += g
                if R in self.cellset:
                    self.acc[R] -= g
            self.cursor += 1
            if self.cursor == len(self.cells):
                for c2 in self.cells:
                    self.u[c2] -= self.dt * self.acc[c2] / prob.geo.volume[c2]
                self.cursor = 0


def _oracle_patch_worker(task):
    """One process on one patch.  Without a step count: whole stages until
    `seconds` have passed.  With one: one untimed stage to size the steps,
    `warmup` untimed steps, then `steps` timed steps of k cell-stages each,
    k chosen so that the timed steps take about `seconds`.  Returns
    (cell-stage updates timed, elapsed, k)."""
    mesh, u0, i0, j0, seconds, warmup, steps = task
    sweep = _PatchSweep(mesh, u0, i0, j0)
    n = len(sweep.cells)
    if steps is None:
        done = 0
        t0 = time.perf_counter()
        while True:
            sweep.advance(n)
            done += n
            if time.perf_counter() - t0 >= seconds:
                break
        return done, time.perf_counter() - t0, n
    t0 = time.perf_counter()
    sweep.advance(n)
    per_cell = (time.perf_counter() - t0) / n
    k = max(1, int(round(seconds / (steps * per_cell))))
    for _ in range(warmup):
        sweep.advance(k)
    t0 = time.perf_counter()
    for _ in range(steps):
        sweep.advance(k)
    return k * steps, time.perf_counter() - t0, k


def host_cores():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_cpu_rate(mesh, u0, seconds, workers=1, warmup=0, steps=None):
    """Oracle cell-stage updates/s on 20x20-square patches of the workload's
    mesh (800 cells each), one process per host core used (patches spread
    over the mesh; processes started with spawn, after the GPU work); with
    `steps`, each process runs `warmup` untimed and `steps` timed steps of
    a fixed number of cell-stages.  Returns (rate, description, cores)."""
    n = mesh.n
    starts = [((n // 2 - PATCH // 2) + 37 * w) % n for w in range(workers)]
    tasks = [(mesh, u0, s, (s + 11 * w) % n, seconds, warmup, steps) for w, s in enumerate(starts)]
    if workers == 1:
        results = [_oracle_patch_worker(tasks[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            results = pool.map(_oracle_patch_worker, tasks)
    rate = sum(d / el for d, el, _ in results)
    cells = 2 * PATCH * PATCH
    stages = sum(d for d, _, _ in results) / cells
    head = (f"oracle (numpy/scipy, FP64) in {workers} process(es), one per core, each on a "
            f"{PATCH}x{PATCH}-square patch ({cells} cells, their facet neighbours reconstructed at the "
            f"start of every stage) of the same mesh; ")
    if steps is None:
        body = f"repeated whole RK stages, {stages:.0f} patch-stages in {seconds:.0f} s; "
    else:
        ks = sorted({k for _, _, k in results})
        body = (f"after one untimed sizing stage and {warmup} untimed warm-up steps, {steps} timed steps of "
                f"{'/'.join(str(k) for k in ks)} cell-stages per process ({stages:.1f} patch-stages in all, "
                f"{max(el for _, el, _ in results):.1f} s); ")
    desc = head + body + "moments built before timing; rate summed over the concurrent processes"
    return rate, desc, workers


# ----------------------------------------------------------------------------
# GPU measurement
# ----------------------------------------------------------------------------

def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def make_context(precision, mesh, dev_index, shape="auto", moments=0):
    from paper_1602_02694_gb300.wlseno import Context
    ctx = Context(dev_index, pde="burgers", precision=precision)
    lanes, rows = (0, 0) if shape == "auto" else (int(v) for v in shape.split(","))
    mode = moments if shape != "auto" and precision == "fp32_bulk" else 0
    ctx.build_stencils(mesh, order_p=P_ORDER, ring=RING, lanes_per_cell=lanes, rows_per_lane=rows,
                       moments_mode=mode)
    ctx.autotune_enabled = shape == "auto"
    return ctx


L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2


def timed_steps(torch, ctx, u, steps, stream, flush):
    """Exactly `steps` TVD-RK3 steps, each one replay of the captured step
    between its own CUDA-event pair on the launching stream, with an L2 flush
    (a 256 MB write) before each step outside the events; returns the summed
    step time in ms."""
    pairs = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.rk_step(u, cfl=CFL, n_steps=1)  # the captured step (same state, dt rule)
        e1.record(stream)
        pairs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in pairs)


def run_precision(torch, ctx, u0, steps, warmup, dist, sampler=None):
    """W untimed steps, then exactly `steps` timed TVD-RK3 steps bracketed by
    a barrier and a device synchronisation (L2 flushed before each, outside
    its events); returns times and the state."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    t_setup = time.perf_counter()
    ctx.precompute_moments()
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t_setup
    u = torch.tensor(u0, dtype=torch.float64, device=dev)
    if getattr(ctx, "autotune_enabled", True):
        shape = ctx.autotune(u, reps=3)
    else:
        info = ctx.info()
        shape = (info["lanes_per_cell"], info["rows_per_lane"], None)
    setup_s = time.perf_counter() - t_setup
    # warm-up (two steps at least: they capture the step graph the timed
    # single-step calls replay)
    ctx.rk_step(u, cfl=CFL, n_steps=max(2, warmup))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    launches0 = ctx.diagnostics()["kernel_launches"]
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_begin = time.time()
    ms = timed_steps(torch, ctx, u, steps, stream, flush)
    torch.cuda.synchronize(dev)
    t_end = time.time()
    if dist:
        dist.barrier()
    if sampler:
        sampler.mark(t_begin, t_end)
    clocks = sampler.stop() if sampler else None
    del flush
    launches = ctx.diagnostics()["kernel_launches"] - launches0
    # kernel split: the same steps again (from a copy of the state) with a
    # CUDA-event pair around every launch on the launching stream
    ctx.set_timing(True)
    v = u.clone()
    ctx.rk_step(v, cfl=CFL, n_steps=steps)
    torch.cuda.synchronize(dev)
    diag = ctx.diagnostics()
    ctx.set_timing(False)
    del v
    ms = max_over_ranks(ms, dist, dev)  # the job is as slow as its slowest rank
    stages = max(1, diag["launches_by_kind"]["flux"])  # one flux/RK launch per stage
    return {"ms": ms, "u": u, "diag": diag, "launches": launches,
            "clocks": clocks, "setup_s": setup_s, "shape": shape[:2], "info": ctx.info(),
            "flagged_per_stage": diag["flagged_cells"] / stages}


def run_moments_mode(torch, mesh, u0, dev_index, mode, steps):
    """The FP32-bulk thread-per-cell kernel in one moments mode: step time
    (captured steps, CUDA events) and the main kernel's mean launch time."""
    ctx = make_context("fp32_bulk", mesh, dev_index, "1,0", mode)
    ctx.precompute_moments()
    dev = torch.device("cuda", dev_index)
    u = torch.tensor(u0, dtype=torch.float64, device=dev)
    ctx.rk_step(u, cfl=CFL, n_steps=3)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    ms = timed_steps(torch, ctx, u, steps, torch.cuda.current_stream(dev), flush)
    del flush
    ctx.set_timing(True)
    ctx.rk_step(u, cfl=CFL, n_steps=steps)
    torch.cuda.synchronize(dev)
    d = ctx.diagnostics()
    ctx.set_timing(False)
    ctx.close()
    k = d["launches_by_kind"]["reconstruct"]
    return {"ms_per_step": ms / steps, "main_kernel_us": 1e3 * d["kernel_ms"]["reconstruct"] / max(1, k)}


def run_e2e(torch, ctx, u0, steps):
    """Same metric through the public call with a pinned HOST buffer: every
    step copies the state host->device, runs one TVD-RK3 step and copies the
    state back (both inside the timed region)."""
    uh = torch.tensor(u0, dtype=torch.float64).pin_memory()
    ctx.rk_step(uh, cfl=CFL, n_steps=1)  # warm the staging buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.rk_step(uh, cfl=CFL, n_steps=1)
    el = time.perf_counter() - t0
    return el, uh.numel() * 8


def roofline(info, diag, n_cells, precision, peaks, sm_mhz):
    """Roofline of the main reconstruction kernel (the dominant kernel): its
    algorithmic bytes and flops per launch over its average CUDA-event launch
    time inside the timed steps.  The follow-up kernels on the cells it flags
    are timed separately (kind "fixup")."""
    n = info["stencil_nnz"] / n_cells
    m = info["m"]
    npts = (info["dim"] + 1) * info["quad_per_facet"]
    otf = precision == "fp32_bulk" and info.get("moments_mode", 0) == 1
    launches = diag["launches_by_kind"]["reconstruct"]
    ms = diag["kernel_ms"]["reconstruct"]
    if launches == 0 or ms <= 0:
        return None
    dur = ms / launches * 1e-3
    flops = algorithmic_flops_per_cell(n, m, npts) * n_cells
    a_bytes = 4 if precision == "fp32_bulk" else 8
    nbytes = algorithmic_bytes_per_cell(n, m, npts, info["dim"], a_bytes, otf) * n_cells
    clock = (sm_mhz or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    if precision == "fp32_bulk":
        alu_peak = N_SMS * FP32_PEAK_LANES_PER_SM * 2 * clock / 1e12
    else:
        alu_peak = FP64_NOMINAL_TFLOPS
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    alu = flops / dur / 1e12
    hbm = nbytes / dur / 1e9
    name = f"main reconstruction kernel ({precision}{', moments on the fly' if otf else ''}), per launch"
    traffic = TRAFFIC_PER_LAUNCH.get((precision, 1 if otf else 0))
    out_alu = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s",
               "frac": alu / alu_peak, "traffic": traffic, "kernel": name,
               "flops_per_launch": flops, "launch_us": dur * 1e6}
    out_hbm = {"bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s",
               "frac": hbm / hbm_peak, "traffic": traffic, "kernel": name,
               "bytes_per_launch": nbytes, "launch_us": dur * 1e6}
    return (out_alu, out_hbm) if out_alu["frac"] >= out_hbm["frac"] else (out_hbm, out_alu)


def burgers_exact_averages(mesh, t):
    """Cell averages of the exact pre-shock solution of u_t + (u^2/2)_x +
    (u^2/2)_y = 0 with u0 = 0.5 + sin(2 pi (x + y)): u = u0(x + y - 2 u t),
    solved by Newton's method at each quadrature point (valid for
    t < 1/(4 pi))."""
    def f(P):
        xi = P[:, 0] + P[:, 1]
        u = 0.5 + np.sin(2 * np.pi * xi)
        for _ in range(50):
            ph = 2 * np.pi * (xi - 2 * u * t)
            u = u - (u - 0.5 - np.sin(ph)) / (1 + 4 * np.pi * t * np.cos(ph))
        return u
    return synth.cell_averages(mesh, f, k=4)


def accuracy_report(torch, mesh, u0, ctx32, ctx64, horizons=(3, 30)):
    """Untimed: both paths from u0 at the same fixed dt (CFL 0.3 at t = 0);
    FP32-bulk vs FP64 and each vs the exact solution after each horizon."""
    dev = torch.device("cuda", torch.cuda.current_device())
    rmin = float(np.min(ctx64.geometry()["inradius"]))
    dt = CFL * rmin / (math.sqrt(2.0) * float(np.max(np.abs(u0))))
    out = {"dt": dt, "steps": list(horizons), "rel_l1_fp32_bulk_vs_fp64": [],
           "rel_l1_vs_exact_fp64": [], "rel_l1_vs_exact_fp32_bulk": []}
    us = {k: torch.tensor(u0, dtype=torch.float64, device=dev) for k in ("32", "64")}
    done = 0
    for h in horizons:
        ctx32.rk_step(us["32"], dt=dt, n_steps=h - done)
        ctx64.rk_step(us["64"], dt=dt, n_steps=h - done)
        done = h
        a32 = us["32"].cpu().numpy()
        a64 = us["64"].cpu().numpy()
        ex = burgers_exact_averages(mesh, h * dt)
        out["rel_l1_fp32_bulk_vs_fp64"].append(float(np.sum(np.abs(a32 - a64)) / np.sum(np.abs(a64))))
        out["rel_l1_vs_exact_fp64"].append(float(np.sum(np.abs(a64 - ex)) / np.sum(np.abs(ex))))
        out["rel_l1_vs_exact_fp32_bulk"].append(float(np.sum(np.abs(a32 - ex)) / np.sum(np.abs(ex))))
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "fallback": True}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n_cells = 2 * args.n * args.n
    workload = WORKLOAD if args.n == N_SIDE else WORKLOAD.replace("256x256", f"{args.n}x{args.n}").replace(
        "131,072", f"{n_cells:,}")
    mesh = synth.tri_mesh(args.n, jitter=JITTER, seed=SEED)
    u0 = synth.burgers_2d_initial(mesh)
    config = {"workload": workload, "cells": n_cells, "p": P_ORDER, "stencil_ring": RING, "cfl": CFL,
              "mesh_seed": SEED, "l2": "flushed: a 256 MB write before every timed step, outside its CUDA "
              "events (each step timed alone; e2e steps run back to back with their state copies)"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        rate, desc, cores = oracle_cpu_rate(mesh, u0, max(2.0, args.cpu_seconds), host_cores(),
                                            warmup=args.warmup, steps=max(1, args.steps))
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": n_cells * 3 / rate * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = load_peaks()
    sampler = ClockSampler(gpu_uuid(torch, dev))

    ctx32 = make_context("fp32_bulk", mesh, dev.index, args.shape, args.moments)
    info = ctx32.info()
    r32 = run_precision(torch, ctx32, u0, args.steps, args.warmup, dist, sampler)
    ctx64 = make_context("fp64", mesh, dev.index, args.shape)
    r64 = run_precision(torch, ctx64, u0, args.steps, args.warmup, dist, None)
    u32 = r32["u"].cpu().numpy()
    u64 = r64["u"].cpu().numpy()
    rel_l1 = float(np.sum(np.abs(u32 - u64)) / np.sum(np.abs(u64)))
    accuracy = accuracy_report(torch, mesh, u0, ctx32, ctx64)
    ctx64.close()

    e2e_steps = max(3, min(args.steps, 50))
    el, state_bytes = run_e2e(torch, ctx32, u0, e2e_steps)
    el = max_over_ranks(el, dist, dev)
    ctx32.close()

    # every rank steps its own replica: the units of all ranks over the
    # slowest rank's time (already max-reduced)
    total = sum_over_ranks(n_cells * 3 * args.steps, dist, dev)
    value = total / (r32["ms"] * 1e-3)
    value64 = total / (r64["ms"] * 1e-3)
    clocks = r32["clocks"] or {}
    roof = roofline(r32["info"], r32["diag"], n_cells, "fp32_bulk", peaks, None)
    roof64 = roofline(r64["info"], r64["diag"], n_cells, "fp64", peaks, None)
    mode_steps = max(3, min(args.steps, 50))
    modes = {name: run_moments_mode(torch, mesh, u0, dev.index, mode, mode_steps)
             for mode, name in ((0, "stored_rows"), (1, "on_the_fly"))}
    modes["chosen"] = "on_the_fly" if r32["info"]["moments_mode"] == 1 else "stored_rows"
    kern = {k: {"launches": r32["diag"]["launches_by_kind"][k], "ms": r32["diag"]["kernel_ms"][k]}
            for k in ("reconstruct", "fixup", "flux", "dt")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r32["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32",
            "precision": "FP32-bulk: f32 weights, QR, evaluation and deviation flux; f64 moments and "
                         "refinement residual; double-float (f32 pair) reference flux, sums and RK update",
            "data": "synthetic", "config": dict(config, parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
            "fp64_gpu": {"value": value64, "ms_per_step": r64["ms"] / args.steps,
                         "speedup_fp32_bulk_vs_fp64": value / value64,
                         "rel_l1_fp32_bulk_vs_fp64_after_timed_steps": rel_l1,
                         "accuracy": accuracy,
                         "roofline": roof64[0] if roof64 else None},
            "e2e": {"value": sum_over_ranks(n_cells * 3 * e2e_steps, dist, dev) / el, "unit": UNIT,
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                    "steps": e2e_steps},
            "gpu_launches": r32["launches"],
            "kernels": kern,
            "roofline": roof[0] if roof else None,
            "roofline_other": roof[1] if roof else None,
            "setup_s": {"moments_and_autotune_fp32": r32["setup_s"],
                        "moments_and_autotune_fp64": r64["setup_s"]},
            "kernel_shape": {"fp32_bulk": list(r32["shape"]), "fp64": list(r64["shape"])},
            "moments_modes": modes,
            "refined_cells_per_stage": r32["flagged_per_stage"],
            "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                       "reasons": clocks.get("reasons", []),
                       "samples_in_timed_region": clocks.get("samples_in_timed_region")},
            "peaks": {"source": "MEASURED_PEAKS.json" if not peaks.get("fallback") else "fallback",
                      "hbm_gbs": peaks.get("hbm_gbs")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate1, desc1, _ = oracle_cpu_rate(mesh, u0, args.cpu_seconds, 1)
        rate, desc, cores = oracle_cpu_rate(mesh, u0, args.cpu_seconds, host_cores())
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                                "single_core": {"value": rate1, "cores": 1, "sample": desc1}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
