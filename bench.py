#!/usr/bin/env python
"""Benchmark of the pseudo-Verlet SPH density loop on GB300.

One step = one pass of the whole hot path over one synthetic particle set:
pv_sort_cells (cell grid + 13 sorted projections), pv_density (rho, drho/dh,
n) and pv_density_backward (dL/dx, dL/dh).  The workload is N = 1,048,576
uniform random particles in a periodic unit cube, h_i = 1.2348 N^(-1/3)
U(0.9, 1.1), 15^3 cells (about 311 per cell).  The metric is density-loop
pair interactions per second: sum_i n_i of the step divided by its time.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the only other place this script runs it).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "density-loop pair interactions/s"
UNIT = "interactions/s"
WORKLOAD = "uniform N=1048576, 15^3 cells, h=1.2348 N^-1/3 U(0.9,1.1), sort+density+backward"
# Algorithmic FP32 work (an FMA counts 2).  Forward: a window candidate is a
# distance test (3 sub, r^2 by 1 mul + 2 fma, compare = 9); a pair in range
# adds q, the two cubic pieces, the select and two accumulations (23).
# Adjoint: a candidate also takes the max of two squared supports (10); each
# own pair adds r, q, the four kernel factors and three accumulations (24),
# each transposed pair its two factors and its term (11), and each pair of
# the union the three gradient FMAs (6).
FWD_FLOP_CAND, FWD_FLOP_PAIR = 9, 23
BWD_FLOP_CAND, BWD_FLOP_OWN, BWD_FLOP_TRANS, BWD_FLOP_PAIR = 10, 24, 11, 6
# The same work in algorithmic FP32-pipe instructions (one FMA = one
# instruction): a distance test is 7 (3 sub, 1 mul, 2 fma, 1 compare), the
# kernel terms of a pair in range 15; the adjoint evaluates about twice the
# per-pair terms (own and transposed), 30.
FWD_INST_CAND, FWD_INST_PAIR = 7, 15
BWD_INST_CAND, BWD_INST_PAIR = 7, 30
FP32_LANES_PER_SM = 128
CSRC = os.path.join(ROOT, "paper_1804_06231_gb300", "csrc")
# sweep kernel -> (ncu summary under profiles/, sources whose hash it was taken on)
PROFILED = {
    "k_backward_cells": ("backward_cells_uniform1m.md", ("pv_backward.cu", "pv_internal.cuh")),
    "k_density_cells": ("density_cells_uniform1m.md", ("pv_density.cu", "pv_internal.cuh")),
}


def sources_sha256(files):
    import hashlib
    hs = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            hs.update(fh.read())
    return hs.hexdigest()


def profiled_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` on the default workload,
    from its ncu summary, or None when the summary is missing or was taken on
    other kernel sources than the current ones."""
    name, files = PROFILED[kernel]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.split(":", 1)[0].strip() in ("dram_bytes_per_launch",
                                                             "sources_sha256"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("sources_sha256") != sources_sha256(files):
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="pv", choices=["pv", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="keep the default launch shape")
    p.add_argument("--launch-shape", default="",
                   help="D,B[,TD,TB]: CTAs per SM of the density and adjoint cell kernels and "
                        "particles per task of their task kernels (no tuning)")
    p.add_argument("--workload", default="uniform1m", choices=["uniform1m", "clustered4m"],
                   help="the timed workload (clustered4m: for profiling the dense-cell paths)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the 4M clustered and 64-box workloads (extra keys)")
    # smaller uniform workloads with the same h rule, for profiler captures
    p.add_argument("--particles", type=int, default=0)
    p.add_argument("--cells", type=int, default=0)
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling (every 20 ms, timestamped) of SM clock and throttle
    reasons; stop() summarises the samples taken inside [t0, t1] (host wall
    clock, set by mark_start / mark_stop)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        import tempfile
        self.proc = None
        self.uuid = uuid
        self.path = os.path.join(tempfile.gettempdir(), f"pv_bench_clocks_{os.getpid()}.csv")
        self.t0 = self.t1 = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "20"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def mark_start(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def mark_stop(self):
        import datetime
        self.t1 = datetime.datetime.now()

    def stop(self) -> dict:
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                t = None
                for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
                    try:
                        t = datetime.datetime.strptime(parts[0], fmt)
                        break
                    except ValueError:
                        pass
                try:
                    rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        pad = datetime.timedelta(milliseconds=25)
        inside = [r for r in rows if r[0] and self.t0 and self.t1 and
                  self.t0 - pad <= r[0] <= self.t1 + pad]
        use = inside or [r for r in rows if r[0] and self.t0 and r[0] >= self.t0] or rows
        reasons = set()
        for r in use:
            for nm, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median([r[1] for r in use]) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": sorted(reasons), "samples": len(use),
                "samples_in_timed_region": len(inside)}


# ------------------------------------------------------------------ workloads

def workload(seed: int, particles: int = 0, cells: int = 0, name: str = "uniform1m"):
    from paper_1804_06231_gb300 import inputs as I
    if particles:
        return I.uniform(particles, seed, nc=cells or None)
    if name == "clustered4m":
        return I.cfg2(I.SEEDS["cfg2"] + seed - 1)
    return I.cfg1(seed)


def timed_steps(step, flush, K: int, W: int = 3) -> float:
    """Median CUDA-event time (ms) of `step` over K runs after W warm-ups, L2
    flushed before each run (outside the events)."""
    import torch
    for _ in range(W):
        step()
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(K):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def phase_times(grid, step_args, flush, K: int) -> tuple:
    """Median CUDA-event times (ms) of sort, density and backward over K steps
    (after 2 warm-ups, L2 flushed before each step), with the sweep kernels'
    own times from the grid's event hooks."""
    import torch
    pos, h, m, gr, gd, rho, D, nn, gp, gh = step_args
    for _ in range(2):
        grid.sort(pos, h, m)
        grid.density(rho, D, nn)
        grid.backward(gr, gd, gp, gh)
    stream = torch.cuda.current_stream()
    grid.time_sweeps(True)
    ts = []
    for _ in range(K):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        grid.sort(pos, h, m)
        e[1].record(stream)
        grid.density(rho, D, nn)
        e[2].record(stream)
        grid.backward(gr, gd, gp, gh)
        e[3].record(stream)
        e[3].synchronize()
        ts.append([e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3]),
                   e[0].elapsed_time(e[3])])
    k_dens, k_bwd = grid.sweep_times()
    grid.time_sweeps(False)
    med = [statistics.median(col) for col in zip(*ts)]
    return med[0], med[1], med[2], med[3], k_dens, k_bwd


def workload_extras(dev, flush, probe: dict, peak_derived: float, K: int = 5) -> dict:
    """The other two throughput workloads of the method: 4,194,304 clustered
    particles on the finest grid (one box), and the 64-box mix as one batched
    grid, as 64 separate grids, and as a CUDA-graph replay of the batched step.
    Each is sort + density + backward with an autotuned launch shape."""
    import torch
    from paper_1804_06231_gb300 import inputs as I, tune
    from paper_1804_06231_gb300.pv import Grid

    def tensors(boxes):
        pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
        h = torch.from_numpy(np.concatenate([b.h for b in boxes])).to(dev)
        m = torch.from_numpy(np.concatenate([b.m for b in boxes])).to(dev)
        rng = np.random.default_rng(7)
        n = pos.shape[0]
        gr = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
        gd = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
        outs = (torch.empty(n, device=dev), torch.empty(n, device=dev),
                torch.empty(n, device=dev, dtype=torch.int32),
                torch.empty((n, 3), device=dev), torch.empty(n, device=dev))
        return pos, h, m, gr, gd, outs

    out = {}
    box = I.cfg2()
    pos, h, m, gr, gd, (rho, D, nn, gp, gh) = tensors([box])
    with Grid((box.n, box.L, box.nc)) as g:
        def step():
            g.sort(pos, h, m)
            g.density(rho, D, nn)
            g.backward(gr, gd, gp, gh)
        step()
        tr = tune.autotune(g, gr, gd, reps=3)
        t = timed_steps(step, flush, K)
        inter = g.stats().interactions
        cand = g.count_candidates()
        stc = g.stats()
        t_sort, t_dens, t_bwd, t_step, k_dens, k_bwd = phase_times(
            g, (pos, h, m, gr, gd, rho, D, nn, gp, gh), flush, K)
        fw, bw = sweep_work(box.n, cand, inter, stc.candidates_adjoint, stc.pairs_adjoint)
        # the dense cells run on the task kernels: the roofline covers the
        # whole pass (plan, cell-centric, warp-per-cell and task kernels)
        out["clustered_4m"] = {
            "workload": f"clustered N={box.n}, {box.nc}^3 cells, 64 Gaussians + 20% uniform",
            "ms_per_step": t, "value": inter / (t * 1e-3), "unit": UNIT,
            "launch_shape": [tr["density_ctas_per_sm"], tr["backward_ctas_per_sm"],
                             tr["density_task_block"], tr["backward_task_block"]],
            "max_cell_count": stc.max_cell_count,
            "breakdown_ms": {"sort": t_sort, "density": t_dens, "backward": t_bwd,
                             "step": t_step, "density_cell_kernel": k_dens,
                             "backward_cell_kernel": k_bwd},
            "fwd_bwd_over_fwd": t_step / (t_sort + t_dens),
            "candidates": cand, "interactions": inter,
            "candidates_adjoint": stc.candidates_adjoint, "pairs_adjoint": stc.pairs_adjoint,
            "symmetric_update": symmetric_update(g, flush, rho, D, nn),
            "roofline_density_pass": sweep_roofline("pv_density (all its kernels)", fw[0], fw[1],
                                                    t_dens, probe, peak_derived),
            "roofline_adjoint_pass": sweep_roofline("pv_density_backward (all its kernels)",
                                                    bw[0], bw[1], t_bwd, probe, peak_derived),
            "roofline_sort": sort_roofline(box.n, t_sort, measured_peaks())}
    del pos, h, m, gr, gd, rho, D, nn, gp, gh
    torch.cuda.empty_cache()

    boxes = I.multibox()
    pos, h, m, gr, gd, (rho, D, nn, gp, gh) = tensors(boxes)
    gb = Grid([(b.n, b.L, b.nc) for b in boxes])

    def step_b():
        gb.sort(pos, h, m)
        gb.density(rho, D, nn)
        gb.backward(gr, gd, gp, gh)
    step_b()
    tr = tune.autotune(gb, gr, gd, reps=3)
    t_b = timed_steps(step_b, flush, K)
    inter = gb.stats().interactions
    views, first = [], 0
    for b in boxes:
        sl = slice(first, first + b.n)
        gg = Grid((b.n, b.L, b.nc))
        gg.set_tuning(tr["density_ctas_per_sm"], tr["backward_ctas_per_sm"],
                      tr["density_task_block"], tr["backward_task_block"])
        views.append((gg, pos[sl], h[sl], m[sl], gr[sl], gd[sl], rho[sl], D[sl], nn[sl],
                      gp[sl], gh[sl]))
        first += b.n

    def step_p():
        for gg, p_, h_, m_, gr_, gd_, r_, d_, n_, gp_, gh_ in views:
            gg.sort(p_, h_, m_)
            gg.density(r_, d_, n_)
            gg.backward(gr_, gd_, gp_, gh_)
    t_p = timed_steps(step_p, flush, K)
    for v in views:
        v[0].close()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step_b()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_b()
    t_g = timed_steps(graph.replay, flush, K)
    gb.close()
    out["multibox_64"] = {
        "workload": f"64 boxes, N={sum(b.n for b in boxes)} (per box log-uniform in "
                    "[4096, 524288], uniform or clustered)",
        "ms_per_step_batched": t_b, "ms_per_step_per_box": t_p, "ms_per_step_graph": t_g,
        "value": inter / (t_g * 1e-3), "unit": UNIT,
        "launch_shape": [tr["density_ctas_per_sm"], tr["backward_ctas_per_sm"],
                         tr["density_task_block"], tr["backward_task_block"]]}
    return out


def fp32_probe(dev, props) -> dict:
    """FP32 peak of this GPU, measured: pv_fp32_probe with 8 CTAs of 256
    threads per SM, each thread running 8 independent FMA chains, timed with
    CUDA events (best of 5 launches after 2 warm-ups), as scalar FFMA and as
    packed fma.rn.f32x2."""
    import torch
    from paper_1804_06231_gb300.pv import pv_fp32_probe
    threads = props.multi_processor_count * 8 * 256
    sink = torch.empty(threads, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    iters = 16384
    out = {"threads": threads, "iters": iters, "chains_per_thread": 8}
    for packed, key in ((0, "ffma_tflops"), (1, "ffma2_tflops")):
        best = 0.0
        for rep in range(7):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = pv_fp32_probe(packed, iters, sink.data_ptr(), threads, stream.cuda_stream)
            b.record(stream)
            b.synchronize()
            if rep >= 2:
                best = max(best, flops / (a.elapsed_time(b) * 1e-3) / 1e12)
        out[key] = best
    out["ffma_inst_per_s"] = out["ffma_tflops"] * 1e12 / 2.0
    return out


def sweep_work(n: int, candidates: int, interactions: int, cand_adj: int, pairs_adj: int):
    """(flops, FP32 instructions) of the density pass and of the adjoint pass:
    window candidates and in-range pairs (j = i included) for the forward,
    adjoint candidates and pairs for the adjoint."""
    pairs = interactions + n
    fwd = (FWD_FLOP_CAND * candidates + FWD_FLOP_PAIR * pairs,
           FWD_INST_CAND * candidates + FWD_INST_PAIR * interactions)
    bwd = (BWD_FLOP_CAND * cand_adj + (BWD_FLOP_OWN + BWD_FLOP_TRANS) * interactions
           + BWD_FLOP_PAIR * (pairs_adj - n),
           BWD_INST_CAND * cand_adj + BWD_INST_PAIR * interactions)
    return fwd, bwd


def sweep_roofline(kernel: str, flops: float, insts: float, ms: float, probe: dict,
                   derived_tflops: float, traffic=None) -> dict:
    """FP32 roofline of a sweep: algorithmic FP32 work per launch over its
    CUDA-event time, against the FFMA peak measured by pv_fp32_probe in this
    run; `instructions` is the same in FP32 instructions (an FMA counts once)."""
    a = flops / (ms * 1e-3) / 1e12
    peak = probe["ffma_tflops"]
    ai = insts / (ms * 1e-3) / 1e12
    pi = probe["ffma_inst_per_s"] / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": a, "peak": peak, "unit": "TFLOP/s",
            "frac": a / peak, "traffic": traffic, "flop_per_launch": flops,
            "ms_per_launch": ms,
            "peak_source": "pv_fp32_probe: scalar FFMA chains on every SM, measured in this run "
                           "(of measured)",
            "peak_derived_tflops": derived_tflops,
            "instructions": {"achieved": ai, "peak": pi, "unit": "T FP32 inst/s",
                             "frac": ai / pi, "inst_per_launch": insts}}


# Algorithmic HBM bytes per particle of pv_sort_cells: the grid build reads
# position, h and mass (32 B) and writes the cell-order record and h (24 B);
# the 13-axis sort reads the record (16 B) and writes 13 16-bit indices (26 B).
SORT_BYTES_PER_PARTICLE = 32 + 24 + 16 + 26


def sort_roofline(n: int, ms: float, peaks: dict) -> dict:
    """HBM roofline of pv_sort_cells (all its kernels): algorithmic bytes per
    sort over its CUDA-event time, against the measured copy bandwidth."""
    b = SORT_BYTES_PER_PARTICLE * n
    a = b / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs")
    return {"bound": "hbm", "kernel": "pv_sort_cells (all its kernels)", "achieved": a,
            "peak": peak, "unit": "GB/s", "frac": a / peak if peak else None, "traffic": None,
            "bytes_per_launch": b, "ms_per_launch": ms,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}


def raw_ceiling(dev, props, peak_tflops: float) -> dict:
    """The interaction arithmetic alone (pv_raw_interactions): 1024 particles
    per SM against 2560 others (the paper's first experiment uses 2560), all
    pairs in range, every lane busy."""
    import torch
    from paper_1804_06231_gb300.pv import raw_interactions
    g = torch.Generator(device="cpu").manual_seed(5)
    H = 0.05

    def ball(n):
        v = torch.randn((n, 3), generator=g, dtype=torch.float64)
        r = 0.45 * H * torch.rand(n, generator=g, dtype=torch.float64) ** (1.0 / 3.0)
        v = v * (r / v.norm(dim=1))[:, None]
        m = torch.full((n, 1), 1.0 / n, dtype=torch.float64)
        return torch.cat([v, m], dim=1).float().to(dev)
    ni, nj, reps = props.multi_processor_count * 1024, 2560, 8
    xi, xj = ball(ni), ball(nj)
    out = torch.empty((ni, 2), device=dev)
    ms = timed_steps(lambda: raw_interactions(xi, xj, H, reps, out), torch.empty(0, device=dev),
                     5, 2)
    rate = ni * nj * reps / (ms * 1e-3)
    tf = rate * FWD_FLOP_PAIR / 1e12
    return {"interactions_per_s": rate, "n_i": ni, "n_j": nj, "reps": reps, "ms": ms,
            "tflops": tf, "frac_of_fp32_peak": tf / peak_tflops,
            "flop_per_interaction": FWD_FLOP_PAIR}


def sort_reuse(grid, box, pos, h, m_uniform, flush, density, backward, dev, K: int = 5) -> dict:
    """pv_update_positions against pv_sort_cells on the same workload: the
    particles are moved by up to 0.05 H_max (seeded; about one time step of an
    SPH code), then the step runs on the kept sort with widened windows."""
    import torch
    rng = np.random.default_rng(11)
    dmax = 0.05 * 1.825742 * float(box.h.max())
    v = rng.standard_normal((box.n, 3))
    v *= (dmax * rng.random(box.n) / np.linalg.norm(v, axis=1))[:, None]
    npos = torch.from_numpy(np.mod(box.pos + v, box.L)).to(dev)
    t_sort = timed_steps(lambda: grid.sort(pos, h, None, m_uniform), flush, K)
    grid.sort(pos, h, None, m_uniform)
    t_upd = timed_steps(lambda: grid.update(npos, h), flush, K)

    def step():
        grid.update(npos, h)
        density()
        backward()
    t_step = timed_steps(step, flush, K)
    t_dens = timed_steps(density, flush, K)
    grid.sort(pos, h, None, m_uniform)
    grid.update(pos, h)  # kept sort, no displacement: the cost of the update mode alone
    t_dens0 = timed_steps(density, flush, K)
    grid.sort(pos, h, None, m_uniform)
    return {"sort_ms": t_sort, "update_ms": t_upd, "density_ms_after_update": t_dens,
            "density_ms_after_update_without_motion": t_dens0,
            "step_ms_with_update": t_step, "displacement": "<= 0.05 H_max"}


def graph_step(step, flush, K: int = 20) -> dict:
    """The step captured once in a CUDA graph and replayed (L2 flushed before
    each replay, outside the events); same kernels, no per-launch host work."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # eager warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    return {"ms_per_step": timed_steps(graph.replay, flush, K)}


def symmetric_update(grid, flush, rho, drho, nngb, K: int = 5) -> dict:
    """The density pass as the gather (pv_density) against the paper's
    symmetric pair update (pv_density_symmetric) on the same sorted grid."""
    t_g = timed_steps(lambda: grid.density(rho, drho, nngb), flush, K)
    t_s = timed_steps(lambda: grid.density(rho, drho, nngb, symmetric=True), flush, K)
    return {"density_ms_gather": t_g, "density_ms_symmetric": t_s,
            "symmetric_over_gather": t_s / t_g}


def orientation_breakdown(grid, st, flush, density, K: int = 5) -> dict:
    """Density pass restricted to each neighbour orientation class in turn
    (slot masks): time, window distance tests and interactions per class."""
    from paper_1804_06231_gb300.pv import SLOT_MASK_ALL, slot_mask_of_class
    ms = []
    for c in range(4):
        grid.set_slot_mask(slot_mask_of_class(c))
        ms.append(timed_steps(density, flush, K))
    grid.set_slot_mask(SLOT_MASK_ALL)
    tot = sum(ms)
    cand = [st.orientation[c][0] for c in range(4)]
    inter = [st.orientation[c][1] for c in range(4)]
    return {"classes": ["self", "face", "edge", "corner"], "density_ms": ms,
            "time_share": [t / tot for t in ms], "candidates": cand, "interactions": inter,
            "in_range_fraction": [i / max(c, 1) for c, i in zip(cand, inter)]}


def cpu_sample(seed: int):
    """Bounded sample of the workload for the CPU oracle: a periodic sub-box of
    7^3 cells of the same edge (1/15), number density and h rule -- 106,572
    particles (1/9.8 of the volume)."""
    from paper_1804_06231_gb300 import inputs as I
    L = 7.0 / 15.0
    n = int(round((1 << 20) * L ** 3))
    b = I.uniform(n, seed + 777, nc=7, L=L)
    b.name = f"uniform sub-box N={n}, L=7/15, 7^3 cells"
    return b


def time_oracle(box, steps: int, warmup: int, threads: int):
    """Times oracle density (pseudo-Verlet sweep) + oracle adjoint per step."""
    import oracle
    from paper_1804_06231_gb300 import inputs as I
    w, v = I.loss_weights(box.n, 0)
    times, inter = [], 0
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        d = oracle.density_pv(box.pos, box.h, box.m, box.L, box.nc, threads=threads)
        g, k = oracle.loss_upstream(d.rho, w, v)
        oracle.backward_cells(box.pos, box.h, box.m, g, k, box.L, box.nc, threads=threads)
        t1 = time.perf_counter()
        if s >= warmup:
            times.append(t1 - t0)
        inter = int(d.n_ngb.sum())
    return inter, times


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ reference arm

def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = host_cores()
    box = cpu_sample(0)
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    # bound the total: each step is ~1-2 s on 16 cores; cap the counts
    steps = min(steps, 40)
    warmup = min(warmup, 10)
    inter, times = time_oracle(box, steps, warmup, cores)
    t = statistics.mean(times)
    value = inter / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": len(times), "warmup": warmup, "ms_per_step": 1e3 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": box.name, "device": "host CPU cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": box.name + "; FP64 pseudo-Verlet density + cell-list adjoint"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist

    from paper_1804_06231_gb300 import build as B
    B.build_library()
    from paper_1804_06231_gb300 import shard
    from paper_1804_06231_gb300.pv import Grid

    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.current_stream()

    box = workload(1 + rank, args.particles, args.cells, args.workload)  # one box per rank
    n = box.n
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    rng = np.random.default_rng(100 + rank)
    g_rho = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    g_d = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    drho = torch.empty_like(rho)
    nngb = torch.empty(n, dtype=torch.int32, device=dev)
    gpos = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gh = torch.empty_like(rho)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2
    grid = Grid((n, 1.0, box.nc))
    m_uniform = float(box.m[0])

    def step():
        grid.sort(pos, h, None, m_uniform)
        grid.density(rho, drho, nngb)
        grid.backward(g_rho, g_d, gpos, gh)

    tuning = None
    shape0 = grid.tuning()
    step()  # first sort, so that the autotuner sees the sorted grid
    if args.launch_shape:
        vals = [int(x) for x in args.launch_shape.split(",")] + [0, 0]
        grid.set_tuning(*vals[:4])
        t = grid.tuning()
        tuning = {"density_ctas_per_sm": t[0], "backward_ctas_per_sm": t[1],
                  "density_task_block": t[2], "backward_task_block": t[3], "source": "given"}
    elif not args.no_tune:
        from paper_1804_06231_gb300 import tune
        tr = tune.autotune(grid, g_rho, g_d, reps=5)
        tuning = {k: tr[k] for k in ("density_ctas_per_sm", "backward_ctas_per_sm",
                                     "density_task_block", "backward_task_block", "source")}
    for _ in range(max(args.warmup, 3)):
        step()
    grid.sync()
    st0 = grid.stats()
    interactions = st0.interactions
    candidates = grid.count_candidates()
    st_c = grid.stats()
    cand_adj, pairs_adj = st_c.candidates_adjoint, st_c.pairs_adjoint

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    uuid = None
    try:
        uuid = "GPU-" + str(props.uuid) if not str(props.uuid).startswith("GPU") else str(props.uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid) if rank == 0 else None
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)  # nvidia-smi up and sampling
    launches0 = grid.stats().kernel_launches
    grid.time_sweeps(True)  # CUDA events around the two sweep kernels
    if clocks:
        clocks.mark_start()
    wall0 = time.perf_counter()
    for k in range(K):
        flush.zero_()  # evict the previous step's data from L2 (outside the events)
        e = ev[k]
        e[0].record(stream)
        grid.sort(pos, h, None, m_uniform)
        e[1].record(stream)
        grid.density(rho, drho, nngb)
        e[2].record(stream)
        grid.backward(g_rho, g_d, gpos, gh)
        e[3].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if clocks:
        clocks.mark_stop()
        time.sleep(0.05)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    launches = grid.stats().kernel_launches - launches0
    k_dens, k_bwd = grid.sweep_times()  # ms per launch of k_density_cells / k_backward_cells
    grid.time_sweeps(False)
    t_sort = sum(e[0].elapsed_time(e[1]) for e in ev) / K
    t_dens = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    t_bwd = sum(e[2].elapsed_time(e[3]) for e in ev) / K
    t_step = sum(e[0].elapsed_time(e[3]) for e in ev) / K  # ms
    st = grid.stats()
    assert st.device_flags == 0

    # one independent box per rank: only the totals are reduced
    tot_inter, t_max = shard.step_totals(interactions, t_step, dev)
    tot_inter = int(tot_inter)
    value = tot_inter / (t_max * 1e-3)

    # ---- end to end through the C ABI with host buffers (pinned).  Every
    # step uploads its inputs (positions, h, upstream gradients) from pinned
    # host memory and downloads its five outputs.  The steps are pipelined
    # over two device buffer sets: step k+1's upload (copy stream) and step
    # k-1's download (a second copy stream) run while step k computes; the
    # timed region runs from the first upload to the last download.
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(box.pos).pin_memory()
        hh = torch.from_numpy(box.h).pin_memory()
        hg = g_rho.cpu().pin_memory()
        hd = g_d.cpu().pin_memory()
        ins = [[torch.empty_like(t) for t in (pos, h, g_rho, g_d)] for _ in range(2)]
        outs = [[torch.empty_like(t) for t in (rho, drho, nngb, gpos, gh)] for _ in range(2)]
        houts = [[torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs[0]]
                 for _ in range(2)]
        bi = sum(t.numel() * t.element_size() for t in (hp, hh, hg, hd))
        bo = sum(t.numel() * t.element_size() for t in houts[0])
        cin, cout = torch.cuda.Stream(), torch.cuda.Stream()

        def run_pipelined(n_steps):
            done = [None] * n_steps      # compute of step k finished
            down = [None] * n_steps      # download of step k finished
            up = [None] * (n_steps + 1)  # upload of step k finished
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)

            def upload(k):
                with torch.cuda.stream(cin):
                    if k >= 2:
                        cin.wait_event(done[k - 2])  # its buffer set is free again
                    for dst, src in zip(ins[k % 2], (hp, hh, hg, hd)):
                        dst.copy_(src, non_blocking=True)
                    up[k] = cin.record_event()

            t0.record(cin)
            upload(0)
            for k in range(n_steps):
                b = k % 2
                if k + 1 < n_steps:
                    upload(k + 1)
                stream.wait_event(up[k])
                if k >= 2:
                    stream.wait_event(down[k - 2])  # its output set has been read
                p_, h_, gr_, gd_ = ins[b]
                r_, d_, n_, gp_, gh_ = outs[b]
                grid.sort(p_, h_, None, m_uniform)
                grid.density(r_, d_, n_)
                grid.backward(gr_, gd_, gp_, gh_)
                done[k] = stream.record_event()
                with torch.cuda.stream(cout):
                    cout.wait_event(done[k])
                    for dst, src in zip(houts[b], outs[b]):
                        dst.copy_(src, non_blocking=True)
                    down[k] = cout.record_event()
            stream.wait_event(down[n_steps - 1])
            t1.record(stream)
            t1.synchronize()
            return t0.elapsed_time(t1) / n_steps

        run_pipelined(3)  # warm-up
        flush.zero_()
        torch.cuda.synchronize()
        t_e2e = shard.step_totals(0, run_pipelined(K), dev)[1]
        e2e = {"value": tot_inter / (t_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": t_e2e,
               "pipelined": "two buffer sets; uploads and downloads overlap the neighbouring steps",
               "l2": "not flushed between steps: each step uploads its inputs from host memory "
                     "and rewrites ~0.25 GB of grid arrays, more than the 126 MB L2"}
        # the last step's outputs reached the host intact
        assert np.array_equal(houts[(K - 1) % 2][2].numpy(), nngb.cpu().numpy())

    # ---- rooflines of the two sweep kernels (FP32 ALU bound); the adjoint
    # sweep is the dominant kernel of the step
    peaks = measured_peaks()
    sm_max = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    peak_derived = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    probe = fp32_probe(dev, props)
    peak_tflops = probe["ffma_tflops"]
    default_size = not (args.particles or args.cells) and args.workload == "uniform1m"
    fw, bw = sweep_work(n, candidates, interactions, cand_adj, pairs_adj)

    def roof(kernel, work, ms):
        return sweep_roofline(kernel, work[0], work[1], ms, probe, peak_derived,
                              profiled_traffic(kernel) if default_size else None)

    roofline = roof("k_backward_cells", bw, k_bwd)
    roofline_fwd = roof("k_density_cells", fw, k_dens)

    extras = None
    if rank == 0 and ws == 1 and not args.no_extras and default_size:
        extras = {"orientation_breakdown": orientation_breakdown(
                      grid, st_c, flush, lambda: grid.density(rho, drho, nngb)),
                  "raw_interaction_ceiling": raw_ceiling(dev, props, peak_tflops),
                  "cuda_graph_step": graph_step(step, flush),
                  "symmetric_update": symmetric_update(grid, flush, rho, drho, nngb),
                  "sort_reuse": sort_reuse(grid, box, pos, h, m_uniform, flush,
                                           lambda: grid.density(rho, drho, nngb),
                                           lambda: grid.backward(g_rho, g_d, gpos, gh), dev)}
        extras.update(workload_extras(dev, flush, probe, peak_derived))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        cores = host_cores()
        cbox = cpu_sample(0)
        # about 10 s of oracle work on 16 cores: 1 warm-up and 10 timed steps
        c_inter, c_times = time_oracle(cbox, 10, 1, cores)
        cpu = {"value": c_inter / statistics.mean(c_times), "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": cbox.name + "; FP64 pseudo-Verlet density + cell-list adjoint, "
                                     f"{len(c_times)} runs"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": (f"uniform N={n}, {box.nc}^3 cells (profiling size)"
                                    if args.particles else
                                    f"clustered N={n}, {box.nc}^3 cells, 64 Gaussians + 20% "
                                    "uniform, sort+density+backward"
                                    if args.workload == "clustered4m" else WORKLOAD),
                       "n_particles_per_gpu": n, "cells": box.nc ** 3,
                       "l2": "flushed between steps (512 MiB write)",
                       "launch_shape": tuning or {"density_ctas_per_sm": shape0[0],
                                                  "backward_ctas_per_sm": shape0[1],
                                                  "density_task_block": shape0[2],
                                                  "backward_task_block": shape0[3],
                                                  "source": "default"},
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "e2e": e2e,
            "gpu_launches": launches,
            "roofline": roofline,
            "roofline_forward": roofline_fwd,
            "roofline_sort": sort_roofline(n, t_sort, peaks),
            "cpu_baseline": cpu,
            "clocks": clk,
            "breakdown_ms": {"sort": t_sort, "density": t_dens, "backward": t_bwd,
                             "density_sweep_kernel": k_dens, "backward_sweep_kernel": k_bwd},
            "density_interactions_per_s": interactions / (t_dens * 1e-3),
            # forward = sort + density (what a forward pass needs); fwd+bwd = the step
            "fwd_bwd_over_fwd": t_step / (t_sort + t_dens),
            "backward_over_density": t_bwd / t_dens,
            "candidates": candidates, "interactions": interactions,
            "candidates_adjoint": cand_adj, "pairs_adjoint": pairs_adj,
            "candidates_per_interaction": candidates / max(interactions, 1),
            "guard_pairs": st.guard_pairs, "wall_s_timed_loop": wall,
            "fp32_probe": probe,
        }
        if extras:
            line.update(extras)
        print(json.dumps(line), flush=True)
    grid.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
