"""Autotuner for the launch shape of the sweeps, with a JSON cache.

Each pass (``pv_density``, ``pv_density_backward``) has a shape per bin of
cells (``pv_grid_set_tuning``):

* the cell-centric bin: resident CTAs per SM of the cell kernel.  It trades
  occupancy against shared memory per CTA, and the shared memory decides
  which cells are swept by the cell kernel and which go to the task bin, so
  the best value depends on the workload: uniform boxes with small cells
  favour more CTAs, clustered boxes with dense cells favour more shared
  memory;
* the task bin (dense cells): particles, and threads, per task (64, 128 or
  256: 2, 4 or 8 warps per task).  Smaller tasks are more numerous and share
  a staged tile among fewer warps.

``autotune`` times the two calls (CUDA events on the current stream, median
of ``reps``) on an already sorted grid: first the CTAs per SM of each pass
at the default task block, then the task block of each pass at the chosen
CTAs.  A choice other than the default is kept only if it is faster by more
than ``TIE`` (on a workload without dense cells the task kernels find no work
and the default stays).  The result is stored under the workload's signature,
so that later grids of the same shape reuse it without timing.  Results do
not depend on the choice beyond FP32 summation order.
"""
from __future__ import annotations

import json
import math
import os
import statistics

DENSITY_CHOICES = (2, 3, 4)
BACKWARD_CHOICES = (1, 2, 3)
DEFAULT = (3, 3)
TASK_CHOICES = (64, 128, 256)
DEFAULT_TASK = 128
TIE = 0.01  # relative margin a choice other than the default must beat


def default_cache_path() -> str:
    return os.environ.get("PV_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1804_06231_gb300", "tuning.json")


def _bucket(x: float) -> int:
    """log2 bucket (0 for x <= 1)."""
    return 0 if x <= 1 else int(math.floor(math.log2(x)))


def signature(n_particles: int, n_cells: int, max_cell_count: int, n_boxes: int,
              device: str, num_sms: int) -> str:
    """Workload key: device, box count, and log2 buckets of the particle
    count, the mean and the largest cell occupancy."""
    mean = n_particles / max(n_cells, 1)
    return (f"{device}|sm{num_sms}|boxes{_bucket(n_boxes)}|n{_bucket(n_particles)}"
            f"|mean{_bucket(mean)}|max{_bucket(max_cell_count)}")


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    """Atomic write (temporary file + rename)."""
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _pick(times: dict, default):
    """The fastest choice, or the default when it is within TIE of it."""
    best = min(times, key=lambda c: times[c])
    return default if times[default] <= times[best] * (1.0 + TIE) else best


def choose(measure, reps: int = 5) -> tuple[tuple[int, int, int, int], dict]:
    """Runs ``measure(density_ctas, backward_ctas, density_block,
    backward_block, reps)`` -> (ms_density, ms_backward) for the combinations
    the passes need and returns the chosen (density CTAs, backward CTAs,
    density task block, backward task block) with the timings.  The passes
    are independent, so the density CTAs are timed with the default backward
    shape and vice versa, and both task blocks in one call per block size."""
    times = {"density": {}, "backward": {}, "density_task": {}, "backward_task": {}}
    for d in DENSITY_CHOICES:
        times["density"][d] = measure(d, DEFAULT[1], DEFAULT_TASK, DEFAULT_TASK, reps)[0]
    for b in BACKWARD_CHOICES:
        times["backward"][b] = measure(DEFAULT[0], b, DEFAULT_TASK, DEFAULT_TASK, reps)[1]
    best_d = _pick(times["density"], DEFAULT[0])
    best_b = _pick(times["backward"], DEFAULT[1])
    for t in TASK_CHOICES:
        times["density_task"][t], times["backward_task"][t] = measure(best_d, best_b, t, t, reps)
    best_td = _pick(times["density_task"], DEFAULT_TASK)
    best_tb = _pick(times["backward_task"], DEFAULT_TASK)
    return (best_d, best_b, best_td, best_tb), times


def grid_measure(grid, g_rho, g_drho_dh, warmup: int = 2):
    """A ``measure`` for ``choose`` on a sorted ``pv.Grid`` (CUDA events)."""
    import torch
    n = grid.n
    dev = g_rho.device
    rho = torch.empty(n, device=dev)
    D = torch.empty(n, device=dev)
    nn = torch.empty(n, device=dev, dtype=torch.int32)
    gp = torch.empty((n, 3), device=dev)
    gh = torch.empty(n, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(warmup):
            fn()
        out = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    def measure(d, b, td, tb, reps):
        grid.set_tuning(d, b, td, tb)
        tf = timed(lambda: grid.density(rho, D, nn), reps)
        tb = timed(lambda: grid.backward(g_rho, g_drho_dh, gp, gh), reps)
        return tf, tb

    return measure


def autotune(grid, g_rho, g_drho_dh=None, reps: int = 5, cache_path: str | None = None,
             use_cache: bool = True, measure=None, device_info=None) -> dict:
    """Picks and sets the launch shape of a sorted grid.  Returns
    {"density_ctas_per_sm", "backward_ctas_per_sm", "density_task_block",
    "backward_task_block", "source": "cache"|"timed", "signature",
    "times_ms"}.  ``device_info`` = (name, SM count), read from
    the device of ``g_rho`` when omitted."""
    st = grid.stats()
    if device_info is None:
        import torch
        props = torch.cuda.get_device_properties(g_rho.device)
        device_info = (props.name, props.multi_processor_count)
    sig = signature(st.n_particles, st.n_cells, st.max_cell_count, len(grid.boxes),
                    device_info[0], device_info[1])
    path = cache_path or default_cache_path()
    cache = load_cache(path) if use_cache else {}
    hit = cache.get(sig)
    if hit and hit.get("density_ctas_per_sm") in DENSITY_CHOICES and \
            hit.get("backward_ctas_per_sm") in BACKWARD_CHOICES and \
            hit.get("density_task_block") in TASK_CHOICES and \
            hit.get("backward_task_block") in TASK_CHOICES:
        grid.set_tuning(hit["density_ctas_per_sm"], hit["backward_ctas_per_sm"],
                        hit["density_task_block"], hit["backward_task_block"])
        return {**hit, "source": "cache", "signature": sig}
    if measure is None:
        if g_drho_dh is None:
            import torch
            g_drho_dh = torch.zeros_like(g_rho)
        measure = grid_measure(grid, g_rho, g_drho_dh)
    (d, b, td, tb), times = choose(measure, reps)
    grid.set_tuning(d, b, td, tb)
    entry = {"density_ctas_per_sm": d, "backward_ctas_per_sm": b, "density_task_block": td,
             "backward_task_block": tb,
             "times_ms": {k: {str(c): t for c, t in v.items()} for k, v in times.items()}}
    if use_cache:
        cache = load_cache(path)
        cache[sig] = entry
        save_cache(path, cache)
    return {**entry, "source": "timed", "signature": sig}
