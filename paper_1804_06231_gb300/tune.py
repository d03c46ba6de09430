"""Autotuner for the launch shape of the two sweep kernels, with a JSON cache.

The only free parameter of the sweep launches is the number of resident CTAs
per SM of each cell-centric kernel (``pv_grid_set_tuning``).  It trades
occupancy against shared memory per CTA, and the shared memory decides which
cells are swept by the cell-centric kernel and which by the task kernel, so
the best value depends on the workload: uniform boxes with small cells favour
more CTAs, clustered boxes with dense cells favour more shared memory.

``autotune`` times ``pv_density`` and ``pv_density_backward`` (the whole
call, CUDA events on the current stream, median of ``reps``) for every
candidate on an already sorted grid, keeps the fastest per pass and stores it
under the workload's signature, so that later grids of the same shape reuse
it without timing.  Results do not depend on the choice beyond FP32 summation
order.
"""
from __future__ import annotations

import json
import math
import os
import statistics

DENSITY_CHOICES = (2, 3, 4)
BACKWARD_CHOICES = (1, 2, 3)
DEFAULT = (3, 3)


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


def choose(measure, reps: int = 5) -> tuple[tuple[int, int], dict]:
    """Runs ``measure(density_ctas, backward_ctas, reps)`` -> (ms_density,
    ms_backward) for every combination the passes need and returns the
    fastest (density, backward) pair with the timings.  The passes are
    independent, so the density choices are timed with the default backward
    shape and vice versa."""
    times = {"density": {}, "backward": {}}
    for d in DENSITY_CHOICES:
        times["density"][d] = measure(d, DEFAULT[1], reps)[0]
    for b in BACKWARD_CHOICES:
        times["backward"][b] = measure(DEFAULT[0], b, reps)[1]
    best_d = min(DENSITY_CHOICES, key=lambda d: (times["density"][d], d != DEFAULT[0]))
    best_b = min(BACKWARD_CHOICES, key=lambda b: (times["backward"][b], b != DEFAULT[1]))
    return (best_d, best_b), times


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

    def measure(d, b, reps):
        grid.set_tuning(d, b)
        tf = timed(lambda: grid.density(rho, D, nn), reps)
        tb = timed(lambda: grid.backward(g_rho, g_drho_dh, gp, gh), reps)
        return tf, tb

    return measure


def autotune(grid, g_rho, g_drho_dh=None, reps: int = 5, cache_path: str | None = None,
             use_cache: bool = True, measure=None, device_info=None) -> dict:
    """Picks and sets the launch shape of a sorted grid.  Returns
    {"density_ctas_per_sm", "backward_ctas_per_sm", "source": "cache"|"timed",
    "signature", "times_ms"}.  ``device_info`` = (name, SM count), read from
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
            hit.get("backward_ctas_per_sm") in BACKWARD_CHOICES:
        grid.set_tuning(hit["density_ctas_per_sm"], hit["backward_ctas_per_sm"])
        return {**hit, "source": "cache", "signature": sig}
    if measure is None:
        if g_drho_dh is None:
            import torch
            g_drho_dh = torch.zeros_like(g_rho)
        measure = grid_measure(grid, g_rho, g_drho_dh)
    (d, b), times = choose(measure, reps)
    grid.set_tuning(d, b)
    entry = {"density_ctas_per_sm": d, "backward_ctas_per_sm": b,
             "times_ms": {k: {str(c): t for c, t in v.items()} for k, v in times.items()}}
    if use_cache:
        cache = load_cache(path)
        cache[sig] = entry
        save_cache(path, cache)
    return {**entry, "source": "timed", "signature": sig}
