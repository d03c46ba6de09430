"""Seeded synthetic particle sets for the pseudo-Verlet SPH density loop.

This module only *draws* inputs: positions, smoothing lengths, masses, loss
weights and the cell-grid size that goes with them.  It contains none of the
method's arithmetic (no kernel, no neighbour search, no density), so that the
FP64 oracle under ``oracle/`` and the CUDA path can both be fed from it
without sharing any computation.

Every workload is a periodic cube ``[0, L)^3`` (``L = 1`` unless stated).
Positions are float64, smoothing lengths ``h`` are rounded to float32 once
(both sides consume exactly those values) and masses are float32.

Workloads (the paper's own benchmark, SWIFT's ``test27cells`` of Section 4,
is not available; these synthetic sets stand in for it):

* ``uniform``     -- positions U[0,1)^3, ``h_i = 1.2348 N^(-1/3) U(0.9, 1.1)``,
                     ``m = 1/N``.
* ``clustered``   -- 64 isotropic Gaussians (sigma ~ U(0.01, 0.05), centres
                     uniform, equal weights) plus a 20 % uniform background,
                     wrapped into the unit cube; ``h_i = 1.2348 (m /
                     rho_analytic(x_i))^(1/3)`` from the mixture's analytic
                     density.
* ``lattice``     -- a simple cubic lattice with constant ``h = 1.2348 a``.
* ``test27cells`` -- 27 cells of 216 uniform random particles each, the shape
                     of the paper's benchmark (Section 4).
* ``multibox``    -- 64 independent unit boxes, ``N_b`` log-uniform in
                     [4096, 524288], each uniform or clustered by coin flip.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: Ratio of kernel support to smoothing length, ``H = GAMMA * h``.
GAMMA = 1.825742
#: Resolution parameter ``eta`` in ``h = eta * (m / rho)^(1/3)``.
ETA = 1.2348

#: Fixed seeds of the named workloads.
SEEDS = {"cfg0": 0, "cfg1": 1, "cfg2": 2, "cfg3": 3, "cfg4": 4,
         "lattice": 5, "test27cells": 6}


@dataclass
class Box:
    """One periodic particle set and the cell grid it is binned on."""
    pos: np.ndarray          # float64 [n, 3], in [0, L)
    h: np.ndarray            # float32 [n]
    m: np.ndarray            # float32 [n]
    L: float = 1.0
    nc: int = 3              # cells per dimension (cubic cells, edge L/nc)
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def H_max(self) -> float:
        return float(GAMMA * np.float64(self.h.max())) if self.n else 0.0


def finest_nc(h: np.ndarray, L: float = 1.0, gamma: float = GAMMA,
              cap: int | None = None) -> int:
    """Largest ``nc`` whose cell edge ``L/nc`` is still >= the largest support."""
    if h.size == 0:
        return 3
    H_max = gamma * float(np.float64(h.max()))
    nc = int(math.floor(L / H_max * (1.0 - 1e-12)))
    # guard against rounding of L/nc below H_max
    while nc > 3 and L / nc < H_max:
        nc -= 1
    if cap is not None:
        nc = min(nc, cap)
    return max(nc, 3)


def nc_for_occupancy(n: int, target: float, h: np.ndarray, L: float = 1.0,
                     gamma: float = GAMMA) -> int:
    """``nc`` giving about ``target`` particles per cell, never finer than allowed."""
    nc = max(3, int(round((n / max(target, 1e-9)) ** (1.0 / 3.0))))
    return min(nc, finest_nc(h, L, gamma))


def _wrap(pos: np.ndarray, L: float = 1.0) -> np.ndarray:
    pos = np.mod(pos, L)
    pos[pos >= L] = 0.0          # np.mod can return L for tiny negatives
    return pos


def uniform(n: int, seed: int, nc: int | None = None, eta: float = ETA,
            spread: float = 0.1, L: float = 1.0) -> Box:
    """Uniform random positions, ``h = eta * (L^3/n)^(1/3) * U(1-spread, 1+spread)``."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    pos = _wrap(pos, L)
    base = eta * L * n ** (-1.0 / 3.0) if n > 0 else 0.0
    h = (base * rng.uniform(1.0 - spread, 1.0 + spread, n)).astype(np.float32)
    m = np.full(n, 1.0 / max(n, 1), dtype=np.float32)
    box = Box(pos, h, m, L, 3, f"uniform{n}")
    box.nc = nc if nc is not None else finest_nc(h, L)
    return box


@dataclass
class Mixture:
    centres: np.ndarray      # [K, 3]
    sigmas: np.ndarray       # [K]
    bg_frac: float


def draw_mixture(rng: np.random.Generator, k: int = 64, bg_frac: float = 0.2,
                 sigma_lo: float = 0.01, sigma_hi: float = 0.05) -> Mixture:
    centres = rng.random((k, 3))
    sigmas = rng.uniform(sigma_lo, sigma_hi, k)
    return Mixture(centres, sigmas, bg_frac)


def mixture_density(x: np.ndarray, mix: Mixture, chunk: int = 1 << 16) -> np.ndarray:
    """Analytic number density of the periodic mixture (unit total mass).

    ``rho(x) = bg + (1-bg)/K * sum_k N(x; c_k, sigma_k^2 I)`` with each Gaussian
    wrapped periodically.  Only the nearest periodic image of each Gaussian is
    summed: with sigma <= 0.05 the next image is >= 0.5 away and contributes
    less than exp(-50) of the peak.
    """
    k = mix.centres.shape[0]
    out = np.empty(x.shape[0], dtype=np.float64)
    norm = (2.0 * np.pi * mix.sigmas ** 2) ** -1.5            # [K]
    inv2s2 = 0.5 / mix.sigmas ** 2
    w = (1.0 - mix.bg_frac) / k
    for s in range(0, x.shape[0], chunk):
        xs = x[s:s + chunk]
        acc = np.zeros(xs.shape[0])
        for c in range(k):
            d = xs - mix.centres[c]
            d -= np.rint(d)
            r2 = np.einsum("ij,ij->i", d, d)
            acc += norm[c] * np.exp(-r2 * inv2s2[c])
        out[s:s + chunk] = mix.bg_frac + w * acc
    return out


def clustered(n: int, seed: int, nc: int | None = None, eta: float = ETA,
              k: int = 64, bg_frac: float = 0.2) -> Box:
    """Gaussian-mixture positions with ``h`` from the mixture's analytic density."""
    rng = np.random.default_rng(seed)
    mix = draw_mixture(rng, k, bg_frac)
    n_bg = int(round(bg_frac * n))
    comp = rng.integers(0, k, n - n_bg)
    pos = np.empty((n, 3))
    pos[:n_bg] = rng.random((n_bg, 3))
    pos[n_bg:] = mix.centres[comp] + rng.standard_normal((n - n_bg, 3)) * mix.sigmas[comp, None]
    pos = _wrap(pos)
    perm = rng.permutation(n)          # interleave background and clusters
    pos = np.ascontiguousarray(pos[perm])
    m = np.full(n, 1.0 / n, dtype=np.float32)
    rho = mixture_density(pos, mix)
    h = (eta * (np.float64(1.0 / n) / rho) ** (1.0 / 3.0)).astype(np.float32)
    box = Box(pos, h, m, 1.0, 3, f"clustered{n}", {"mixture": mix})
    box.nc = nc if nc is not None else finest_nc(h)
    return box


def lattice(n_side: int, nc: int | None = None, eta: float = ETA,
            shift: float = 0.25) -> Box:
    """Simple cubic lattice of ``n_side^3`` points, spacing ``a = 1/n_side``.

    Points sit at ``(i + shift) a`` so that none lies on a cell face when
    ``nc`` divides ``n_side``.
    """
    a = 1.0 / n_side
    g = (np.arange(n_side) + shift) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).copy()
    n = pos.shape[0]
    h = np.full(n, eta * a, dtype=np.float32)
    m = np.full(n, 1.0 / n, dtype=np.float32)
    box = Box(pos, h, m, 1.0, 3, f"lattice{n_side}")
    box.nc = nc if nc is not None else finest_nc(h)
    return box


def test27cells(seed: int = SEEDS["test27cells"], per_cell: int = 216) -> Box:
    """27 cells (3^3 grid) of ``per_cell`` uniform random particles each.

    Smoothing lengths follow the uniform rule for the total count, which keeps
    ``H_max`` below the cell edge 1/3.
    """
    rng = np.random.default_rng(seed)
    n = 27 * per_cell
    cells = np.stack(np.meshgrid(np.arange(3), np.arange(3), np.arange(3),
                                 indexing="ij"), -1).reshape(-1, 3)
    pos = (np.repeat(cells, per_cell, 0) + rng.random((n, 3))) / 3.0
    pos = _wrap(pos)
    h = (ETA * n ** (-1.0 / 3.0) * rng.uniform(0.9, 1.1, n)).astype(np.float32)
    m = np.full(n, 1.0 / n, dtype=np.float32)
    return Box(pos, h, m, 1.0, 3, "test27cells")


def loss_weights(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Weights ``w, v ~ N(0,1)`` of ``L = sum w_i (rho_i - 1)^2 + sum v_i drho/dh_i``."""
    rng = np.random.default_rng(seed + 1000)
    return rng.standard_normal(n), rng.standard_normal(n)


def cfg0(seed: int = SEEDS["cfg0"]) -> Box:
    """N = 32768 uniform, 12^3 cells (about 19 per cell)."""
    b = uniform(32768, seed, nc=12)
    b.name = "uniform-32768-nc12"
    return b


def cfg1(seed: int = SEEDS["cfg1"]) -> Box:
    """N = 1048576 uniform, 15^3 cells (about 311 per cell)."""
    b = uniform(1 << 20, seed, nc=15)
    b.name = "uniform-1048576-nc15"
    return b


def cfg2(seed: int = SEEDS["cfg2"], n: int = 1 << 22) -> Box:
    """N = 4194304 clustered, finest grid for the global H_max."""
    b = clustered(n, seed)
    b.name = f"clustered-{n}-nc{b.nc}"
    return b


def cfg3(seed: int = SEEDS["cfg3"], n: int = 1 << 18) -> Box:
    """N = 262144 uniform (differentiation workload), finest grid."""
    b = uniform(n, seed)
    b.name = f"uniform-{n}-nc{b.nc}"
    return b


def multibox(seed: int = SEEDS["cfg4"], n_boxes: int = 64, n_lo: int = 4096,
             n_hi: int = 524288, scale: float = 1.0) -> list[Box]:
    """Independent unit boxes, ``N_b`` log-uniform in [n_lo, n_hi] (times ``scale``)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_boxes))
    sizes = np.maximum((sizes * scale).astype(np.int64), 64)
    kinds = rng.integers(0, 2, n_boxes)
    sub = rng.integers(0, 2 ** 31, n_boxes)
    boxes = []
    for b in range(n_boxes):
        if kinds[b] == 0:
            bx = uniform(int(sizes[b]), int(sub[b]))
        else:
            bx = clustered(int(sizes[b]), int(sub[b]))
        bx.name = f"box{b}-{bx.name}"
        boxes.append(bx)
    return boxes
