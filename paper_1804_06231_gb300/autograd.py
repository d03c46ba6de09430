"""``torch.autograd.Function`` around pv_sort_cells / pv_density / pv_density_backward.

``PVDensity.apply(pos, h, m, grid)`` returns ``(rho, drho_dh, n_ngb)`` and
back-propagates ``dL/drho`` and ``dL/d(drho_dh)`` to ``dL/dpos`` and ``dL/dh``
through the adjoint kernel (masses are constants).  The grid keeps the sorted
cells of the forward pass; if the same grid was re-sorted for other inputs
before ``backward`` runs, the saved inputs are sorted again first.
"""
from __future__ import annotations

import torch

from .pv import Grid


class PVDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos: torch.Tensor, h: torch.Tensor, m: torch.Tensor | None, grid: Grid):
        pos_d, h_d = pos.detach().contiguous(), h.detach().contiguous()
        m_d = None if m is None else m.detach().contiguous()
        grid.sort(pos_d, h_d, m_d)
        grid._version = getattr(grid, "_version", 0) + 1
        rho, drho_dh, n_ngb = grid.density()
        ctx.grid = grid
        ctx.version = grid._version
        ctx.save_for_backward(pos_d, h_d, *( [] if m_d is None else [m_d]))
        ctx.has_m = m_d is not None
        ctx.mark_non_differentiable(n_ngb)
        return rho, drho_dh, n_ngb

    @staticmethod
    def backward(ctx, g_rho, g_drho_dh, _g_n):
        grid: Grid = ctx.grid
        saved = ctx.saved_tensors
        if getattr(grid, "_version", 0) != ctx.version:
            grid.sort(saved[0], saved[1], saved[2] if ctx.has_m else None)
            grid._version = ctx.version
        n = grid.n
        dev = saved[0].device
        if g_rho is None:
            g_rho = torch.zeros(n, dtype=torch.float32, device=dev)
        g_rho = g_rho.detach().to(torch.float32).contiguous()
        g_d = None if g_drho_dh is None else g_drho_dh.detach().to(torch.float32).contiguous()
        g_pos, g_h = grid.backward(g_rho, g_d)
        return g_pos.to(saved[0].dtype), g_h.to(saved[1].dtype), None, None


def density(pos, h, m=None, grid: Grid | None = None, boxes=None):
    """Differentiable density of one or more periodic boxes.

    ``grid`` (a ``Grid``) is reused when given, else built from ``boxes``
    (``(n, L, nc)`` tuples).
    """
    if grid is None:
        grid = Grid(boxes)
    return PVDensity.apply(pos, h, m, grid)
