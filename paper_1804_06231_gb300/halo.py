"""Halo sharding of one periodic box over ranks (one process per GPU).

The cell grid of the method (cells of edge L/nc >= H_max, Section 2) is split
into slabs of whole cell layers along x: rank r owns the layers
[x0_r, x1_r) and every particle whose cell lies in them.  A particle's density
and adjoint need only the particles of the 27 cells around its own, so a rank
that also holds one cell layer on each side of its slab (the halo, with
periodic wrap) computes its own particles exactly:

* before the sort, one halo exchange of {pos, h, m}: each rank sends the
  particles of its first and last layer to the neighbour that needs them;
* the forward pass is a gather and needs nothing more;
* before the adjoint, one halo exchange of the upstream gradients
  {dL/drho, dL/d(drho/dh)} of the same particles, in the same order, for the
  transposed term.

Each rank then runs the ordinary full-size periodic grid (same L and nc) on
its owned particles followed by its halo particles; cells outside the slab
and its halo are empty.  Every cell that an owned particle touches holds the
same particles in the same order as in the single-box grid, so the owned
results equal the single-box results.  The exchanges are torch.distributed
point-to-point messages (NCCL between GPUs, gloo on CPU); a layer needed twice
by the same rank (two slabs of a periodic box) is sent once.  Particles are
assigned to layers by the grid's own binning rule (FP64 x nc / L, truncated,
on the position wrapped into [0, L)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def wrap(x: np.ndarray, L: float) -> np.ndarray:
    """Positions wrapped into [0, L) the way the grid does (x - L floor(x/L),
    values that round to L or below 0 become 0)."""
    x = np.asarray(x, np.float64)
    inside = (x >= 0.0) & (x < L)
    y = np.where(inside, x, x - L * np.floor(x / L))
    return np.where((y >= L) | (y < 0.0), 0.0, y)


def cell_layer(x: np.ndarray, L: float, nc: int) -> np.ndarray:
    """Cell layer (0 .. nc-1) of each x coordinate under the grid's binning."""
    ci = (wrap(x, L) * (nc / L)).astype(np.int64)
    return np.clip(ci, 0, nc - 1)


@dataclass
class Slabs:
    """Layers [x0, x1) of each of `world_size` ranks: contiguous, as equal as
    possible, every rank at least one layer (so nc >= world_size)."""
    nc: int
    world_size: int
    bounds: list = field(init=False)

    def __post_init__(self):
        if self.world_size < 1:
            raise ValueError("world_size must be >= 1")
        if self.nc < 3 or self.nc < self.world_size:
            raise ValueError("need nc >= 3 and at least one cell layer per rank")
        q, r = divmod(self.nc, self.world_size)
        x0, self.bounds = 0, []
        for k in range(self.world_size):
            x1 = x0 + q + (1 if k < r else 0)
            self.bounds.append((x0, x1))
            x0 = x1

    def owner(self, layer: int) -> int:
        for k, (x0, x1) in enumerate(self.bounds):
            if x0 <= layer < x1:
                return k
        raise ValueError(f"layer {layer} outside [0, {self.nc})")

    def halo_layers(self, rank: int) -> list:
        """The layers next to the slab (periodic) that the rank does not own,
        each once, in increasing order."""
        if self.world_size == 1:
            return []
        x0, x1 = self.bounds[rank]
        need = {(x0 - 1) % self.nc, x1 % self.nc}
        return sorted(y for y in need if not (x0 <= y < x1))

    def sends(self, rank: int) -> dict:
        """{destination rank: its halo layers owned by `rank`}, destinations in
        increasing order."""
        out = {}
        for dst in range(self.world_size):
            if dst == rank:
                continue
            lay = [y for y in self.halo_layers(dst) if self.owner(y) == rank]
            if lay:
                out[dst] = lay
        return out

    def recvs(self, rank: int) -> dict:
        """{source rank: the halo layers of `rank` it owns}, sources in
        increasing order."""
        out = {}
        for y in self.halo_layers(rank):
            out.setdefault(self.owner(y), []).append(y)
        return dict(sorted(out.items()))


def owned_mask(pos: np.ndarray, L: float, slabs: Slabs, rank: int) -> np.ndarray:
    """Particles (rows of pos) whose cell layer lies in the rank's slab."""
    x0, x1 = slabs.bounds[rank]
    lay = cell_layer(pos[:, 0], L, slabs.nc)
    return (lay >= x0) & (lay < x1)


def _exchange(payload, sel_by_dst: dict, src_ranks: list, group=None):
    """Point-to-point exchange of rows of `payload` (a 2-D torch tensor):
    rows sel_by_dst[d] (an index tensor) go to rank d; from every rank in
    src_ranks a block of rows arrives.  Counts travel first (int64), then the
    rows.  Returns the received blocks concatenated in the order of src_ranks."""
    import torch
    import torch.distributed as dist
    dev = payload.device
    k = payload.shape[1]
    reqs = []
    counts = {}
    for d, sel in sel_by_dst.items():
        reqs.append(dist.isend(torch.tensor([sel.numel()], dtype=torch.int64, device=dev), d,
                               group=group))
    for s in src_ranks:
        counts[s] = torch.zeros(1, dtype=torch.int64, device=dev)
        reqs.append(dist.irecv(counts[s], s, group=group))
    for r in reqs:
        r.wait()
    reqs = []
    blocks = {}
    for d, sel in sel_by_dst.items():
        if sel.numel():
            reqs.append(dist.isend(payload.index_select(0, sel).contiguous(), d, group=group))
    for s in src_ranks:
        nrow = int(counts[s].item())
        blocks[s] = torch.empty((nrow, k), dtype=payload.dtype, device=dev)
        if nrow:
            reqs.append(dist.irecv(blocks[s], s, group=group))
    for r in reqs:
        r.wait()
    if not src_ranks:
        return torch.empty((0, k), dtype=payload.dtype, device=dev)
    return torch.cat([blocks[s] for s in src_ranks], dim=0)


class HaloDomain:
    """One rank's part of a halo-sharded box.

    Built from the rank's owned particles (pos [n, 3] float64, h [n] float32,
    m [n] float32 torch tensors, in the order the caller keeps them; all ranks
    call it together).  After construction, `pos`, `h`, `m` hold the owned
    particles followed by the halo particles (`n_owned` of the first), ready
    for a Grid((n_local, L, nc)); outputs of the first n_owned rows are the
    owned particles' exact results.  `halo_gradients` exchanges upstream
    gradients of the owned particles for the adjoint."""

    def __init__(self, slabs: Slabs, rank: int, L: float, pos, h, m, group=None):
        import torch
        self.slabs, self.rank, self.L, self.group = slabs, rank, float(L), group
        self.n_owned = int(pos.shape[0])
        dev = pos.device
        lay = torch.from_numpy(cell_layer(pos[:, 0].cpu().numpy(), self.L, slabs.nc)).to(dev)
        x0, x1 = slabs.bounds[rank]
        if self.n_owned and not bool(((lay >= x0) & (lay < x1)).all()):
            raise ValueError("a particle outside the rank's slab was passed as owned")
        # rows sent to each neighbour: its halo layers in increasing order,
        # particles of a layer in the caller's order
        self.sel = {}
        for d, layers in slabs.sends(rank).items():
            idx = [torch.nonzero(lay == y, as_tuple=False).flatten() for y in layers]
            self.sel[d] = torch.cat(idx) if idx else torch.empty(0, dtype=torch.int64, device=dev)
        self.srcs = list(slabs.recvs(rank).keys())
        payload = torch.cat([pos.to(torch.float64), h.to(torch.float64)[:, None],
                             m.to(torch.float64)[:, None]], dim=1)
        halo = _exchange(payload, self.sel, self.srcs, group) if slabs.world_size > 1 else \
            payload[:0]
        self.n_halo = int(halo.shape[0])
        self.pos = torch.cat([pos.to(torch.float64), halo[:, :3]], dim=0).contiguous()
        self.h = torch.cat([h.to(torch.float32), halo[:, 3].to(torch.float32)]).contiguous()
        self.m = torch.cat([m.to(torch.float32), halo[:, 4].to(torch.float32)]).contiguous()

    @property
    def n_local(self) -> int:
        return self.n_owned + self.n_halo

    def halo_gradients(self, g_rho, g_drho_dh):
        """Upstream gradients of the owned particles (torch [n_owned], float32
        or float64) -> the same for all local particles (owned, then halo),
        exchanged with the neighbours like the positions, dtype kept."""
        import torch
        payload = torch.stack([g_rho.to(torch.float64), g_drho_dh.to(torch.float64)], dim=1)
        halo = _exchange(payload, self.sel, self.srcs, self.group) \
            if self.slabs.world_size > 1 else payload[:0]
        return (torch.cat([g_rho, halo[:, 0].to(g_rho.dtype)]).contiguous(),
                torch.cat([g_drho_dh, halo[:, 1].to(g_drho_dh.dtype)]).contiguous())


def local_sets(slabs: Slabs, L: float, pos: np.ndarray) -> list:
    """For a box whose particles are all in one process (single-GPU runs of
    the sharded path, and checks of the exchange): per rank, the global
    indices of its local particles in the order HaloDomain builds them when
    every rank passes its owned particles in increasing global index: owned
    particles, then for each source rank in increasing order its halo layers
    in increasing order."""
    lay = cell_layer(pos[:, 0], L, slabs.nc)
    out = []
    for r in range(slabs.world_size):
        x0, x1 = slabs.bounds[r]
        owned = np.nonzero((lay >= x0) & (lay < x1))[0]
        halo = [np.nonzero(lay == y)[0] for layers in slabs.recvs(r).values() for y in layers]
        out.append((owned, np.concatenate(halo) if halo else np.zeros(0, np.int64)))
    return out
