"""Python binding of the C ABI in ``include/pv.h`` (argument marshalling only).

The functions named ``pv_*`` mirror the C entry points one to one: they take
device pointers as Python ints (e.g. ``tensor.data_ptr()``) and a CUDA stream
handle (``torch.cuda.current_stream().cuda_stream``), and raise ``PvError`` on
any status other than ``PV_OK``.  ``Grid`` wraps a ``pv_grid*`` for torch
tensors.  All computation happens in ``libpv.so``; if the library is missing
this module raises on import of the library, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpv.so")

PV_OK = 0
STATUS = {0: "PV_OK", 1: "PV_ERR_INVALID_ARGUMENT", 2: "PV_ERR_CELL_TOO_SMALL",
          3: "PV_ERR_OUT_OF_MEMORY", 4: "PV_ERR_CUDA", 5: "PV_ERR_NOT_SORTED",
          6: "PV_ERR_DEVICE", 7: "PV_ERR_TOO_LARGE"}
FLAG_SUPPORT_EXCEEDS_CELL = 1
FLAG_BAD_POSITION = 2
FLAG_BAD_SMOOTHING = 4
FLAG_CELL_OVERFLOW = 8
MAX_CELL_COUNT = 65535
GAMMA = 1.825742

#: Every symbol ``include/pv.h`` declares.
EXPORTS = ("pv_grid_create", "pv_grid_destroy", "pv_sort_cells", "pv_density",
           "pv_density_backward", "pv_count_candidates", "pv_grid_sync", "pv_grid_stats",
           "pv_status_str", "pv_last_cuda_error", "pv_density_static", "pv_grid_time_sweeps",
           "pv_grid_sweep_times", "pv_grid_set_tuning", "pv_grid_get_tuning",
           "pv_grid_set_slot_mask", "pv_raw_interactions", "pv_update_positions",
           "pv_fp32_probe", "pv_density_symmetric")
STATIC_MAX_PARTICLES = 65536
STATIC_MAX_CELLS = 4096


class PvError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class pv_box_desc(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int64), ("n", ctypes.c_int64), ("L", ctypes.c_double),
                ("nc", ctypes.c_int32)]


class pv_grid_desc(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int32), ("boxes", ctypes.POINTER(pv_box_desc)),
                ("gamma", ctypes.c_double), ("flags", ctypes.c_uint32)]


class pv_stats(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("max_cell_count", ctypes.c_int32), ("device_flags", ctypes.c_uint32),
                ("interactions", ctypes.c_int64), ("guard_pairs", ctypes.c_int64),
                ("candidates", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("candidates_adjoint", ctypes.c_int64),
                ("pairs_adjoint", ctypes.c_int64), ("orientation", (ctypes.c_int64 * 2) * 4)]


class pv_tuning(ctypes.Structure):
    _fields_ = [("density_ctas_per_sm", ctypes.c_int32), ("backward_ctas_per_sm", ctypes.c_int32),
                ("density_task_block", ctypes.c_int32), ("backward_task_block", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads ``libpv.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1804_06231_gb300.build "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    lib.pv_grid_create.argtypes = [ctypes.POINTER(pv_grid_desc), ctypes.POINTER(vp)]
    lib.pv_grid_destroy.argtypes = [vp]
    lib.pv_sort_cells.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp]
    lib.pv_density.argtypes = [vp, vp, vp, vp, vp]
    lib.pv_density_backward.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.pv_density_symmetric.argtypes = [vp, vp, vp, vp, vp]
    lib.pv_count_candidates.argtypes = [vp, vp]
    lib.pv_grid_sync.argtypes = [vp, vp]
    lib.pv_grid_stats.argtypes = [vp, ctypes.POINTER(pv_stats)]
    lib.pv_grid_time_sweeps.argtypes = [vp, i32]
    lib.pv_grid_set_slot_mask.argtypes = [vp, ctypes.c_uint32]
    lib.pv_update_positions.argtypes = [vp, vp, vp, vp]
    lib.pv_raw_interactions.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_float,
                                        ctypes.c_int32, vp, vp]
    lib.pv_fp32_probe.argtypes = [i32, i32, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                  vp]
    lib.pv_grid_set_tuning.argtypes = [vp, ctypes.POINTER(pv_tuning)]
    lib.pv_grid_get_tuning.argtypes = [vp, ctypes.POINTER(pv_tuning)]
    lib.pv_grid_sweep_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]
    for name in ("pv_grid_create", "pv_grid_destroy", "pv_sort_cells", "pv_density",
                 "pv_density_backward", "pv_count_candidates", "pv_grid_sync", "pv_grid_stats",
                 "pv_grid_time_sweeps", "pv_grid_sweep_times", "pv_grid_set_tuning",
                 "pv_grid_get_tuning", "pv_grid_set_slot_mask", "pv_raw_interactions",
                 "pv_update_positions", "pv_fp32_probe", "pv_density_symmetric"):
        getattr(lib, name).restype = i32
    lib.pv_status_str.argtypes = [i32]
    lib.pv_status_str.restype = ctypes.c_char_p
    lib.pv_density_static.argtypes = [vp, vp, vp, ctypes.c_float, ctypes.c_int64,
                                      ctypes.c_double, ctypes.c_int32, ctypes.c_double, vp, vp,
                                      vp, vp, vp]
    lib.pv_density_static.restype = i32
    lib.pv_last_cuda_error.argtypes = []
    lib.pv_last_cuda_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != PV_OK:
        detail = ""
        if status == 4:
            detail = load_library().pv_last_cuda_error().decode()
        raise PvError(status, where, detail)


# ---------------------------------------------------------------- C-ABI mirrors

def pv_status_str(status: int) -> str:
    return load_library().pv_status_str(int(status)).decode()


def pv_grid_create(boxes, gamma: float = 0.0) -> int:
    """boxes: sequence of (first, n, L, nc).  Returns the opaque grid handle."""
    arr = (pv_box_desc * len(boxes))(*[pv_box_desc(int(f), int(n), float(L), int(nc))
                                       for f, n, L, nc in boxes])
    desc = pv_grid_desc(len(boxes), arr, float(gamma), 0)
    out = ctypes.c_void_p()
    _check(load_library().pv_grid_create(ctypes.byref(desc), ctypes.byref(out)), "pv_grid_create")
    return out.value


def pv_grid_destroy(grid: int) -> None:
    _check(load_library().pv_grid_destroy(grid), "pv_grid_destroy")


def pv_sort_cells(grid: int, pos: int, h: int, m: int | None, m_uniform: float = 0.0,
                  stream: int = 0) -> None:
    _check(load_library().pv_sort_cells(grid, pos, h, m, ctypes.c_float(m_uniform), stream),
           "pv_sort_cells")


def pv_density(grid: int, rho: int, drho_dh: int | None, n_ngb: int | None,
               stream: int = 0) -> None:
    _check(load_library().pv_density(grid, rho, drho_dh, n_ngb, stream), "pv_density")


def pv_density_symmetric(grid: int, rho: int, drho_dh: int | None, n_ngb: int | None,
                         stream: int = 0) -> None:
    _check(load_library().pv_density_symmetric(grid, rho, drho_dh, n_ngb, stream),
           "pv_density_symmetric")


def pv_density_backward(grid: int, g_rho: int, g_drho_dh: int | None, g_pos: int,
                        g_h: int | None, stream: int = 0) -> None:
    _check(load_library().pv_density_backward(grid, g_rho, g_drho_dh, g_pos, g_h, stream),
           "pv_density_backward")


def pv_count_candidates(grid: int, stream: int = 0) -> None:
    _check(load_library().pv_count_candidates(grid, stream), "pv_count_candidates")


def pv_grid_sync(grid: int, stream: int = 0) -> None:
    _check(load_library().pv_grid_sync(grid, stream), "pv_grid_sync")


def pv_density_static(pos: int, h: int, m: int | None, m_uniform: float, n: int, L: float,
                      nc: int, gamma: float, rho: int, drho_dh: int | None, n_ngb: int | None,
                      flags_out: int | None = None, stream: int = 0) -> None:
    """One box, no allocation: see the header (fixed device scratch, shared by all calls)."""
    _check(load_library().pv_density_static(pos, h, m, ctypes.c_float(m_uniform), int(n),
                                            float(L), int(nc), float(gamma), rho, drho_dh,
                                            n_ngb, flags_out, stream), "pv_density_static")


def pv_grid_set_tuning(grid: int, density_ctas_per_sm: int = 0, backward_ctas_per_sm: int = 0,
                       density_task_block: int = 0, backward_task_block: int = 0) -> None:
    t = pv_tuning(int(density_ctas_per_sm), int(backward_ctas_per_sm), int(density_task_block),
                  int(backward_task_block))
    _check(load_library().pv_grid_set_tuning(grid, ctypes.byref(t)), "pv_grid_set_tuning")


def pv_grid_get_tuning(grid: int) -> tuple[int, int, int, int]:
    """(density CTAs per SM, adjoint CTAs per SM, density task block, adjoint task block)"""
    t = pv_tuning()
    _check(load_library().pv_grid_get_tuning(grid, ctypes.byref(t)), "pv_grid_get_tuning")
    return (t.density_ctas_per_sm, t.backward_ctas_per_sm, t.density_task_block,
            t.backward_task_block)


SLOT_MASK_ALL = (1 << 27) - 1
FLAG_SKIN_EXCEEDED = 16
FLAG_BAD_GRADIENT = 32


def pv_update_positions(grid: int, pos: int, h: int, stream: int = 0) -> None:
    _check(load_library().pv_update_positions(grid, pos, h, stream), "pv_update_positions")


def pv_raw_interactions(xi: int, n_i: int, xj: int, n_j: int, H: float, reps: int, out: int,
                        stream: int = 0) -> None:
    _check(load_library().pv_raw_interactions(xi, int(n_i), xj, int(n_j), ctypes.c_float(H),
                                              int(reps), out, stream), "pv_raw_interactions")


def pv_fp32_probe(packed: int, iters: int, sink: int, threads: int, stream: int = 0) -> float:
    """Queues the FP32 throughput probe; returns its FP32 operations (FMA = 2)."""
    flops = ctypes.c_double(0.0)
    _check(load_library().pv_fp32_probe(int(packed), int(iters), sink, int(threads),
                                        ctypes.byref(flops), stream), "pv_fp32_probe")
    return flops.value


def raw_interactions(xi, xj, H: float, reps: int = 1, out=None, stream=None):
    """Torch front end of pv_raw_interactions: xi [n_i, 4], xj [n_j, 4] float32
    CUDA tensors {x, y, z, m}; returns [n_i, 2] {sum m wh, sum m th}."""
    import torch
    if out is None:
        out = torch.empty((xi.shape[0], 2), dtype=torch.float32, device=xi.device)
    for t, name in ((xi, "xi"), (xj, "xj"), (out, "out")):
        Grid._dev(t, torch.float32, None, name)
    st = torch.cuda.current_stream().cuda_stream if stream is None else \
        getattr(stream, "cuda_stream", stream)
    pv_raw_interactions(xi.data_ptr(), xi.shape[0], xj.data_ptr(), xj.shape[0], H, reps,
                        out.data_ptr(), st)
    return out


def pv_grid_set_slot_mask(grid: int, mask: int) -> None:
    _check(load_library().pv_grid_set_slot_mask(grid, int(mask)), "pv_grid_set_slot_mask")


def slot_mask_of_class(cls: int) -> int:
    """Mask of the slots of one orientation class (0 self, 1 face, 2 edge, 3 corner)."""
    m = 0
    for o in range(27):
        ox, oy, oz = o // 9 - 1, (o // 3) % 3 - 1, o % 3 - 1
        if ox * ox + oy * oy + oz * oz == cls:
            m |= 1 << o
    return m


def pv_grid_time_sweeps(grid: int, enable: bool) -> None:
    _check(load_library().pv_grid_time_sweeps(grid, 1 if enable else 0), "pv_grid_time_sweeps")


def pv_grid_sweep_times(grid: int):
    """((ms density, ms adjoint), (launches density, launches adjoint)) since the last reset."""
    ms = (ctypes.c_double * 2)()
    nl = (ctypes.c_int64 * 2)()
    _check(load_library().pv_grid_sweep_times(grid, ms, nl), "pv_grid_sweep_times")
    return (ms[0], ms[1]), (nl[0], nl[1])


@dataclass
class Stats:
    n_particles: int
    n_cells: int
    max_cell_count: int
    device_flags: int
    interactions: int
    guard_pairs: int
    candidates: int
    device_bytes: int
    kernel_launches: int
    candidates_adjoint: int
    pairs_adjoint: int
    orientation: list  # [4][2]: (self, face, edge, corner) x (candidates, interactions)


def pv_grid_stats(grid: int, raise_on_flags: bool = True) -> Stats:
    st = pv_stats()
    status = load_library().pv_grid_stats(grid, ctypes.byref(st))
    vals = [getattr(st, f) for f, _ in pv_stats._fields_]
    vals[-1] = [[int(st.orientation[c][0]), int(st.orientation[c][1])] for c in range(4)]
    out = Stats(*vals)
    if status != PV_OK and (raise_on_flags or status != 6):
        raise PvError(status, "pv_grid_stats", f"device_flags={out.device_flags}")
    return out


# ---------------------------------------------------------------- torch wrapper

class Grid:
    """A ``pv_grid`` for particles held in torch tensors on the current device.

    ``boxes`` is a sequence of ``(n, L, nc)`` (or one tuple): the particles of
    box b are the next ``n`` rows of the arrays passed to ``sort``.
    """

    def __init__(self, boxes, gamma: float = GAMMA):
        if isinstance(boxes, tuple) and len(boxes) == 3 and not isinstance(boxes[0], tuple):
            boxes = [boxes]
        first, descs = 0, []
        for n, L, nc in boxes:
            descs.append((first, int(n), float(L), int(nc)))
            first += int(n)
        self.n = first
        self.boxes = descs
        self.gamma = float(gamma)
        self.handle = pv_grid_create(descs, gamma)

    def close(self) -> None:
        if getattr(self, "handle", None):
            pv_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _stream(stream):
        import torch
        if stream is None:
            return torch.cuda.current_stream().cuda_stream
        return getattr(stream, "cuda_stream", stream)

    @staticmethod
    def _dev(t, dtype, shape=None, name=""):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        return t.data_ptr()

    def sort(self, pos, h, m=None, m_uniform: float = 0.0, stream=None) -> None:
        import torch
        p = self._dev(pos, torch.float64, (self.n, 3), "pos")
        hp = self._dev(h, torch.float32, (self.n,), "h")
        mp = None if m is None else self._dev(m, torch.float32, (self.n,), "m")
        pv_sort_cells(self.handle, p, hp, mp, m_uniform, self._stream(stream))

    def update(self, pos, h, stream=None) -> None:
        """New positions and smoothing lengths, keeping the last sort (windows
        widen by twice the largest displacement since it)."""
        import torch
        p = self._dev(pos, torch.float64, (self.n, 3), "pos")
        hp = self._dev(h, torch.float32, (self.n,), "h")
        pv_update_positions(self.handle, p, hp, self._stream(stream))

    def density(self, rho=None, drho_dh=None, n_ngb=None, stream=None, symmetric=False):
        """pv_density (or, with symmetric=True, pv_density_symmetric)."""
        import torch
        if rho is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            rho = torch.empty(self.n, dtype=torch.float32, device=dev)
            drho_dh = torch.empty(self.n, dtype=torch.float32, device=dev)
            n_ngb = torch.empty(self.n, dtype=torch.int32, device=dev)
        (pv_density_symmetric if symmetric else pv_density)(
                   self.handle, self._dev(rho, torch.float32, (self.n,), "rho"),
                   None if drho_dh is None else self._dev(drho_dh, torch.float32, (self.n,),
                                                          "drho_dh"),
                   None if n_ngb is None else self._dev(n_ngb, torch.int32, (self.n,), "n_ngb"),
                   self._stream(stream))
        return rho, drho_dh, n_ngb

    def backward(self, g_rho, g_drho_dh=None, g_pos=None, g_h=None, stream=None):
        import torch
        if g_pos is None:
            g_pos = torch.empty((self.n, 3), dtype=torch.float32, device=g_rho.device)
            g_h = torch.empty(self.n, dtype=torch.float32, device=g_rho.device)
        pv_density_backward(
            self.handle, self._dev(g_rho, torch.float32, (self.n,), "g_rho"),
            None if g_drho_dh is None else self._dev(g_drho_dh, torch.float32, (self.n,),
                                                     "g_drho_dh"),
            self._dev(g_pos, torch.float32, (self.n, 3), "g_pos"),
            None if g_h is None else self._dev(g_h, torch.float32, (self.n,), "g_h"),
            self._stream(stream))
        return g_pos, g_h

    def count_candidates(self, stream=None) -> int:
        pv_count_candidates(self.handle, self._stream(stream))
        return pv_grid_stats(self.handle).candidates

    def sync(self, stream=None) -> None:
        pv_grid_sync(self.handle, self._stream(stream))

    def set_tuning(self, density_ctas_per_sm: int = 0, backward_ctas_per_sm: int = 0,
                   density_task_block: int | None = None,
                   backward_task_block: int | None = None) -> None:
        """CTAs per SM of the two cell-centric sweep kernels (0 = default) and
        particles per task of the two task kernels (64, 128 or 256; 0 =
        default, None = keep the current value)."""
        cur = self.tuning()
        pv_grid_set_tuning(self.handle, density_ctas_per_sm, backward_ctas_per_sm,
                           cur[2] if density_task_block is None else density_task_block,
                           cur[3] if backward_task_block is None else backward_task_block)

    def tuning(self) -> tuple[int, int, int, int]:
        """(density CTAs per SM, adjoint CTAs per SM, density task block,
        adjoint task block)"""
        return pv_grid_get_tuning(self.handle)

    def set_slot_mask(self, mask: int = SLOT_MASK_ALL) -> None:
        """Visit only the neighbour slots in `mask` (measurement aid)."""
        pv_grid_set_slot_mask(self.handle, mask)

    def time_sweeps(self, enable: bool = True) -> None:
        """Start (or stop) timing the sweep kernels with CUDA events; resets the totals."""
        pv_grid_time_sweeps(self.handle, enable)

    def sweep_times(self):
        """Mean sweep-kernel time in ms per launch: (density, adjoint); NaN if none."""
        (a, b), (na, nb) = pv_grid_sweep_times(self.handle)
        return (a / na if na else float("nan"), b / nb if nb else float("nan"))

    def stats(self, raise_on_flags: bool = True) -> Stats:
        return pv_grid_stats(self.handle, raise_on_flags)
