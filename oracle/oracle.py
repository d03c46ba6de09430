"""ctypes front end of the FP64 oracle (``pv_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).  Every
function here converts its arguments to float64 numpy arrays, calls the C
routine and returns numpy arrays.  See ``pv_oracle.c`` for what each routine
computes and which part of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
GAMMA_DEFAULT = 1.825742

_lib = None


def build(force: bool = False) -> str:
    """Compile ``pv_oracle.c`` with gcc (OpenMP) into ``liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        for name in ("or_w", "or_dw", "or_d2w"):
            getattr(lib, name).restype = d
            getattr(lib, name).argtypes = [d]
        lib.or_W.restype = d; lib.or_W.argtypes = [d, d]
        lib.or_W_r.restype = d; lib.or_W_r.argtypes = [d, d]
        for name in ("or_W_h", "or_W_hh", "or_W_hr"):
            getattr(lib, name).restype = d
            getattr(lib, name).argtypes = [d, d, d]
        lib.or_max_threads.restype = i32
        lib.or_density_brute.restype = None
        lib.or_density_brute.argtypes = [i64, p, p, p, d, d, p, p, p, p, p, i32]
        lib.or_density_cells.restype = i32
        lib.or_density_cells.argtypes = [i64, p, p, p, d, i32, d, p, p, p, p, p, i32]
        lib.or_density_pv.restype = i32
        lib.or_density_pv.argtypes = [i64, p, p, p, d, i32, d, p, p, p, p, p, p, i32]
        lib.or_backward_brute.restype = None
        lib.or_backward_brute.argtypes = [i64, p, p, p, d, d, p, p, p, p, i32]
        lib.or_backward_cells.restype = i32
        lib.or_backward_cells.argtypes = [i64, p, p, p, d, i32, d, p, p, p, p, i32]
        lib.or_backward_pv.restype = i32
        lib.or_backward_pv.argtypes = [i64, p, p, p, d, i32, d, p, p, p, p, i32]
        lib.or_adjoint_counts.restype = i32
        lib.or_adjoint_counts.argtypes = [i64, p, p, d, i32, d, p, i32]
        lib.or_fd_loss.restype = d
        lib.or_fd_loss.argtypes = [i64, p, p, p, d, d, p, p, i64, i32, d]
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Kernel
# --------------------------------------------------------------------------

def w(q: float) -> float:
    """Cubic-spline shape function w(q), including the 8/pi factor."""
    return _load().or_w(float(q))


def dw(q: float) -> float:
    return _load().or_dw(float(q))


def d2w(q: float) -> float:
    return _load().or_d2w(float(q))


def W(r: float, H: float) -> float:
    return _load().or_W(float(r), float(H))


def W_h(r: float, h: float, gamma: float = GAMMA_DEFAULT) -> float:
    return _load().or_W_h(float(r), float(h), float(gamma))


def W_hh(r: float, h: float, gamma: float = GAMMA_DEFAULT) -> float:
    return _load().or_W_hh(float(r), float(h), float(gamma))


def W_r(r: float, H: float) -> float:
    return _load().or_W_r(float(r), float(H))


def W_hr(r: float, h: float, gamma: float = GAMMA_DEFAULT) -> float:
    return _load().or_W_hr(float(r), float(h), float(gamma))


def max_threads() -> int:
    return int(_load().or_max_threads())


# --------------------------------------------------------------------------
# Density
# --------------------------------------------------------------------------

@dataclass
class Density:
    rho: np.ndarray       # float64 [n]
    drho_dh: np.ndarray   # float64 [n]
    n_ngb: np.ndarray     # int32 [n]
    S: np.ndarray         # float64 [n]  sum_j m_j |dW/dh|, the scale of drho_dh
    band: np.ndarray      # int32 [n]  pairs with |r/H_i - 1| < 1e-6 (j != i)
    counters: np.ndarray | None = None   # int64 [4, 2] (self/face/edge/corner; cand, inter)


def _outs(n):
    return (np.zeros(n), np.zeros(n), np.zeros(n, np.int32), np.zeros(n),
            np.zeros(n, np.int32))


_ERR = {-1: "out of memory", -2: "nc < 3", -3: "H_max exceeds the cell edge"}


def density_brute(pos, h, m, L=1.0, gamma=GAMMA_DEFAULT, threads=0) -> Density:
    """O(N^2) definition of rho, drho/dh and n with minimum-image distances."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m)
    rho, D, nn, S, band = _outs(n)
    _load().or_density_brute(n, _ptr(pos), _ptr(h), _ptr(m), float(L), float(gamma),
                             _ptr(rho), _ptr(D), _ptr(nn), _ptr(S), _ptr(band), int(threads))
    return Density(rho, D, nn, S, band)


def density_cells(pos, h, m, L=1.0, nc=3, gamma=GAMMA_DEFAULT, threads=0) -> Density:
    """Cell list: every pair in the 27 neighbouring cells is tested."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m)
    rho, D, nn, S, band = _outs(n)
    rc = _load().or_density_cells(n, _ptr(pos), _ptr(h), _ptr(m), float(L), int(nc),
                                  float(gamma), _ptr(rho), _ptr(D), _ptr(nn), _ptr(S),
                                  _ptr(band), int(threads))
    if rc:
        raise ValueError(f"oracle density_cells: {_ERR.get(rc, rc)}")
    return Density(rho, D, nn, S, band)


def density_pv(pos, h, m, L=1.0, nc=3, gamma=GAMMA_DEFAULT, threads=0) -> Density:
    """Pseudo-Verlet sorted sweep (13 axes, trimmed one-sided pair windows)."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m)
    rho, D, nn, S, band = _outs(n)
    cnt = np.zeros((4, 2), np.int64)
    rc = _load().or_density_pv(n, _ptr(pos), _ptr(h), _ptr(m), float(L), int(nc), float(gamma),
                               _ptr(rho), _ptr(D), _ptr(nn), _ptr(S), _ptr(band), _ptr(cnt),
                               int(threads))
    if rc:
        raise ValueError(f"oracle density_pv: {_ERR.get(rc, rc)}")
    return Density(rho, D, nn, S, band, cnt)


# --------------------------------------------------------------------------
# Adjoint
# --------------------------------------------------------------------------

def backward_brute(pos, h, m, g_rho, g_D, L=1.0, gamma=GAMMA_DEFAULT, threads=0):
    """O(N^2) adjoint: returns (dL/dx [n,3], dL/dh [n])."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m); g_rho = _f64(g_rho); g_D = _f64(g_D)
    gp = np.zeros((n, 3)); gh = np.zeros(n)
    _load().or_backward_brute(n, _ptr(pos), _ptr(h), _ptr(m), float(L), float(gamma),
                              _ptr(g_rho), _ptr(g_D), _ptr(gp), _ptr(gh), int(threads))
    return gp, gh


def backward_cells(pos, h, m, g_rho, g_D, L=1.0, nc=3, gamma=GAMMA_DEFAULT, threads=0):
    """Cell-list adjoint: returns (dL/dx [n,3], dL/dh [n])."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m); g_rho = _f64(g_rho); g_D = _f64(g_D)
    gp = np.zeros((n, 3)); gh = np.zeros(n)
    rc = _load().or_backward_cells(n, _ptr(pos), _ptr(h), _ptr(m), float(L), int(nc),
                                   float(gamma), _ptr(g_rho), _ptr(g_D), _ptr(gp), _ptr(gh),
                                   int(threads))
    if rc:
        raise ValueError(f"oracle backward_cells: {_ERR.get(rc, rc)}")
    return gp, gh


def backward_pv(pos, h, m, g_rho, g_D, L=1.0, nc=3, gamma=GAMMA_DEFAULT, threads=0):
    """Adjoint by the pseudo-Verlet sweep (windows widened to max(H_i, Hmax_b)):
    returns (dL/dx [n,3], dL/dh [n]); equal to backward_cells up to summation
    order, and fast on dense clustered cells."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m); g_rho = _f64(g_rho); g_D = _f64(g_D)
    gp = np.zeros((n, 3)); gh = np.zeros(n)
    rc = _load().or_backward_pv(n, _ptr(pos), _ptr(h), _ptr(m), float(L), int(nc),
                                float(gamma), _ptr(g_rho), _ptr(g_D), _ptr(gp), _ptr(gh),
                                int(threads))
    if rc:
        raise ValueError(f"oracle backward_pv: {_ERR.get(rc, rc)}")
    return gp, gh


def loss_upstream(rho, w_weights, v_weights):
    """dL/drho and dL/d(drho/dh) of L = sum w (rho - 1)^2 + sum v drho/dh."""
    return 2.0 * np.asarray(w_weights) * (np.asarray(rho) - 1.0), np.asarray(v_weights, float)


def fd_loss_grad(pos, h, m, w_weights, v_weights, p, comp, delta=1e-6, L=1.0,
                 gamma=GAMMA_DEFAULT) -> float:
    """Central difference of L w.r.t. x_p[comp] (0..2) or h_p (comp = 3)."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h); m = _f64(m)
    wv = _f64(w_weights); vv = _f64(v_weights)
    return float(_load().or_fd_loss(n, _ptr(pos), _ptr(h), _ptr(m), float(L), float(gamma),
                                    _ptr(wv), _ptr(vv), int(p), int(comp), float(delta)))


def adjoint_counts(pos, h, L=1.0, nc=3, gamma=GAMMA_DEFAULT, threads=0):
    """(candidates, pairs) of the adjoint sweep: window and pair cut-off max(H_i, H_j)."""
    pos = _f64(pos, (-1, 3)); n = pos.shape[0]
    h = _f64(h)
    out = np.zeros(2, np.int64)
    rc = _load().or_adjoint_counts(n, _ptr(pos), _ptr(h), float(L), int(nc), float(gamma),
                                   _ptr(out), int(threads))
    if rc:
        raise ValueError(f"oracle adjoint_counts: {_ERR.get(rc, rc)}")
    return int(out[0]), int(out[1])
