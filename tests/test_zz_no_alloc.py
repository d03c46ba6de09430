"""pv_density_static: the entry point for callers that may not allocate device
memory (an application memory pool that owns the GPU, a plugin inside such a
host, a loop that cannot take cudaMalloc's synchronisation).  It keeps its
intermediates in a fixed device array inside libpv.so instead of a pv_grid.

Checked through the C ABI against the FP64 oracle and against the allocating
path (pv_sort_cells + pv_density on a one-box grid) at the tolerances of the
other GPU tests, on two calls in a row with different inputs (the shared array
keeps the previous call's contents, so the second call also checks that what
must start at zero is cleared); with per-particle masses and with a uniform
mass; and with an invalid input whose latched flag must not leak into the next
call (the flag word lives in the shared array too).  This file sorts last so
that a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I
from gpu_util import check_density

pytestmark = pytest.mark.gpu

RHO_RTOL = 1e-5
D_STOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06231_gb300 import build, pv
    build.build_library()
    return pv


def _static(pv, box, dev, uniform_mass=False, pos=None):
    """pv_density_static on `box` (positions `pos` if given); returns the
    outputs widened to float64 on the device and the latched flags."""
    import torch
    pos = torch.from_numpy(box.pos if pos is None else pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    m = None if uniform_mass else torch.from_numpy(box.m).to(dev)
    rho = torch.full((box.n,), -1.0, dtype=torch.float32, device=dev)
    D = torch.full((box.n,), -1.0, dtype=torch.float32, device=dev)
    n = torch.full((box.n,), -1, dtype=torch.int32, device=dev)
    flags = torch.full((1,), 12345, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    pv.pv_density_static(pos.data_ptr(), h.data_ptr(), None if m is None else m.data_ptr(),
                         float(box.m[0]) if uniform_mass else 0.0, box.n, box.L, box.nc,
                         0.0, rho.data_ptr(), D.data_ptr(), n.data_ptr(), flags.data_ptr(),
                         stream)
    torch.cuda.synchronize()
    return (rho.double().cpu().numpy(), D.double().cpu().numpy(), n.cpu().numpy(),
            int(flags.cpu()[0]))


def _grid(pv, box, dev, uniform_mass=False):
    import torch
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    m = torch.from_numpy(box.m).to(dev)
    with pv.Grid((box.n, box.L, box.nc)) as g:
        if uniform_mass:
            g.sort(pos, h, None, m_uniform=float(box.m[0]))
        else:
            g.sort(pos, h, m)
        rho, D, n = g.density()
        g.sync()
    return (rho.double().cpu().numpy(), D.double().cpu().numpy(), n.cpu().numpy())


def _check_both(lib, oracle_lib, box, dev, uniform_mass=False):
    rho, D, n, flags = _static(lib, box, dev, uniform_mass=uniform_mass)
    assert flags == 0
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    check_density(rho, D, n, ref)            # the oracle decides
    rho0, D0, n0 = _grid(lib, box, dev, uniform_mass=uniform_mass)
    assert np.abs(rho / rho0 - 1).max() <= RHO_RTOL
    assert np.all(np.abs(D - D0) <= D_STOL * ref.S)
    assert np.array_equal(n, n0)


def test_static_matches_oracle_and_allocating_path_twice(lib, oracle_lib):
    dev = __import__("torch").device("cuda", 0)
    first = I.uniform(20000, 61, nc=8)
    second = I.clustered(9000, 62)          # other size and grid: stale contents must not leak
    for box in (first, second):
        _check_both(lib, oracle_lib, box, dev)


def test_static_uniform_mass(lib, oracle_lib):
    """m = NULL with m_uniform = 1/N (the masses of the uniform workloads)."""
    dev = __import__("torch").device("cuda", 0)
    _check_both(lib, oracle_lib, I.uniform(16384, 63, nc=6), dev, uniform_mass=True)


def test_static_flag_does_not_leak(lib, oracle_lib):
    """A non-finite position latches PV_FLAG_BAD_POSITION in flags_out (the
    outputs stay unwritten); the next, valid call starts from a clear flag
    word and gives the oracle's result."""
    dev = __import__("torch").device("cuda", 0)
    box = I.uniform(5000, 64, nc=5)
    bad = box.pos.copy()
    bad[17, 1] = np.nan
    rho, D, n, flags = _static(lib, box, dev, pos=bad)
    assert flags & lib.FLAG_BAD_POSITION
    assert np.all(rho == -1.0) and np.all(n == -1)
    _check_both(lib, oracle_lib, box, dev)


def test_static_rejects_oversize(lib):
    import torch
    dev = torch.device("cuda", 0)
    big = lib.STATIC_MAX_PARTICLES + 1
    x = torch.zeros((big, 3), dtype=torch.float64, device=dev)
    hh = torch.full((big,), 0.01, dtype=torch.float32, device=dev)
    out = torch.empty(big, dtype=torch.float32, device=dev)
    with pytest.raises(lib.PvError) as e:
        lib.pv_density_static(x.data_ptr(), hh.data_ptr(), None, 1.0, big, 1.0, 10, 0.0,
                              out.data_ptr(), None, None, None, 0)
    assert e.value.status == 7    # PV_ERR_TOO_LARGE
    with pytest.raises(lib.PvError) as e:   # 17^3 cells > PV_STATIC_MAX_CELLS
        lib.pv_density_static(x.data_ptr(), hh.data_ptr(), None, 1.0, 100, 1.0, 17, 0.0,
                              out.data_ptr(), None, None, None, 0)
    assert e.value.status == 7
