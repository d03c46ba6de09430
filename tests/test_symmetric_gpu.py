"""pv_density_symmetric (the paper's symmetric pair update, Section 3.3):
the same outputs as the gather path, against the FP64 oracle at the standard
tolerances on uniform, clustered, test27cells-shaped and multi-box inputs,
equal counts to pv_density, and bit-reproducible."""
import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I

pytestmark = pytest.mark.gpu

from gpu_util import check_density  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06231_gb300 import build
    build.build_library()


def _both(boxes):
    """(symmetric, gather) outputs of one grid holding `boxes`."""
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    h = torch.from_numpy(np.concatenate([b.h for b in boxes])).to(dev)
    m = torch.from_numpy(np.concatenate([b.m for b in boxes])).to(dev)
    outs = []
    with Grid([(b.n, b.L, b.nc) for b in boxes]) as g:
        g.sort(pos, h, m)
        for sym in (True, False, True):
            r, d, n = g.density(symmetric=sym)
            g.sync()
            outs.append((r.double().cpu().numpy(), d.double().cpu().numpy(), n.cpu().numpy()))
        st = g.stats()
    assert st.device_flags == 0
    s1, gth, s2 = outs
    for a, b in zip(s1, s2):   # bit-reproducible
        assert np.array_equal(a, b)
    return s1, gth


@pytest.mark.parametrize("kind", ["uniform", "clustered", "test27cells"])
def test_symmetric_vs_oracle(oracle_lib, kind):
    box = {"uniform": lambda: I.uniform(32768, 51, nc=12),
           "clustered": lambda: I.clustered(40000, 52),
           "test27cells": lambda: I.test27cells(53)}[kind]()
    (rho, D, n), (rho0, D0, n0) = _both([box])
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    check_density(rho, D, n, ref)
    assert np.array_equal(n, n0)
    assert np.abs(rho / rho0 - 1).max() <= 2e-6


def test_symmetric_multibox(oracle_lib):
    boxes = I.multibox(n_boxes=6, scale=0.3, seed=54)
    (rho, D, n), _ = _both(boxes)
    first = 0
    for b in boxes:
        sl = slice(first, first + b.n)
        ref = oracle_lib.density_cells(b.pos, b.h, b.m, b.L, b.nc)
        check_density(rho[sl], D[sl], n[sl], ref)
        first += b.n
