"""Halo sharding on the GPU path: the ranks of a slab decomposition run one
after another on one GPU (their exchanges done by indexing, in the order the
point-to-point exchange builds), each on the full-size periodic grid of its
owned + halo particles.  The owned particles' density and adjoint equal the
single-grid results bit for bit (uniform masses: the same mass unit on every
rank) and match the FP64 oracle at the usual tolerances."""
import numpy as np
import pytest

from paper_1804_06231_gb300 import halo
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


def _run(pos, h, m_uniform, L, nc, g_rho, g_d, shape=(4, 3)):
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    with Grid((pos.shape[0], L, nc)) as g:
        g.set_tuning(*shape)
        g.sort(torch.from_numpy(pos).to(dev), torch.from_numpy(h).to(dev), None,
               m_uniform=m_uniform)
        rho, D, n = g.density()
        gp, gh = g.backward(torch.from_numpy(g_rho).to(dev), torch.from_numpy(g_d).to(dev))
        g.sync()
    return [t.cpu().numpy() for t in (rho, D, n, gp, gh)]


@pytest.mark.parametrize("ws", [2, 3, 4])
def test_sharded_equals_single_grid(oracle_lib, ws):
    box = I.uniform(120000, 41, nc=9)
    mu = float(box.m[0])
    rng = np.random.default_rng(42)
    g_rho = rng.standard_normal(box.n).astype(np.float32)
    g_d = rng.standard_normal(box.n).astype(np.float32)
    full = _run(box.pos, box.h, mu, box.L, box.nc, g_rho, g_d)
    s = halo.Slabs(box.nc, ws)
    seen = np.zeros(box.n, bool)
    for owned, hset in halo.local_sets(s, box.L, box.pos):
        loc = np.concatenate([owned, hset])
        part = _run(box.pos[loc], box.h[loc], mu, box.L, box.nc, g_rho[loc], g_d[loc])
        no = len(owned)
        for a, b in zip(part, full):
            assert np.array_equal(a[:no], b[owned])
        seen[owned] = True
    assert seen.all()
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    check_density(full[0].astype(np.float64), full[1].astype(np.float64), full[2], ref)
