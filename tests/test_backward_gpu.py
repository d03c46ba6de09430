"""GPU adjoint (pv_density_backward) against the FP64 oracle adjoint and FP64
central finite differences of L = sum_i w_i (rho_i - 1)^2 + sum_i v_i drho/dh_i."""
import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ADJ_RTOL = 1e-4   # relative L2 error of dL/dx and of dL/dh
ADJ_PTOL = 1e-4   # per particle: error below this fraction of the largest component


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06231_gb300 import build
    build.build_library()


def gpu_adjoint(box, g_rho, g_d, uniform_mass=False, launch_shape=None):
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    m = torch.from_numpy(box.m).to(dev)
    with Grid((box.n, box.L, box.nc)) as g:
        if launch_shape:
            g.set_tuning(*launch_shape)
        if uniform_mass:
            g.sort(pos, h, None, m_uniform=float(box.m[0]))
        else:
            g.sort(pos, h, m)
        gr = torch.from_numpy(np.asarray(g_rho, np.float32)).to(dev)
        gd = None if g_d is None else torch.from_numpy(np.asarray(g_d, np.float32)).to(dev)
        gp, gh = g.backward(gr, gd)
        g.sync()
    return gp.cpu().numpy().astype(np.float64), gh.cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_adjoint(gp, gh, gp0, gh0):
    """Relative L2 <= ADJ_RTOL for dL/dx and dL/dh, and every particle within
    ADJ_PTOL of the largest component, so that an error on a few particles
    cannot hide inside the norm."""
    assert rel_l2(gp, gp0) <= ADJ_RTOL, f"dL/dx rel L2 {rel_l2(gp, gp0):.3e}"
    assert rel_l2(gh, gh0) <= ADJ_RTOL, f"dL/dh rel L2 {rel_l2(gh, gh0):.3e}"
    ep = np.abs(gp - gp0).max() / np.abs(gp0).max()
    eh = np.abs(gh - gh0).max() / np.abs(gh0).max()
    assert ep <= ADJ_PTOL, f"dL/dx worst particle {ep:.3e} of the largest component"
    assert eh <= ADJ_PTOL, f"dL/dh worst particle {eh:.3e} of the largest component"


def _upstream(oracle_lib, box, seed):
    w, v = I.loss_weights(box.n, seed)
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, 1.0, box.nc)
    g, k = oracle_lib.loss_upstream(ref.rho, w, v)
    return w, v, g, k


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_adjoint_vs_oracle(oracle_lib, kind):
    box = I.uniform(40000, 3) if kind == "uniform" else I.clustered(40000, 4)
    w, v, g, k = _upstream(oracle_lib, box, 3)
    gp, gh = gpu_adjoint(box, g, k)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, 1.0, box.nc)
    check_adjoint(gp, gh, gp0, gh0)


def test_adjoint_rho_only_and_large_cells(oracle_lib):
    box = I.uniform(30000, 11, nc=3)     # ~1100 per cell: big-cell sort, tiled windows
    w, v, g, k = _upstream(oracle_lib, box, 11)
    gp, gh = gpu_adjoint(box, g, None)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, np.zeros(box.n), 1.0, 3)
    check_adjoint(gp, gh, gp0, gh0)


def test_adjoint_differentiation_workload(oracle_lib):
    """N = 262,144 uniform, finest grid: vs the oracle adjoint (rel L2 <= 1e-4)
    and vs FP64 central differences (step 1e-6) on 64 random particles."""
    box = I.cfg3()
    w, v, g, k = _upstream(oracle_lib, box, I.SEEDS["cfg3"])
    gp, gh = gpu_adjoint(box, g, k, uniform_mass=True)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, 1.0, box.nc)
    check_adjoint(gp, gh, gp0, gh0)
    rng = np.random.default_rng(64)
    idx = rng.choice(box.n, 64, replace=False)
    fd = np.array([[oracle_lib.fd_loss_grad(box.pos, box.h, box.m, w, v, p, c, 1e-6)
                    for c in range(4)] for p in idx])
    got = np.concatenate([gp[idx], gh[idx, None]], axis=1)
    assert rel_l2(got[:, :3], fd[:, :3]) <= ADJ_RTOL
    assert rel_l2(got[:, 3], fd[:, 3]) <= ADJ_RTOL


def test_autograd_function(oracle_lib):
    import torch
    from paper_1804_06231_gb300.autograd import PVDensity
    from paper_1804_06231_gb300.pv import Grid
    box = I.uniform(20000, 19)
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(box.pos).to(dev).requires_grad_(True)
    h = torch.from_numpy(box.h).to(dev).requires_grad_(True)
    m = torch.from_numpy(box.m).to(dev)
    w, v = I.loss_weights(box.n, 19)
    wt = torch.from_numpy(w).to(dev)
    vt = torch.from_numpy(v).to(dev)
    grid = Grid((box.n, 1.0, box.nc))
    rho, D, n = PVDensity.apply(pos, h, m, grid)
    L = (wt * (rho.double() - 1) ** 2).sum() + (vt * D.double()).sum()
    L.backward()
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, 1.0, box.nc)
    g, k = oracle_lib.loss_upstream(rho.detach().cpu().numpy().astype(np.float64), w, v)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, 1.0, box.nc)
    assert rel_l2(pos.grad.cpu().numpy(), gp0) <= ADJ_RTOL
    assert rel_l2(h.grad.cpu().numpy().astype(np.float64), gh0) <= ADJ_RTOL
    assert np.abs(rho.detach().cpu().numpy() / ref.rho - 1).max() < 1e-5
    grid.close()


@pytest.mark.slow
def test_adjoint_1m_every_particle(oracle_lib):
    """The benchmark workload (N = 1,048,576 uniform, 15^3 cells): the whole
    adjoint against the oracle's cell-list adjoint (relative L2 <= 1e-4 for
    dL/dx and dL/dh) and per particle within 1e-4 of the largest component."""
    box = I.cfg1()
    w, v = I.loss_weights(box.n, 3)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    g, k = oracle_lib.loss_upstream(ref.rho, w, v)
    gp, gh = gpu_adjoint(box, g, k, uniform_mass=True, launch_shape=(4, 3))
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, 1.0, box.nc)
    check_adjoint(gp, gh, gp0, gh0)


@pytest.mark.slow
def test_adjoint_clustered_4m_every_particle(oracle_lib):
    """N = 4,194,304 clustered particles on the finest grid (41^3 cells, up to
    21,392 in a cell), at the launch shape the benchmark tunes to for it (4 / 3
    CTAs per SM): dense cells run on the task kernel.  The whole adjoint
    against the oracle's pseudo-Verlet adjoint (relative L2 <= 1e-4 for dL/dx
    and dL/dh, and per particle within 1e-4 of the largest component)."""
    box = I.cfg2()
    w, v = I.loss_weights(box.n, 3)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    g, k = oracle_lib.loss_upstream(ref.rho, w, v)
    gp, gh = gpu_adjoint(box, g, k, uniform_mass=True, launch_shape=(4, 3))
    gp0, gh0 = oracle_lib.backward_pv(box.pos, box.h, box.m, g, k, 1.0, box.nc)
    check_adjoint(gp, gh, gp0, gh0)


def test_adjoint_box_of_other_size_with_unwrapped_positions(oracle_lib):
    """Edge L = 3.7, positions anywhere in [-L, 2L), varied masses: the adjoint
    against the oracle on the same (wrapped by both) positions."""
    from test_density_gpu import _scaled_wrapped_box
    box = _scaled_wrapped_box(93)
    w, v = I.loss_weights(box.n, 4)
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    g, k = oracle_lib.loss_upstream(ref.rho, w, v)
    gp, gh = gpu_adjoint(box, g, k)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, box.L, box.nc)
    check_adjoint(gp, gh, gp0, gh0)


def test_adjoint_deterministic():
    """The adjoint is bit-reproducible: fixed-point sums make it independent
    of which warp or CTA took which work item.  Twice on one grid and once on
    a fresh grid, for a clustered box (dense cells on the task path, tiny
    cells on the warp path) and for a batched grid of several boxes."""
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    cases = [[I.clustered(50000, 21)], I.multibox(n_boxes=5, scale=0.3, seed=22)]
    for boxes in cases:
        pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
        h = torch.from_numpy(np.concatenate([b.h for b in boxes])).to(dev)
        m = torch.from_numpy(np.concatenate([b.m for b in boxes])).to(dev)
        rng = np.random.default_rng(23)
        gr = torch.from_numpy(rng.standard_normal(pos.shape[0]).astype(np.float32)).to(dev)
        gd = torch.from_numpy(rng.standard_normal(pos.shape[0]).astype(np.float32)).to(dev)
        outs = []
        grid = None
        for fresh in (True, False, True):
            if fresh:
                if grid is not None:
                    grid.close()
                grid = Grid([(b.n, b.L, b.nc) for b in boxes])
                grid.sort(pos, h, m)
            gp, gh = grid.backward(gr, gd)
            grid.sync()
            outs.append((gp.cpu().numpy(), gh.cpu().numpy()))
        grid.close()
        for gp, gh in outs[1:]:
            assert np.array_equal(gp, outs[0][0])
            assert np.array_equal(gh, outs[0][1])


def test_adjoint_non_finite_gradient_is_flagged():
    """A NaN upstream gradient latches PV_FLAG_BAD_GRADIENT and leaves the
    outputs untouched."""
    import torch
    from paper_1804_06231_gb300 import pv
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    box = I.uniform(8000, 24, nc=6)
    gr = np.ones(box.n, np.float32)
    gr[123] = np.nan
    with Grid((box.n, box.L, box.nc)) as g:
        g.sort(torch.from_numpy(box.pos).to(dev), torch.from_numpy(box.h).to(dev),
               torch.from_numpy(box.m).to(dev))
        gp = torch.full((box.n, 3), 7.0, dtype=torch.float32, device=dev)
        gh = torch.full((box.n,), 7.0, dtype=torch.float32, device=dev)
        g.backward(torch.from_numpy(gr).to(dev), None, gp, gh)
        st = g.stats(raise_on_flags=False)
    assert st.device_flags & pv.FLAG_BAD_GRADIENT
    assert torch.all(gp == 7.0) and torch.all(gh == 7.0)
