"""pv_update_positions: the sort of one step re-used for the positions of the
next (windows widened by twice the largest displacement since the sort),
against the FP64 oracle on the moved particles and against a fresh sort."""
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


def _moved(box, frac, seed, h_jitter=0.0):
    """Positions moved by up to `frac` of the free skin (edge - H_max) / 2,
    wrapped into the box, and h scaled by up to (1 +- h_jitter) while keeping
    H_max + 2 displacement below the edge."""
    rng = np.random.default_rng(seed)
    edge = box.L / box.nc
    H = 1.825742 * box.h.astype(np.float64)
    skin = (edge - H.max()) / 2
    v = rng.standard_normal((box.n, 3))
    v *= (frac * skin * rng.random(box.n) / np.linalg.norm(v, axis=1))[:, None]
    pos = np.mod(box.pos + v, box.L)
    h = box.h * (1.0 + h_jitter * rng.uniform(-1, 1, box.n)).astype(np.float32)
    return pos, h


def _tensors(*arrs):
    import torch
    dev = torch.device("cuda", 0)
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrs]


def test_update_with_unmoved_particles_is_bit_identical():
    from paper_1804_06231_gb300.pv import Grid
    box = I.uniform(50000, 41, nc=9)
    pos, h, m = _tensors(box.pos, box.h, box.m)
    with Grid((box.n, box.L, box.nc)) as g:
        g.sort(pos, h, m)
        a = [t.cpu().numpy() for t in g.density()]
        g.update(pos, h)
        b = [t.cpu().numpy() for t in g.density()]
        g.sync()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_update_matches_oracle_on_moved_particles(oracle_lib, kind):
    import torch
    from paper_1804_06231_gb300.pv import Grid
    box = I.uniform(60000, 42, nc=None) if kind == "uniform" else I.clustered(60000, 43, nc=None)
    # room for motion: cells of the finest grid for h shrunk by 15 %
    box.h = (box.h * 0.85).astype(np.float32)
    pos, h, m = _tensors(box.pos, box.h, box.m)
    new_pos, new_h = _moved(box, 0.8, 7, h_jitter=0.01)
    H = 1.825742 * new_h.astype(np.float64)
    d = new_pos - box.pos
    d -= np.round(d / box.L) * box.L
    assert H.max() + 2 * np.linalg.norm(d, axis=1).max() < box.L / box.nc
    npos, nh = _tensors(new_pos, new_h)
    rng = np.random.default_rng(3)
    gr, gd = _tensors(rng.standard_normal(box.n).astype(np.float32),
                      rng.standard_normal(box.n).astype(np.float32))
    with Grid((box.n, box.L, box.nc)) as g:
        g.sort(pos, h, m)
        g.density()
        g.update(npos, nh)
        rho, D, n = g.density()
        gp, gh = g.backward(gr, gd)
        st = g.stats(raise_on_flags=False)
        assert st.device_flags == 0
        rho, D, n = (t.cpu().numpy() for t in (rho, D, n))
        gp, gh = gp.cpu().numpy(), gh.cpu().numpy()
    ref = oracle_lib.density_cells(new_pos, new_h, box.m, box.L, box.nc)
    check_density(rho.astype(np.float64), D.astype(np.float64), n, ref)
    gp0, gh0 = oracle_lib.backward_cells(new_pos, new_h, box.m, gr.cpu().numpy(),
                                         gd.cpu().numpy(), box.L, box.nc)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(gp.astype(np.float64), gp0) <= 1e-4
    assert rel(gh.astype(np.float64), gh0) <= 1e-4
    # and the same neighbour counts as a fresh sort of the moved particles
    with Grid((box.n, box.L, box.nc)) as g2:
        g2.sort(npos, nh, _tensors(box.m)[0])
        n2 = g2.density()[2].cpu().numpy()
    ok = ref.band == 0
    assert np.array_equal(n[ok], n2[ok])


def test_update_beyond_the_skin_is_flagged_then_resort_recovers():
    from paper_1804_06231_gb300 import pv
    from paper_1804_06231_gb300.pv import Grid
    box = I.uniform(30000, 44, nc=None)
    pos, h, m = _tensors(box.pos, box.h, box.m)
    new_pos, _ = _moved(box, 4.0, 8)  # moves far beyond the skin
    npos, = _tensors(new_pos)
    with Grid((box.n, box.L, box.nc)) as g:
        g.sort(pos, h, m)
        g.update(npos, h)
        rho, _, _ = g.density()
        st = g.stats(raise_on_flags=False)
        assert st.device_flags & pv.FLAG_SKIN_EXCEEDED
        with pytest.raises(pv.PvError):
            g.sync()
        g.sort(npos, h, m)
        rho, D, n = g.density()
        g.sync()
        assert g.stats().device_flags == 0


def test_update_on_a_batched_grid_tracks_each_box(oracle_lib):
    """Several boxes in one grid, moved by different amounts: each box's
    windows widen by its own displacement, and every box still matches the
    oracle on its moved particles."""
    import torch
    from paper_1804_06231_gb300.pv import Grid
    boxes = [I.uniform(20000, 50 + k, nc=None) for k in range(3)]
    for b in boxes:
        b.h = (b.h * 0.85).astype(np.float32)
    moved = [_moved(b, f, 60 + k) for k, (b, f) in enumerate(zip(boxes, (0.0, 0.3, 0.8)))]
    cat = lambda arrs: np.ascontiguousarray(np.concatenate(arrs))
    pos, h, m = _tensors(cat([b.pos for b in boxes]), cat([b.h for b in boxes]),
                         cat([b.m for b in boxes]))
    npos, = _tensors(cat([p for p, _ in moved]))
    with Grid([(b.n, b.L, b.nc) for b in boxes]) as g:
        g.sort(pos, h, m)
        g.update(npos, h)
        rho, D, n = (t.cpu().numpy() for t in g.density())
        assert g.stats().device_flags == 0
    first = 0
    for b, (p, _) in zip(boxes, moved):
        sl = slice(first, first + b.n)
        ref = oracle_lib.density_cells(p, b.h, b.m, b.L, b.nc)
        check_density(rho[sl].astype(np.float64), D[sl].astype(np.float64), n[sl], ref)
        first += b.n


def test_update_of_empty_and_single_particle_grids():
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    with Grid([(0, 1.0, 3), (1, 1.0, 3)]) as g:
        pos = torch.tensor([[0.5, 0.5, 0.5]], dtype=torch.float64, device=dev)
        h = torch.tensor([0.1], dtype=torch.float32, device=dev)
        g.sort(pos, h, None, 1.0)
        g.update(pos + 0.01, h)
        rho, D, n = g.density()
        g.sync()
        H = 1.825742 * 0.1
        assert rho.item() == pytest.approx(8.0 / np.pi / H ** 3, rel=1e-6)
        assert n.item() == 0
