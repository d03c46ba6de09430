"""Batched execution: many independent boxes in one grid (one plan and one
persistent launch per pass), and the whole step captured in a CUDA graph."""
import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06231_gb300 import build
    build.build_library()


def _run(boxes, g_seed=7, launch_shape=None):
    """sort + density + backward of `boxes` in ONE grid; returns numpy outputs."""
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    h = torch.from_numpy(np.concatenate([b.h for b in boxes])).to(dev)
    m = torch.from_numpy(np.concatenate([b.m for b in boxes])).to(dev)
    n = pos.shape[0]
    rng = np.random.default_rng(g_seed)
    gr = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    gd = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    with Grid([(b.n, b.L, b.nc) for b in boxes]) as g:
        if launch_shape:
            g.set_tuning(*launch_shape)
        g.sort(pos, h, m)
        rho, D, nn = g.density()
        gp, gh = g.backward(gr, gd)
        g.sync()
    return [t.cpu().numpy() for t in (rho, D, nn, gp, gh)], gr.cpu().numpy(), gd.cpu().numpy()


def test_batched_equals_per_box():
    boxes = I.multibox(n_boxes=6, scale=0.5, seed=11)
    (rho, D, n, gp, gh), gr, gd = _run(boxes)
    first = 0
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    for b in boxes:
        sl = slice(first, first + b.n)
        with Grid((b.n, b.L, b.nc)) as g:
            g.sort(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.h).to(dev),
                   torch.from_numpy(b.m).to(dev))
            r1, d1, n1 = g.density()
            gp1, gh1 = g.backward(torch.from_numpy(gr[sl]).to(dev),
                                  torch.from_numpy(gd[sl]).to(dev))
            g.sync()
        # forward: fixed-point accumulation, identical bits
        assert np.array_equal(rho[sl], r1.cpu().numpy())
        assert np.array_equal(D[sl], d1.cpu().numpy())
        assert np.array_equal(n[sl], n1.cpu().numpy())
        # adjoint: fixed-point accumulation too, identical bits
        assert np.array_equal(gp[sl], gp1.cpu().numpy())
        assert np.array_equal(gh[sl], gh1.cpu().numpy())
        first += b.n


def test_batched_vs_oracle(oracle_lib):
    boxes = I.multibox(n_boxes=4, scale=0.5, seed=12)
    (rho, D, n, _, _), _, _ = _run(boxes)
    first = 0
    for b in boxes:
        ref = oracle_lib.density_cells(b.pos, b.h, b.m, b.L, b.nc)
        sl = slice(first, first + b.n)
        assert np.abs(rho[sl] / ref.rho - 1).max() < 1e-5
        assert np.all(np.abs(D[sl] - ref.drho_dh) <= 1e-4 * ref.S)
        ok = ref.band == 0
        assert np.array_equal(n[sl][ok], ref.n_ngb[ok])
        first += b.n


@pytest.mark.slow
def test_multibox_64_full_size_vs_oracle(oracle_lib):
    """The whole 64-box mix (9,314,318 particles, N per box log-uniform in
    [4096, 524288], uniform or clustered) in one grid at the benchmark's
    launch shape (4 / 3 CTAs per SM): the density of every particle of every
    box against the oracle's pseudo-Verlet sweep, and the adjoint of six
    boxes (the three largest of each kind) against the oracle's pseudo-Verlet
    adjoint."""
    boxes = I.multibox()
    (rho, D, n, gp, gh), gr, gd = _run(boxes, launch_shape=(4, 3))
    firsts = np.concatenate([[0], np.cumsum([b.n for b in boxes])])
    for b, f in zip(boxes, firsts):
        sl = slice(f, f + b.n)
        ref = oracle_lib.density_pv(b.pos, b.h, b.m, b.L, b.nc)
        assert np.abs(rho[sl] / ref.rho - 1).max() <= 1e-5, b.name
        assert np.all(np.abs(D[sl] - ref.drho_dh) <= 1e-4 * ref.S), b.name
        ok = ref.band == 0
        assert np.array_equal(n[sl][ok], ref.n_ngb[ok]), b.name
        assert np.all(np.abs(n[sl][~ok] - ref.n_ngb[~ok]) <= ref.band[~ok]), b.name
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)
    for kind in ("uniform", "clustered"):
        picks = sorted((i for i, b in enumerate(boxes) if kind in b.name),
                       key=lambda i: -boxes[i].n)[:3]
        for i in picks:
            b, sl = boxes[i], slice(firsts[i], firsts[i] + boxes[i].n)
            gp0, gh0 = oracle_lib.backward_pv(b.pos, b.h, b.m, gr[sl].astype(np.float64),
                                              gd[sl].astype(np.float64), b.L, b.nc)
            assert rel(gp[sl].astype(np.float64), gp0) <= 1e-4, b.name
            assert rel(gh[sl].astype(np.float64), gh0) <= 1e-4, b.name


def test_cuda_graph_replay_matches_eager():
    """sort + density + backward captured once in a CUDA graph and replayed."""
    import torch
    from paper_1804_06231_gb300.pv import Grid
    dev = torch.device("cuda", 0)
    box = I.uniform(50000, 21, nc=10)
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    gr = torch.randn(box.n, device=dev, dtype=torch.float32)
    gd = torch.randn(box.n, device=dev, dtype=torch.float32)
    rho = torch.empty(box.n, device=dev)
    D = torch.empty_like(rho)
    nn = torch.empty(box.n, device=dev, dtype=torch.int32)
    gp = torch.empty((box.n, 3), device=dev)
    gh = torch.empty_like(rho)
    grid = Grid((box.n, 1.0, box.nc))

    def step():
        grid.sort(pos, h, None, float(box.m[0]))
        grid.density(rho, D, nn)
        grid.backward(gr, gd, gp, gh)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()          # eager warm-up (sets kernel attributes outside the capture)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref = [t.clone() for t in (rho, D, nn)]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for t in (rho, D, gp, gh):
        t.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ref[0], rho) and torch.equal(ref[1], D) and torch.equal(ref[2], nn)
    assert torch.isfinite(gp).all() and gp.abs().sum() > 0
    grid.close()


def test_launch_shapes_meet_parity_and_autotune(oracle_lib, tmp_path):
    """Launch shapes of the sweeps (CTAs per SM of the cell kernels, which
    moves dense cells between the cell-centric and the task kernels, and
    particles per task of the task kernels) meet the parity bar against the
    oracle, out-of-range shapes are refused, and the autotuner picks a shape,
    sets it and caches it."""
    import torch
    from paper_1804_06231_gb300 import tune
    from paper_1804_06231_gb300.pv import Grid
    from gpu_util import check_density  # noqa: E402
    box = I.clustered(60000, 31)
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    m = torch.from_numpy(box.m).to(dev)
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    w, v = I.loss_weights(box.n, 5)
    g_up, k_up = oracle_lib.loss_upstream(ref.rho, w, v)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g_up, k_up, box.L, box.nc)
    gr = torch.from_numpy(np.asarray(g_up, np.float32)).to(dev)
    gd = torch.from_numpy(np.asarray(k_up, np.float32)).to(dev)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    with Grid((box.n, box.L, box.nc)) as g:
        g.sort(pos, h, m)
        assert g.tuning() == (*tune.DEFAULT, tune.DEFAULT_TASK, tune.DEFAULT_TASK)
        for d, b, td, tb in ((2, 1, 64, 256), (3, 2, 128, 64), (4, 3, 256, 128), (4, 1, 64, 64),
                             (2, 1, 256, 256)):
            g.set_tuning(d, b, td, tb)
            assert g.tuning() == (d, b, td, tb)
            rho, D, n = g.density()
            gp, gh = g.backward(gr, gd)
            g.sync()
            check_density(rho.cpu().numpy().astype(np.float64),
                          D.cpu().numpy().astype(np.float64), n.cpu().numpy(), ref)
            assert rel(gp.cpu().numpy().astype(np.float64), gp0) <= 1e-4
            assert rel(gh.cpu().numpy().astype(np.float64), gh0) <= 1e-4
        from paper_1804_06231_gb300.pv import PvError
        with pytest.raises(PvError):
            g.set_tuning(5, 2)
        with pytest.raises(PvError):
            g.set_tuning(3, 4)
        with pytest.raises(PvError):
            g.set_tuning(3, 3, 96, 128)
        with pytest.raises(PvError):
            g.set_tuning(3, 3, 128, 512)
        path = str(tmp_path / "tuning.json")
        r1 = tune.autotune(g, gr, gd, reps=2, cache_path=path)
        assert r1["source"] == "timed"
        assert g.tuning() == (r1["density_ctas_per_sm"], r1["backward_ctas_per_sm"],
                              r1["density_task_block"], r1["backward_task_block"])
        r2 = tune.autotune(g, gr, gd, reps=2, cache_path=path)
        assert r2["source"] == "cache" and r2["signature"] == r1["signature"]
