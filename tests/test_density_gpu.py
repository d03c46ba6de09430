"""GPU parity of pv_sort_cells + pv_density against the FP64 oracle.

Bar: rho within 1e-5 relative; drho/dh within 1e-4 of S_i = sum_j m_j |dW/dh|
(drho/dh is a sum of terms of both signs, so a plain relative test is
ill-conditioned); n_i bit-exact except where the oracle finds a pair within
1e-6 relative of the cut-off, where the difference is bounded by that count.
"""
import math

import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I

pytestmark = pytest.mark.gpu

from gpu_util import check_density, run_density  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06231_gb300 import build
    build.build_library()


@pytest.mark.parametrize("nc", [3, 5, 12])
def test_uniform_32k_vs_brute_force(oracle_lib, nc):
    box = I.cfg0()
    box.nc = nc
    rho, D, n, st, _ = run_density(box, uniform_mass=True)
    ref = oracle_lib.density_brute(box.pos, box.h, box.m)
    check_density(rho, D, n, ref)
    assert st.interactions == int(n.sum())
    assert st.device_flags == 0


def test_clustered_vs_oracle(oracle_lib):
    box = I.clustered(60000, 17)
    rho, D, n, st, _ = run_density(box)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    check_density(rho, D, n, ref)
    assert st.max_cell_count > 512   # exercises the large-cell sort path


def test_large_cells_vs_oracle(oracle_lib):
    """Coarse grid: ~1200 particles per cell (large-cell sort, many j tiles)."""
    box = I.uniform(32768, 41, nc=3)
    rho, D, n, st, _ = run_density(box)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, 3)
    check_density(rho, D, n, ref)


def test_every_sort_path_vs_oracle(oracle_lib):
    """One cell of each size class of pv_sort_cells on a 3^3 grid: 26,000
    particles (above what the largest sort instance stages in shared memory,
    so its global-memory path), 8,000 (the staged largest instance), 3,000,
    1,000, 200, 40 and 10 particles, empty cells, and 100 in each of the
    rest.  A wrong order along any axis would drop pairs from the windows."""
    rng = np.random.default_rng(23)
    counts = [26000, 8000, 3000, 1000, 200, 40, 10, 0, 0] + [100] * 18
    cells = np.stack(np.meshgrid(np.arange(3), np.arange(3), np.arange(3),
                                 indexing="ij"), -1).reshape(-1, 3)
    pos = np.concatenate([(cells[c] + rng.random((k, 3))) / 3.0
                          for c, k in enumerate(counts) if k])
    pos = np.ascontiguousarray(pos[rng.permutation(len(pos))])
    n = len(pos)
    h = np.full(n, 0.012, dtype=np.float32) * rng.uniform(0.9, 1.1, n).astype(np.float32)
    m = np.full(n, 1.0 / n, dtype=np.float32)
    box = I.Box(pos, h, m, 1.0, 3, "sort-classes")
    rho, D, n_ngb, st, _ = run_density(box)
    assert st.max_cell_count == 26000
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, 3)
    check_density(rho, D, n_ngb, ref)


def test_masses_vary(oracle_lib):
    box = I.uniform(20000, 9)
    rng = np.random.default_rng(1)
    box.m = (box.m * rng.uniform(0.2, 5.0, box.n)).astype(np.float32)
    rho, D, n, _, _ = run_density(box)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    check_density(rho, D, n, ref)


def test_lattice_exact_constant(oracle_lib):
    box = I.lattice(24, nc=8)
    rho, D, n, _, _ = run_density(box)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    check_density(rho, D, n, ref)
    assert np.all(n == 56)


def test_test27cells_shape(oracle_lib):
    box = I.test27cells()
    rho, D, n, _, _ = run_density(box)
    ref = oracle_lib.density_brute(box.pos, box.h, box.m)
    check_density(rho, D, n, ref)


def test_edge_cases(oracle_lib):
    """Particles on cell faces, at x = 1 - eps, duplicates, an isolated particle."""
    rng = np.random.default_rng(3)
    n = 3000
    pos = rng.random((n, 3))
    nc = 5                       # edge 0.2 >= H_max = 0.172
    pos[:200, 0] = np.floor(pos[:200, 0] * nc) / nc          # exactly on faces
    pos[200:300, 1] = 1.0 - 1e-13                             # just below the wrap
    pos[300:320] = pos[320:340]                               # duplicates
    pos[340] = [1.0, 0.5, -0.25]                              # needs wrapping
    h = (I.ETA * n ** (-1 / 3) * rng.uniform(0.9, 1.1, n)).astype(np.float32)
    m = np.full(n, 1.0 / n, np.float32)
    box = I.Box(pos, h, m, 1.0, nc)
    rho, D, nn, _, _ = run_density(box)
    ref = oracle_lib.density_brute(pos, h, m)
    check_density(rho, D, nn, ref)


def test_tiny_and_empty_boxes(oracle_lib):
    one = I.Box(np.array([[0.3, 0.4, 0.5]]), np.array([0.05], np.float32),
                np.array([2.0], np.float32), 1.0, 3)
    empty = I.Box(np.zeros((0, 3)), np.zeros(0, np.float32), np.zeros(0, np.float32), 1.0, 4)
    small = I.uniform(700, 5)
    rho, D, n, st, _ = run_density([one, empty, small])
    ref_one = oracle_lib.density_brute(one.pos, one.h, one.m)
    ref_small = oracle_lib.density_brute(small.pos, small.h, small.m)
    check_density(rho[:1], D[:1], n[:1], ref_one)
    check_density(rho[1:], D[1:], n[1:], ref_small)
    assert n[0] == 0


def test_symmetries(oracle_lib):
    box = I.uniform(40000, 77, nc=10)
    rho0, D0, n0, _, _ = run_density(box)
    rot = I.Box(np.ascontiguousarray(box.pos[:, [1, 2, 0]]), box.h, box.m, 1.0, box.nc)
    rho1, D1, n1, _, _ = run_density(rot)
    sh = I.Box(np.mod(box.pos + [0.123, 0.456, 0.789], 1.0), box.h, box.m, 1.0, box.nc)
    rho2, D2, n2, _, _ = run_density(sh)
    for r, nn in ((rho1, n1), (rho2, n2)):
        assert np.abs(r / rho0 - 1).max() < 2e-6
        assert (nn != n0).sum() <= 2


def test_support_above_edge_is_flagged(oracle_lib):
    """A support larger than the cell edge latches a device flag; outputs untouched."""
    from paper_1804_06231_gb300 import pv
    box = I.uniform(3000, 4, nc=6)          # H_max = 0.172 > 1/6
    rho, D, n, st, _ = run_density(box, expect_flags=True)
    assert st.device_flags & pv.FLAG_SUPPORT_EXCEEDS_CELL


def test_deterministic(oracle_lib):
    box = I.clustered(50000, 5)
    a = run_density(box)
    b = run_density(box)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


def test_candidates_match_oracle_windows(oracle_lib):
    """pv_count_candidates counts the sorted-window distance tests of the method."""
    box = I.uniform(30000, 8, nc=8)
    _, _, _, st, cand = run_density(box, count_candidates=True)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    assert cand == pytest.approx(int(ref.counters[:, 0].sum()), rel=1e-5)


def test_adjoint_counts_match_oracle(oracle_lib):
    """The adjoint window and pair counts (cut-off max(H_i, H_j)) of the
    diagnostic pass equal the oracle's, up to pairs at the FP32 boundary."""
    for box in (I.uniform(30000, 8, nc=8), I.clustered(20000, 9, nc=3)):
        _, _, _, st, _ = run_density(box, count_candidates=True)
        cand, pairs = oracle_lib.adjoint_counts(box.pos, box.h, 1.0, box.nc)
        assert st.candidates_adjoint == pytest.approx(cand, rel=1e-5)
        assert st.pairs_adjoint == pytest.approx(pairs, rel=1e-5)


@pytest.mark.slow
def test_uniform_1m_every_particle(oracle_lib):
    """N = 1,048,576 at 15^3 cells, at the launch shape the benchmark tunes to
    (4 / 3 CTAs per SM): all particles against the oracle's pseudo-Verlet
    sweep."""
    box = I.cfg1()
    rho, D, n, st, _ = run_density(box, uniform_mass=True, launch_shape=(4, 3))
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    check_density(rho, D, n, ref)
    assert st.interactions == int(ref.n_ngb.sum()) or \
        abs(st.interactions - int(ref.n_ngb.sum())) <= int(ref.band.sum())


def test_sweep_timing_hooks():
    """pv_grid_time_sweeps records one event pair per sweep call; the per-launch
    times are positive and below the time of the whole call sequence."""
    import time
    import torch
    from paper_1804_06231_gb300.pv import Grid
    box = I.uniform(100000, 31, nc=10)
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    gr = torch.ones(box.n, device=dev)
    with Grid((box.n, 1.0, box.nc)) as g:
        g.sort(pos, h, None, float(box.m[0]))
        g.time_sweeps(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(70):  # more calls than the event ring holds
            g.density()
            g.backward(gr, gr)
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - t0) * 1e3
        td, tb = g.sweep_times()
        assert 0 < td and 0 < tb and 70 * (td + tb) < wall_ms
        assert all(math.isnan(t) for t in g.sweep_times())  # totals were reset
        g.time_sweeps(False)
        g.density()
        assert all(math.isnan(t) for t in g.sweep_times())


def test_orientation_counts_match_oracle(oracle_lib):
    """Per orientation class (self, face, edge, corner): the window distance
    tests and the interactions of the diagnostic pass equal the oracle's
    per-class counters (Section 2's statistics), up to FP32 boundary cases."""
    box = I.uniform(30000, 8, nc=8)
    _, _, _, st, _ = run_density(box, count_candidates=True)
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    band = int(ref.band.sum())
    for c in range(4):
        assert st.orientation[c][0] == pytest.approx(int(ref.counters[c, 0]), rel=1e-5)
        assert abs(st.orientation[c][1] - int(ref.counters[c, 1])) <= band
    assert abs(sum(st.orientation[c][1] for c in range(4)) - st.interactions) <= band


def test_slot_mask_partial_sums_add_up():
    """Masking the neighbour slots by orientation class splits rho and n into
    partial sums that add up to the full pass."""
    import torch
    from paper_1804_06231_gb300.pv import Grid, SLOT_MASK_ALL, slot_mask_of_class
    box = I.uniform(60000, 12, nc=9)
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(box.pos).to(dev)
    h = torch.from_numpy(box.h).to(dev)
    with Grid((box.n, 1.0, box.nc)) as g:
        g.sort(pos, h, None, float(box.m[0]))
        full = [t.cpu().numpy().astype(np.float64) for t in g.density()]
        parts = []
        for c in range(4):
            g.set_slot_mask(slot_mask_of_class(c))
            parts.append([t.cpu().numpy().astype(np.float64) for t in g.density()])
        g.set_slot_mask(SLOT_MASK_ALL)
        again = [t.cpu().numpy() for t in g.density()]
        g.sync()
    rho = sum(p[0] for p in parts)
    assert np.abs(rho / full[0] - 1).max() < 1e-6
    n = sum(p[2] + 1 for p in parts) - 1  # every pass reports pairs - 1 (the self pair)
    assert np.array_equal(n, full[2])
    assert np.array_equal(again[0], full[0].astype(np.float32))


def test_raw_interactions_match_oracle_kernel(oracle_lib):
    """pv_raw_interactions (every i against every j, no cut-off test) sums the
    half-scaled kernel terms: sum m wh = (pi/16) H^3 sum m W and
    sum m th = -(pi/16) h H^3 sum m dW/dh, per the oracle's kernel functions."""
    import torch
    from paper_1804_06231_gb300.pv import raw_interactions
    rng = np.random.default_rng(9)
    H = 0.05
    def ball(n):
        v = rng.standard_normal((n, 3))
        v *= (0.45 * H * rng.random(n) ** (1 / 3) / np.linalg.norm(v, axis=1))[:, None]
        return np.concatenate([v, rng.uniform(0.5, 1.5, (n, 1))], axis=1).astype(np.float32)
    xi, xj = ball(64), ball(2560)
    dev = torch.device("cuda", 0)
    out = raw_interactions(torch.from_numpy(xi).to(dev), torch.from_numpy(xj).to(dev), H,
                           reps=2).cpu().numpy().astype(np.float64) / 2
    h = H / 1.825742
    c = np.pi / 16 * H ** 3
    for i in range(xi.shape[0]):
        r = np.linalg.norm(xj[:, :3].astype(np.float64) - xi[i, :3], axis=1)
        W = np.array([oracle_lib.W(x, H) for x in r])
        Wh = np.array([oracle_lib.W_h(x, h) for x in r])
        m = xj[:, 3].astype(np.float64)
        assert out[i, 0] == pytest.approx(c * (m * W).sum(), rel=2e-5)
        assert abs(out[i, 1] + c * h * (m * Wh).sum()) <= 1e-4 * c * h * (m * np.abs(Wh)).sum()


@pytest.mark.slow
def test_clustered_4m_every_particle(oracle_lib):
    """N = 4,194,304 clustered particles on the finest grid (41^3 cells, up to
    21,392 particles in a cell: both the cell-centric and the task kernels and
    the per-axis sort of dense cells): every particle against the oracle's
    pseudo-Verlet sweep."""
    box = I.cfg2()
    rho, D, n, st, _ = run_density(box, uniform_mass=True, launch_shape=(4, 3))
    ref = oracle_lib.density_pv(box.pos, box.h, box.m, 1.0, box.nc)
    check_density(rho, D, n, ref)
    assert abs(st.interactions - int(ref.n_ngb.sum())) <= int(ref.band.sum())


def _scaled_wrapped_box(seed):
    """A box of edge L = 3.7 (not 1) whose positions are given anywhere in
    [-L, 2L) (each coordinate shifted by -L, 0 or +L) with masses in
    [0.5, 1.5] of the mean."""
    base = I.uniform(20000, seed, nc=None)
    L = 3.7
    rng = np.random.default_rng(seed + 1)
    pos = base.pos * L + L * rng.integers(-1, 2, (base.n, 3))
    h = (base.h.astype(np.float64) * L).astype(np.float32)
    m = (base.m * rng.uniform(0.5, 1.5, base.n)).astype(np.float32)
    return I.Box(np.ascontiguousarray(pos), h, m, L, base.nc)


def test_box_of_other_size_with_unwrapped_positions(oracle_lib):
    box = _scaled_wrapped_box(91)
    rho, D, n, _, _ = run_density(box)
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    check_density(rho, D, n, ref)
