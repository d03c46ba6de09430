"""Seeded generators: reproducible, right shapes and dtypes, valid cell grids."""
import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I


def test_uniform_reproducible_and_typed():
    a = I.uniform(1000, 5)
    b = I.uniform(1000, 5)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.h, b.h)
    assert a.pos.dtype == np.float64 and a.h.dtype == np.float32 and a.m.dtype == np.float32
    assert a.pos.min() >= 0 and a.pos.max() < 1
    base = I.ETA * 1000 ** (-1 / 3)
    assert a.h.min() >= 0.9 * base * (1 - 1e-6) and a.h.max() <= 1.1 * base * (1 + 1e-6)
    assert a.H_max <= 1.0 / a.nc


def test_named_configs_cell_rules():
    b0 = I.cfg0()
    assert b0.n == 32768 and b0.nc == 12 and b0.H_max <= 1 / 12
    b3 = I.cfg3(n=1 << 15)
    assert b3.H_max <= 1 / b3.nc and b3.H_max > 1 / (b3.nc + 1)


def test_clustered_density_rule():
    b = I.clustered(20000, 3)
    mix = b.extra["mixture"]
    rho = I.mixture_density(b.pos[:100], mix)
    h_expect = (I.ETA * (1.0 / b.n / rho) ** (1 / 3)).astype(np.float32)
    assert np.array_equal(h_expect, b.h[:100])
    assert b.H_max <= 1 / b.nc
    # the mixture has unit mass: a Monte Carlo average of rho over the cube is ~1
    rng = np.random.default_rng(0)
    assert I.mixture_density(rng.random((200000, 3)), mix).mean() == pytest.approx(1.0, rel=0.03)


def test_multibox_sizes():
    boxes = I.multibox(n_boxes=8, scale=0.5)
    assert len(boxes) == 8
    for b in boxes:
        assert b.n >= 64 and b.H_max <= 1 / b.nc + 1e-12


def test_lattice_and_test27cells():
    L = I.lattice(8, nc=4)
    assert L.n == 512 and np.all(L.h == L.h[0])
    t = I.test27cells(per_cell=216)
    assert t.n == 27 * 216
    cells = np.floor(t.pos * 3).astype(int)
    ids = (cells[:, 0] * 3 + cells[:, 1]) * 3 + cells[:, 2]
    assert np.all(np.bincount(ids, minlength=27) == 216)
