"""Halo sharding of one box over ranks, on the CPU: the slab plan, the local
particle sets, the FP64 oracle run per rank on its owned + halo particles
(results of the owned particles equal the single-box oracle bit for bit,
density and adjoint), and the same through real point-to-point exchanges on
two and three gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_1804_06231_gb300 import halo
from paper_1804_06231_gb300 import inputs as I


def test_slab_plan():
    for nc in (3, 4, 7, 15):
        for ws in range(1, nc + 1):
            s = halo.Slabs(nc, ws)
            assert s.bounds[0][0] == 0 and s.bounds[-1][1] == nc
            assert all(x1 > x0 for x0, x1 in s.bounds)
            assert all(s.bounds[k][1] == s.bounds[k + 1][0] for k in range(ws - 1))
            for r in range(ws):
                hl = s.halo_layers(r)
                x0, x1 = s.bounds[r]
                assert len(hl) == len(set(hl)) <= 2
                assert all(not (x0 <= y < x1) for y in hl)
                if ws > 1:  # both neighbouring layers are owned or in the halo
                    for y in ((x0 - 1) % nc, x1 % nc):
                        assert (x0 <= y < x1) or y in hl
                for d, lay in s.sends(r).items():
                    assert s.recvs(d)[r] == lay
                    assert all(s.owner(y) == r for y in lay)
    with pytest.raises(ValueError):
        halo.Slabs(3, 4)
    with pytest.raises(ValueError):
        halo.Slabs(2, 1)


def test_cell_layer_matches_wrapped_binning():
    L, nc = 3.7, 9
    x = np.array([-L, -1e-300, 0.0, L / nc, 2 * L / nc - 1e-12, L - 1e-15, L, 2.5 * L])
    lay = halo.cell_layer(x, L, nc)
    assert lay.min() >= 0 and lay.max() < nc
    assert lay[2] == 0 and lay[3] == 1 and lay[6] == 0


def test_local_sets_partition():
    box = I.uniform(6000, 31, nc=6)
    for ws in (1, 2, 3, 6):
        s = halo.Slabs(box.nc, ws)
        sets = halo.local_sets(s, box.L, box.pos)
        owned = np.concatenate([o for o, _ in sets])
        assert np.array_equal(np.sort(owned), np.arange(box.n))
        lay = halo.cell_layer(box.pos[:, 0], box.L, box.nc)
        for r, (o, hset) in enumerate(sets):
            assert np.all(np.diff(o) > 0)
            want = set(range(*s.bounds[r])) | set(s.halo_layers(r))
            assert set(np.unique(lay[np.concatenate([o, hset])])) <= want
            assert len(np.intersect1d(o, hset)) == 0


def _emulated(oracle_lib, box, ws, w, v):
    """Per-rank oracle runs on owned + halo particles; returns the owned
    particles' results scattered back to global order."""
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    g, k = oracle_lib.loss_upstream(ref.rho, w, v)
    s = halo.Slabs(box.nc, ws)
    rho = np.full(box.n, np.nan)
    n = np.full(box.n, -1, np.int64)
    gp = np.full((box.n, 3), np.nan)
    gh = np.full(box.n, np.nan)
    for owned, hset in halo.local_sets(s, box.L, box.pos):
        loc = np.concatenate([owned, hset])
        d = oracle_lib.density_cells(box.pos[loc], box.h[loc], box.m[loc], box.L, box.nc)
        no = len(owned)
        rho[owned], n[owned] = d.rho[:no], d.n_ngb[:no]
        # the halo's upstream gradients come from their owners
        p, q = oracle_lib.backward_cells(box.pos[loc], box.h[loc], box.m[loc], g[loc], k[loc],
                                         box.L, box.nc)
        gp[owned], gh[owned] = p[:no], q[:no]
    return ref, (g, k), rho, n, gp, gh


@pytest.mark.parametrize("ws", [1, 2, 3, 5])
def test_emulated_ranks_equal_single_box(oracle_lib, ws):
    box = I.uniform(8000, 32, nc=5)
    box.m = (box.m * (1.0 + 0.5 * np.random.default_rng(3).random(box.n))).astype(np.float32)
    w, v = I.loss_weights(box.n, 33)
    ref, (g, k), rho, n, gp, gh = _emulated(oracle_lib, box, ws, w, v)
    assert np.array_equal(rho, ref.rho)
    assert np.array_equal(n, ref.n_ngb)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, box.L, box.nc)
    assert np.array_equal(gp, gp0)
    assert np.array_equal(gh, gh0)


def test_emulated_ranks_clustered(oracle_lib):
    box = I.clustered(6000, 34)
    w, v = I.loss_weights(box.n, 35)
    ref, (g, k), rho, n, gp, gh = _emulated(oracle_lib, box, 3, w, v)
    assert np.array_equal(rho, ref.rho) and np.array_equal(n, ref.n_ngb)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, box.L, box.nc)
    assert np.array_equal(gp, gp0) and np.array_equal(gh, gh0)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        box = I.uniform(7000, 36, nc=6)
        w, v = I.loss_weights(box.n, 37)
        s = halo.Slabs(box.nc, ws)
        mine = np.nonzero(halo.owned_mask(box.pos, box.L, s, rank))[0]
        dom = halo.HaloDomain(s, rank, box.L, torch.from_numpy(box.pos[mine]),
                              torch.from_numpy(box.h[mine]), torch.from_numpy(box.m[mine]))
        pos, h, m = dom.pos.numpy(), dom.h.numpy(), dom.m.numpy()
        d = oracle.density_cells(pos, h, m, box.L, box.nc, threads=1)
        no = dom.n_owned
        g, k = oracle.loss_upstream(d.rho[:no], w[mine], v[mine])
        gl, kl = dom.halo_gradients(torch.from_numpy(g), torch.from_numpy(k))
        gp, gh = oracle.backward_cells(pos, h, m, gl.numpy(), kl.numpy(), box.L, box.nc,
                                       threads=1)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), idx=mine, pos=pos, rho=d.rho[:no],
                 n=d.n_ngb[:no], gp=gp[:no], gh=gh[:no])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_gloo_halo_exchange(tmp_path, oracle_lib, ws):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    box = I.uniform(7000, 36, nc=6)
    w, v = I.loss_weights(box.n, 37)
    ref = oracle_lib.density_cells(box.pos, box.h, box.m, box.L, box.nc)
    g, k = oracle_lib.loss_upstream(ref.rho, w, v)
    gp0, gh0 = oracle_lib.backward_cells(box.pos, box.h, box.m, g, k, box.L, box.nc)
    sets = halo.local_sets(halo.Slabs(box.nc, ws), box.L, box.pos)
    seen = np.zeros(box.n, bool)
    for r in range(ws):
        z = np.load(tmp_path / f"rank{r}.npz")
        idx = z["idx"]
        seen[idx] = True
        # the exchange built the local set in the documented order
        assert np.array_equal(z["pos"], box.pos[np.concatenate(sets[r])])
        assert np.array_equal(z["rho"], ref.rho[idx])
        assert np.array_equal(z["n"], ref.n_ngb[idx])
        assert np.array_equal(z["gp"], gp0[idx])
        assert np.array_equal(z["gh"], gh0[idx])
    assert seen.all()
