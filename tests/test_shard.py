"""Host-side sharding of independent boxes over ranks: the assignment, its
balance bound, and a two-rank gloo run on CPU in which each rank handles its
own boxes (oracle density as the per-box work) and only the totals are
reduced."""
import os
import socket

import numpy as np
import pytest

from paper_1804_06231_gb300 import inputs as I
from paper_1804_06231_gb300 import shard


def test_assignment_covers_every_box_once():
    rng = np.random.default_rng(3)
    costs = rng.lognormal(0, 1.5, 64)
    for ws in (1, 2, 3, 8, 64, 100):
        plan = shard.assign_boxes(costs, ws)
        assert len(plan) == ws
        flat = sorted(b for p in plan for b in p)
        assert flat == list(range(64))
        assert plan == shard.assign_boxes(list(costs), ws)  # deterministic
        for r in range(ws):
            assert shard.local_boxes(costs, r, ws) == plan[r]


def test_assignment_balance_bound():
    """Largest load <= 4/3 of the optimum; the optimum is at least the mean
    load and at least the largest single cost."""
    rng = np.random.default_rng(4)
    for trial in range(20):
        costs = rng.lognormal(0, 1.0, int(rng.integers(5, 80)))
        for ws in (2, 4, 8):
            loads = shard.rank_loads(costs, shard.assign_boxes(costs, ws))
            lower = max(costs.sum() / ws, costs.max())
            assert max(loads) <= 4.0 / 3.0 * lower + 1e-9


def test_assignment_small_cases():
    assert shard.assign_boxes([], 2) == [[], []]
    assert shard.assign_boxes([5.0], 3) == [[0], [], []]
    # LPT on {3,3,2,2,2} over 2 ranks: 7 / 5 (optimum 6 / 6; 7 <= 4/3 * 6)
    plan = shard.assign_boxes([3, 3, 2, 2, 2], 2)
    assert sorted(shard.rank_loads([3, 3, 2, 2, 2], plan)) == [5.0, 7.0]
    with pytest.raises(ValueError):
        shard.assign_boxes([1.0], 0)
    with pytest.raises(ValueError):
        shard.assign_boxes([-1.0], 1)
    with pytest.raises(ValueError):
        shard.local_boxes([1.0], 2, 2)


def test_box_cost_model():
    assert shard.box_cost(1000, 10) == 1000.0
    # edge 0.1, H_max 0.05: windows cover (edge/H)^3 = 8x the pairs in range
    assert shard.box_cost(1000, 10, 1.0, 0.05) == pytest.approx(8000.0)
    assert shard.box_cost(1000, 10, 1.0, 0.2) == 1000.0


def _boxes():
    """Six independent small boxes of different sizes (finest cell grids)."""
    return [I.uniform(n, 40 + k) for k, n in enumerate((600, 900, 1500, 2500, 4000, 6000))]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        boxes = _boxes()
        costs = [shard.box_cost(b.n, b.nc, b.L, 1.825742 * float(b.h.max())) for b in boxes]
        mine = shard.local_boxes(costs, rank, ws)
        inter = 0
        for b in mine:
            d = oracle.density_cells(boxes[b].pos, boxes[b].h, boxes[b].m, boxes[b].L,
                                     boxes[b].nc, threads=1)
            inter += int(d.n_ngb.sum())
        ms = 10.0 + rank  # a per-rank step time
        tot, tmax = shard.step_totals(inter, ms)
        seen = [None] * ws
        dist.all_gather_object(seen, mine)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{tot} {tmax} {inter} {' '.join(map(str, sorted(sum(seen, []))))}\n")
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharded_step(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    import oracle
    boxes = _boxes()
    total = sum(int(oracle.density_cells(b.pos, b.h, b.m, b.L, b.nc).n_ngb.sum()) for b in boxes)
    lines = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(ws)]
    for tok in lines:
        assert float(tok[0]) == total          # sum over ranks = single-process total
        assert float(tok[1]) == 10.0 + ws - 1  # max of the step times
        assert list(map(int, tok[3:])) == list(range(len(boxes)))  # every box once
    assert int(lines[0][2]) + int(lines[1][2]) == total
    assert int(lines[0][2]) > 0 and int(lines[1][2]) > 0


def test_step_totals_without_process_group():
    assert shard.step_totals(5, 2.5) == (5.0, 2.5)
