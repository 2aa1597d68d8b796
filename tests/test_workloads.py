"""The seeded synthetic inputs have the structure the benchmark workloads are
specified with (sizes, walls, exits, obstacle fractions, agent counts and
placements), and the same seed always gives the same input.  Large layouts
are checked at a reduced side where the generator takes one."""
import numpy as np
import pytest
from scipy import ndimage

from paper_0911_2900_gb300 import workloads as wl

FREE, WALL, EXIT = wl.FREE, wl.WALL, wl.EXIT
EIGHT = np.ones((3, 3), bool)


def assert_valid(w, n=None):
    t = w.cell_type
    H, W = t.shape
    # border: walls and exits only; exits only on the border
    border = np.zeros_like(t, bool)
    border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
    assert np.all(t[border] != FREE)
    assert not np.any(t[~border] == EXIT)
    assert (t == EXIT).any()
    # agents: distinct free cells inside the grid
    c = w.cells.astype(np.int64)
    assert len(np.unique(c)) == len(c)
    assert np.all((c >= 0) & (c < H * W))
    assert np.all(t.ravel()[c] == FREE)
    if n is not None:
        assert len(c) == n
    # every free cell reaches an exit through non-wall cells (8-connected)
    lab, _ = ndimage.label(t != WALL, structure=EIGHT)
    good = np.unique(lab[t == EXIT])
    assert np.all(np.isin(lab[t == FREE], good[good > 0]))


def test_small_room():
    w = wl.config_small_room()
    assert w.cell_type.shape == (200, 200) and w.v_m == 4 and w.k_S == 1.2
    assert_valid(w, 2000)
    ex = np.argwhere(w.cell_type == EXIT)
    assert len(ex) == 4 and np.all(ex[:, 0] == 199)
    assert sorted(ex[:, 1]) == [98, 99, 100, 101]  # centred on the bottom wall
    assert int((w.cell_type == WALL).sum()) == 4 * 199 - 4  # nothing but the border


@pytest.mark.parametrize("v", [1, 5])
def test_corridors(v):
    w = wl.config_corridors(v_m=v)
    t = w.cell_type
    assert t.shape == (500, 1000) and w.v_m == v
    assert_valid(w, 40_000)
    assert int((t == EXIT).sum()) == 16  # four 4-cell exits
    inner = t[1:-1, 1:-1]
    # about 10% of the inner cells blocked beyond the fixed walls
    assert 0.10 <= (inner == WALL).mean() <= 0.20
    # ten doors of 4 cells from the room into the corridors
    col = t[1:-1, 500]
    assert int((col != WALL).sum()) == 40


def test_gmm_placement_is_clustered():
    w = wl.config_precision(side=400, n=10_000)
    t = w.cell_type
    assert t.shape == (400, 400)
    assert_valid(w, 10_000)
    assert int((t == EXIT).sum()) == 16 * 4
    # clustered: far more crowded 10x10 blocks than a uniform placement gives
    occ = np.zeros(t.size, bool)
    occ[w.cells] = True
    blocks = occ.reshape(40, 10, 40, 10).sum(axis=(1, 3))
    u = wl.place_uniform(t, 10_000, 9)
    occ_u = np.zeros(t.size, bool)
    occ_u[u] = True
    blocks_u = occ_u.reshape(40, 10, 40, 10).sum(axis=(1, 3))
    assert blocks.max() > 3 * blocks_u.max()


def test_stress_layout_small_side():
    w = wl.config_stress(side=512, n=20_000)
    assert w.v_m == 5
    assert_valid(w, 20_000)
    assert int((w.cell_type == EXIT).sum()) == 64 * 4


def test_batch_replicates():
    reps = wl.config_batch(n_rep=12, cells_hi=300 ** 2, agents_hi=5_000)
    assert len(reps) == 12
    for w in reps:
        H, W = w.cell_type.shape
        assert 1.0 <= W / H <= 2.3 and W >= 16 and H >= 16
        assert 1 <= w.v_m <= 5
        free = int((w.cell_type == FREE).sum())
        assert 1 <= len(w.cells) <= max(1, int(0.3 * free))
        assert_valid(w)
        # no obstacle within 3 cells of an exit
        apron = wl.exit_apron(w.cell_type, 3)
        border = np.zeros_like(apron)
        border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
        assert not np.any((w.cell_type == WALL) & apron & ~border)
    assert len({w.seed for w in reps}) == len(reps)


def test_same_seed_same_input():
    a, b = wl.config_corridors(seed=3), wl.config_corridors(seed=3)
    assert np.array_equal(a.cell_type, b.cell_type) and np.array_equal(a.cells, b.cells)
    c = wl.config_corridors(seed=4)
    assert not np.array_equal(a.cells, c.cells)
    x = wl.config_batch(n_rep=3, cells_hi=200 ** 2, agents_hi=2_000, seed=7)
    y = wl.config_batch(n_rep=3, cells_hi=200 ** 2, agents_hi=2_000, seed=7)
    for p, q in zip(x, y):
        assert np.array_equal(p.cell_type, q.cell_type) and np.array_equal(p.cells, q.cells)
