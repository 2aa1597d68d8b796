"""The library's host-side floor field (fast_floor_field, no GPU needed)
against the oracle's, and the checks on a caller's own field.

The library computes S exactly as step counts (a, b) with Dial's buckets; the
oracle with a heap Dijkstra of its own.  Both must give the same (a, b) and
the same doubles S = fl(a + fl(b*sqrt2)) on every cell.  A caller's field
must decompose into such step counts exactly; any other value is refused and
the first offending cell named."""
import math

import numpy as np
import pytest

from paper_0911_2900_gb300 import workloads as wl


@pytest.fixture(scope="module")
def fg():
    import paper_0911_2900_gb300 as fg

    fg.load()
    return fg


def grids():
    yield "room", wl.config_small_room(W=60, H=45, n=10, seed=1).cell_type
    yield "corridors", wl.config_corridors(v_m=2).cell_type
    for seed in range(4):
        rng = np.random.default_rng(seed)
        W, H = int(rng.integers(8, 40)), int(rng.integers(8, 30))
        t = wl.room(W, H)
        t[1:-1, 1:-1][rng.random((H - 2, W - 2)) < 0.3] = wl.WALL
        t[0, int(rng.integers(1, W - 1))] = wl.EXIT
        t[H - 1, int(rng.integers(1, W - 1))] = wl.EXIT
        yield f"walled{seed}", t


@pytest.mark.parametrize("name,t", list(grids()))
def test_library_field_equals_the_oracle(fg, orc, name, t):
    S, a, b = fg.floor_field(t)
    oa, ob, oS = orc.floor_field(t)
    assert np.array_equal(a, oa) and np.array_equal(b, ob)
    assert np.array_equal(S, oS)          # +inf at the same cells too


@pytest.mark.parametrize("name,t", list(grids()))
def test_caller_field_round_trip(fg, orc, name, t):
    """The oracle's field, given as the caller's, decomposes into the
    oracle's own step counts."""
    oa, ob, oS = orc.floor_field(t)
    S, a, b = fg.floor_field(t, static_field=oS)
    assert np.array_equal(a, oa) and np.array_equal(b, ob) and np.array_equal(S, oS)


def test_caller_field_with_a_virtual_wall(fg, orc):
    """A field computed around a wall that is not in the grid (a route the
    caller wants agents to prefer) is of the right form everywhere and
    decomposes into the step counts it was made of."""
    t = wl.room(50, 40)
    wl.add_exit(t, "bottom", 22, 4)
    tv = t.copy()
    tv[20, 5:45] = wl.WALL
    va, vb, vS = orc.floor_field(tv)
    vS = np.where(t == wl.WALL, np.inf, vS)   # the virtual wall cells are free in t
    hole = (t != wl.WALL) & np.isinf(vS)
    vS[hole] = 1000.0 + 7 * math.sqrt(2.0)     # a far-away value on the wall itself
    S, a, b = fg.floor_field(t, static_field=vS)
    ok = ~hole & (t != wl.WALL)
    assert np.array_equal(a[ok], va[ok]) and np.array_equal(b[ok], vb[ok])
    assert (a[hole] == 1000).all() and (b[hole] == 7).all()
    assert np.array_equal(S[ok], vS[ok])


def test_caller_field_refusals(fg, orc):
    t = wl.room(20, 15)
    wl.add_exit(t, "left", 6, 3)
    _, _, S = orc.floor_field(t)
    free = np.argwhere(t == wl.FREE)
    y, x = (int(v) for v in free[len(free) // 2])
    ex = tuple(int(v) for v in np.argwhere(t == wl.EXIT)[0])
    cases = []
    bad = S.copy()
    bad[y, x] = np.nextafter(bad[y, x], np.inf)          # one ulp off the form
    cases.append((bad, y * 20 + x))
    bad = S.copy()
    bad[y, x] = 2.5                                      # not a + b*sqrt2
    cases.append((bad, y * 20 + x))
    bad = S.copy()
    bad[ex] = 1.0                                        # an exit must be 0
    cases.append((bad, ex[0] * 20 + ex[1]))
    bad = S.copy()
    bad[y, x] = 0.0                                      # only exits are 0
    cases.append((bad, y * 20 + x))
    for v in (-1.0, np.nan, -np.inf):
        bad = S.copy()
        bad[y, x] = v
        cases.append((bad, y * 20 + x))
    for bad, cell in cases:
        with pytest.raises(fg.FastError, match=f"cell {cell}$"):
            fg.floor_field(t, static_field=bad)
    # +inf marks a free cell treated as a wall
    ok = S.copy()
    ok[y, x] = np.inf
    S2, a2, b2 = fg.floor_field(t, static_field=ok)
    assert a2[y, x] == -1 and b2[y, x] == -1 and math.isinf(S2[y, x])
    # the largest step counts the records hold, and one beyond
    big = S.copy()
    big[y, x] = 32766.0 + 32766.0 * math.sqrt(2.0)
    S3, a3, b3 = fg.floor_field(t, static_field=big)
    assert (a3[y, x], b3[y, x]) == (32766, 32766)
    big[y, x] = 32767.0 + 5.0 * math.sqrt(2.0)
    with pytest.raises(fg.FastError):
        fg.floor_field(t, static_field=big)
