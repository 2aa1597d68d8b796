"""The movement of Sec. 1 is sequential: agents walk one after the other in
priority order (reading R7).  The GPU emulates it in rounds: every agent that
can move has a footprint (its start cell and its path cells up to the first
wall or cell of an agent that stays this step, or up to the exit it would
leave by); in each round every waiting agent that has the best priority on
all its footprint cells walks, against the occupancy of that moment.  The
claim is that this gives exactly the sequential result, because an agent's
walk reads and writes only its footprint (and exits, which stay free).

This file checks the claim on the CPU: a plain Python model of the round
schedule, and one with the two filters the GPU kernel applies after the first
round (only cells not held yet are re-checked; later claims cover only those
and the held cells another agent lost), against the oracle's sequential loop
on random dense scenes with walls and exits, for v_m = 1..5.  It also checks
that the comparison would catch the plausible mistakes in such a schedule (a
footprint without the start cell, one cut short, the wrong priority order,
later claims without the held contested cells)."""
import numpy as np
import pytest

import oracle

FREE, WALL, EXIT = 0, 1, 2


def make_scene(rng, W, H, density, v):
    t = np.zeros((H, W), np.uint8)
    t[0, :] = t[-1, :] = WALL
    t[:, 0] = t[:, -1] = WALL
    inner = rng.random((H - 2, W - 2)) < 0.08
    t[1:-1, 1:-1][inner] = WALL
    border = [(0, x) for x in range(1, W - 1)] + [(H - 1, x) for x in range(1, W - 1)] + \
             [(y, 0) for y in range(1, H - 1)] + [(y, W - 1) for y in range(1, H - 1)]
    for k in rng.choice(len(border), 3, replace=False):
        t[border[k]] = EXIT
    free = np.flatnonzero(t.ravel() == FREE)
    n = max(1, int(density * len(free)))
    cells = rng.choice(free, n, replace=False).astype(np.int32)
    desired = cells.copy()
    for i, c in enumerate(cells):
        if rng.random() < 0.15:
            continue  # stays this step
        x0, y0 = int(c) % W, int(c) // W
        while True:
            dx, dy = (int(d) for d in rng.integers(-v, v + 1, 2))
            x, y = x0 + dx, y0 + dy
            if (dx or dy) and 0 <= x < W and 0 <= y < H:
                break
        desired[i] = y * W + x
    return t, cells, desired


def round_schedule(t, cells, desired, prio, foot_mode="exact", order="min"):
    """Final cells (-1: left by an exit) and the number of rounds."""
    H, W = t.shape
    flat = t.ravel()
    n = len(cells)
    cell = [int(c) for c in cells]
    stays = {cell[i] for i in range(n) if desired[i] == cell[i]}
    paths, foot = {}, {}
    for i in range(n):
        if desired[i] == cell[i]:
            continue
        x0, y0 = cell[i] % W, cell[i] // W
        dx, dy = int(desired[i]) % W - x0, int(desired[i]) // W - y0
        p = [(y0 + py) * W + (x0 + px) for px, py in oracle.path(dx, dy)]
        fp, leaves = [], False
        for c in p:
            if flat[c] == WALL or c in stays:
                break
            if flat[c] == EXIT:
                leaves = True
                break
            fp.append(c)
        if not fp and not leaves:
            continue  # blocked at once: stays where it is
        if foot_mode == "no_start":
            foot[i] = fp
        elif foot_mode == "first_only":
            foot[i] = [cell[i]] + fp[:1]
        else:
            foot[i] = [cell[i]] + fp
        paths[i] = p
    occ = set(cell)
    waiting = set(foot)
    better = (lambda a, b: a < b) if order == "min" else (lambda a, b: a > b)
    rounds = 0
    while waiting:
        rounds += 1
        owner = {}
        for i in waiting:
            for c in foot[i]:
                if c not in owner or better(prio[i], prio[owner[c]]):
                    owner[c] = i
        winners = [i for i in waiting if all(owner[c] == i for c in foot[i])]
        assert winners, "a round without progress"
        for i in winners:
            cur, gone = cell[i], False
            for c in paths[i]:
                if flat[c] == WALL or c in occ:
                    break
                cur = c
                if flat[c] == EXIT:
                    gone = True
                    break
            occ.discard(cell[i])
            if gone:
                cell[i] = -1
            else:
                occ.add(cur)
                cell[i] = cur
            waiting.discard(i)
    return np.array(cell, np.int32), rounds


def refined_schedule(t, cells, desired, prio, keep_contested=True):
    """The same schedule with the two filters the GPU kernel applies after the
    first round: an agent re-checks only the footprint cells it has not held
    yet (a cell once held stays held, since its other claimants can only
    wait), and from the second round on it claims only those cells plus the
    held ones that another agent lost in the first round (a cell that nobody
    else claimed is nobody else's concern).  keep_contested=False drops the
    held contested cells from the later claims (a planted mistake)."""
    H, W = t.shape
    flat = t.ravel()
    n = len(cells)
    cell = [int(c) for c in cells]
    stays = {cell[i] for i in range(n) if desired[i] == cell[i]}
    paths, foot = {}, {}
    for i in range(n):
        if desired[i] == cell[i]:
            continue
        x0, y0 = cell[i] % W, cell[i] // W
        dx, dy = int(desired[i]) % W - x0, int(desired[i]) // W - y0
        p = [(y0 + py) * W + (x0 + px) for px, py in oracle.path(dx, dy)]
        fp, leaves = [], False
        for c in p:
            if flat[c] == WALL or c in stays:
                break
            if flat[c] == EXIT:
                leaves = True
                break
            fp.append(c)
        if not fp and not leaves:
            continue
        foot[i] = [cell[i]] + fp
        paths[i] = p
    occ = set(cell)

    def walk(i):
        cur, gone = cell[i], False
        for c in paths[i]:
            if flat[c] == WALL or c in occ:
                break
            cur = c
            if flat[c] == EXIT:
                gone = True
                break
        occ.discard(cell[i])
        if gone:
            cell[i] = -1
        else:
            occ.add(cur)
            cell[i] = cur

    def owners(claims):
        own = {}
        for i, cs in claims.items():
            for c in cs:
                if c not in own or prio[i] < prio[own[c]]:
                    own[c] = i
        return own

    # first round: every mover claims its whole footprint
    own = owners(foot)
    need, contested = {}, set()
    for i in foot:
        lost = [c for c in foot[i] if own[c] != i]
        if lost:
            need[i] = set(lost)
            contested.update(lost)
        else:
            walk(i)
    clm = {i: need[i] | ({c for c in foot[i] if c in contested} if keep_contested else set())
           for i in need}
    rounds = 1
    while need:
        rounds += 1
        own = owners({i: clm[i] for i in need})
        done = []
        for i in need:
            still = {c for c in need[i] if own.get(c) != i}
            if not still:
                done.append(i)
            else:
                need[i] = still
        assert done, "a round without progress"
        for i in done:
            walk(i)
            del need[i]
    return np.array(cell, np.int32), rounds


def sequential(t, cells, desired, v, seed, step):
    sim = oracle.Sim(t, v=v, seed=seed)
    sim.place(cells)
    sim.move(desired, step)
    return sim.cell.copy()


def scenes(v, count=40):
    rng = np.random.default_rng(100 + v)
    for k in range(count):
        W, H = int(rng.integers(8, 20)), int(rng.integers(6, 16))
        density = (0.3, 0.6, 0.9)[k % 3]
        t, cells, desired = make_scene(rng, W, H, density, v)
        yield t, cells, desired, int(rng.integers(0, 2 ** 40)), int(rng.integers(0, 400))


@pytest.mark.parametrize("v", [1, 2, 3, 4, 5])
def test_rounds_equal_the_sequential_loop(v):
    most_rounds = 0
    for t, cells, desired, seed, step in scenes(v):
        prio = [oracle.move_priority(seed, i, step) for i in range(len(cells))]
        got, rounds = round_schedule(t, cells, desired, prio)
        want = sequential(t, cells, desired, v, seed, step)
        assert np.array_equal(got, want)
        most_rounds = max(most_rounds, rounds)
    assert most_rounds > 2  # the scenes do chain agents behind one another


@pytest.mark.parametrize("mistake", [dict(foot_mode="no_start"), dict(foot_mode="first_only"),
                                     dict(order="max")])
def test_comparison_catches_a_wrong_schedule(mistake):
    differ = 0
    for v in (2, 4, 5):
        for t, cells, desired, seed, step in scenes(v):
            prio = [oracle.move_priority(seed, i, step) for i in range(len(cells))]
            got, _ = round_schedule(t, cells, desired, prio, **mistake)
            differ += not np.array_equal(got, sequential(t, cells, desired, v, seed, step))
    assert differ > 0


@pytest.mark.parametrize("v", [1, 2, 3, 4, 5])
def test_held_and_contested_filters_keep_the_sequential_result(v):
    for t, cells, desired, seed, step in scenes(v):
        prio = [oracle.move_priority(seed, i, step) for i in range(len(cells))]
        got, _ = refined_schedule(t, cells, desired, prio)
        assert np.array_equal(got, sequential(t, cells, desired, v, seed, step))


def test_dropping_the_contested_cells_is_caught():
    differ = 0
    for v in (2, 3, 4, 5):
        for t, cells, desired, seed, step in scenes(v):
            prio = [oracle.move_priority(seed, i, step) for i in range(len(cells))]
            got, _ = refined_schedule(t, cells, desired, prio, keep_contested=False)
            differ += not np.array_equal(got, sequential(t, cells, desired, v, seed, step))
    assert differ > 0
