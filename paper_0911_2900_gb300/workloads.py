"""Seeded synthetic inputs: grids (walls, exits, obstacles) and agent placements.

This module holds none of the method's arithmetic (no floor field, no weights,
no sampling rule, no movement); it only builds the inputs that both the CUDA
library and the CPU oracle consume, so that they see identical grids and
starting cells.  All randomness comes from numpy's PCG64 generator seeded
explicitly.

The paper gives no geometry for its timings (it only fixes k_S, v_m, the number
of steps and the agent counts, Sec. 2-3); the layouts below are stand-ins with
the sizes, obstacle fractions, exit counts and agent densities of the five
workloads this library is measured on.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FREE, WALL, EXIT = 0, 1, 2


@dataclasses.dataclass
class Workload:
    name: str
    cell_type: np.ndarray          # uint8 [H, W]
    cells: np.ndarray              # int32 [n] starting cells (row-major index)
    v_m: int
    k_S: float = 1.2
    seed: int = 0
    steps: int = 396

    @property
    def shape(self):
        return self.cell_type.shape


# ----------------------------------------------------------------------------- grids
def room(W: int, H: int) -> np.ndarray:
    """W x H cells, walls on the border, free inside."""
    t = np.zeros((H, W), np.uint8)
    t[0, :] = WALL
    t[-1, :] = WALL
    t[:, 0] = WALL
    t[:, -1] = WALL
    return t


def add_exit(t: np.ndarray, side: str, pos: int, width: int = 4) -> None:
    """Turns `width` border wall cells into exit cells, starting at `pos`."""
    H, W = t.shape
    if side == "bottom":
        t[H - 1, pos:pos + width] = EXIT
    elif side == "top":
        t[0, pos:pos + width] = EXIT
    elif side == "left":
        t[pos:pos + width, 0] = EXIT
    elif side == "right":
        t[pos:pos + width, W - 1] = EXIT
    else:
        raise ValueError(side)


def spread_exits(t: np.ndarray, n_exits: int, width: int = 4) -> None:
    """n_exits exits spread evenly over the four sides (n_exits/4 per side)."""
    H, W = t.shape
    per = max(1, n_exits // 4)
    sides = ["bottom", "right", "top", "left"]
    made = 0
    for s in sides:
        L = W if s in ("bottom", "top") else H
        for j in range(per):
            if made == n_exits:
                return
            pos = int((2 * j + 1) * L / (2 * per)) - width // 2
            pos = min(max(pos, 1), L - 1 - width)
            add_exit(t, s, pos, width)
            made += 1


def add_obstacles(t: np.ndarray, fraction: float, rng: np.random.Generator,
                  side_lo: int = 2, side_hi: int = 20, protect=None) -> None:
    """Seeded axis-aligned rectangles (sides uniform in [side_lo, side_hi]) in
    the interior until `fraction` of all cells are walls; `protect` (bool mask)
    marks cells that must stay free (doors)."""
    H, W = t.shape
    target = int(fraction * H * W)
    walls = int((t == WALL).sum())
    interior_walls0 = walls
    want = interior_walls0 + target
    while walls < want:
        batch = max(16, (want - walls) // 100)
        ws = rng.integers(side_lo, side_hi + 1, size=batch)
        hs = rng.integers(side_lo, side_hi + 1, size=batch)
        xs = rng.integers(1, max(2, W - 1), size=batch)
        ys = rng.integers(1, max(2, H - 1), size=batch)
        for x, y, w, h in zip(xs, ys, ws, hs):
            x1, y1 = min(x + w, W - 1), min(y + h, H - 1)
            if x1 <= x or y1 <= y:
                continue
            sub = t[y:y1, x:x1]
            if protect is not None and protect[y:y1, x:x1].any():
                continue
            before = int((sub == WALL).sum())
            sub[sub == FREE] = WALL
            walls += int((sub == WALL).sum()) - before
            if walls >= want:
                break


def exit_apron(t: np.ndarray, depth: int = 3) -> np.ndarray:
    """Bool mask of the cells within `depth` (Chebyshev) of an exit cell, for
    add_obstacles' `protect`, so that no rectangle walls an exit in."""
    from scipy import ndimage

    return ndimage.binary_dilation(t == EXIT, structure=np.ones((3, 3), bool),
                                   iterations=depth)


def seal_unreachable(t: np.ndarray) -> int:
    """Turns every free cell that no 8-connected walk through non-wall cells
    links to an exit into a wall; returns how many cells were sealed."""
    from scipy import ndimage

    passable = t != WALL
    lab, _ = ndimage.label(passable, structure=np.ones((3, 3), bool))
    good = np.unique(lab[t == EXIT])
    good = good[good > 0]
    keep = np.isin(lab, good)
    sealed = passable & ~keep
    t[sealed] = WALL
    return int(sealed.sum())


# ----------------------------------------------------------------------------- placement
def _free_cells(t: np.ndarray) -> np.ndarray:
    return np.flatnonzero(t.ravel() == FREE).astype(np.int64)


def place_uniform(t: np.ndarray, n: int, seed: int) -> np.ndarray:
    """n distinct free (non-exit, non-wall) cells, uniformly at random."""
    rng = np.random.default_rng(seed)
    free = _free_cells(t)
    if n > len(free):
        raise ValueError(f"{n} agents but only {len(free)} free cells")
    if n * 4 > len(free):
        return np.sort(rng.choice(free, size=n, replace=False)).astype(np.int32)
    chosen = np.zeros(0, np.int64)
    while len(chosen) < n:
        extra = rng.choice(free, size=int((n - len(chosen)) * 1.1) + 16, replace=True)
        chosen = np.unique(np.concatenate([chosen, extra]))
    chosen = rng.permutation(chosen)[:n]
    return np.sort(chosen).astype(np.int32)


def place_gmm(t: np.ndarray, n: int, n_comp: int, seed: int,
              sigma_lo: float = 0.01, sigma_hi: float = 0.08) -> np.ndarray:
    """n distinct free cells drawn from a Gaussian mixture: n_comp equal-weight
    components, means uniform over the grid, sigma log-uniform in
    [sigma_lo, sigma_hi] x side; a draw that lands outside the grid, on a
    non-free cell or on a taken cell is rejected and redrawn."""
    rng = np.random.default_rng(seed)
    H, W = t.shape
    side = max(H, W)
    mx = rng.uniform(0, W, n_comp)
    my = rng.uniform(0, H, n_comp)
    sig = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_comp)) * side
    taken = np.zeros(H * W, bool)
    flat_t = t.ravel()
    out = []
    need = n
    rounds = 0
    while need > 0:
        rounds += 1
        m = int(need * 1.5) + 64
        comp = rng.integers(0, n_comp, m)
        x = np.floor(rng.normal(mx[comp], sig[comp])).astype(np.int64)
        y = np.floor(rng.normal(my[comp], sig[comp])).astype(np.int64)
        ok = (x >= 0) & (x < W) & (y >= 0) & (y < H)
        c = (y[ok] * W + x[ok])
        c = c[flat_t[c] == FREE]
        c = c[~taken[c]]
        # keep the first occurrence of each cell, in draw order
        _, first = np.unique(c, return_index=True)
        c = c[np.sort(first)][:need]
        taken[c] = True
        out.append(c)
        need -= len(c)
        if rounds > 10000:
            raise RuntimeError("gmm placement did not converge")
    return np.sort(np.concatenate(out)).astype(np.int32)


# ----------------------------------------------------------------------------- the five workloads
def config_small_room(W=200, H=200, n=2000, seed=0, v_m=4) -> Workload:
    """200x200 room, border walls, one 4-cell exit centred on the bottom wall,
    2,000 agents uniform in distinct free cells (FP64 workload)."""
    t = room(W, H)
    add_exit(t, "bottom", W // 2 - 2, 4)
    return Workload("room200_2k_v4", t, place_uniform(t, n, seed), v_m, seed=seed)


def config_corridors(v_m=4, seed=0, n=40000) -> Workload:
    """1000x500: a 500x500 room on the left, the right half split into ten
    corridors of width 48 by 1-cell walls, each with a 4-cell door to the
    room; 10% of the cells blocked by seeded rectangles (sides 2..20), free
    pockets cut off from every exit sealed; 4 exits (top and bottom of the
    room, two on the right wall); 40,000 agents uniform."""
    W, H = 1000, 500
    t = room(W, H)
    protect = np.zeros_like(t, bool)
    t[:, 500] = WALL
    rows = []
    for j in range(10):
        y0 = 1 + 49 * j
        rows.append((y0, y0 + 48))
        if j < 9:
            t[y0 + 48, 500:] = WALL
        door = y0 + 22
        t[door:door + 4, 500] = FREE
        protect[door - 2:door + 6, 495:506] = True
    t[490:H - 1, 501:W - 1] = WALL
    add_exit(t, "top", 248, 4)
    add_exit(t, "bottom", 248, 4)
    for j in (1, 8):
        add_exit(t, "right", rows[j][0] + 22, 4)
    for side_x, side_y in ((248, 1), (248, H - 2)):
        protect[max(0, side_y - 3):side_y + 4, side_x - 2:side_x + 6] = True
    for j in (1, 8):
        protect[rows[j][0] + 19:rows[j][0] + 29, W - 6:W] = True
    rng = np.random.default_rng(seed + 1)
    add_obstacles(t, 0.10, rng, protect=protect)
    seal_unreachable(t)
    return Workload(f"corridors1000x500_40k_v{v_m}", t, place_uniform(t, n, seed), v_m, seed=seed)


def config_precision(seed=0, side=4000, n=1_000_000, n_exits=16, v_m=4) -> Workload:
    """4000x4000, 10% rectangles, 16 exits spread over the border, 1,000,000
    agents from a 32-component Gaussian mixture (sigma 1%..8% of the side)."""
    t = room(side, side)
    spread_exits(t, n_exits, 4)
    rng = np.random.default_rng(seed + 1)
    add_obstacles(t, 0.10, rng)
    seal_unreachable(t)
    return Workload(f"gmm{side}x{side}_{n // 1000}k_v{v_m}", t,
                    place_gmm(t, n, 32, seed + 2), v_m, seed=seed)


def config_stress(seed=0, side=16384, n=10_000_000, n_exits=64, v_m=5) -> Workload:
    """16384x16384, 5% rectangles, 64 exits, 10,000,000 agents uniform, v_m=5."""
    t = room(side, side)
    spread_exits(t, n_exits, 4)
    rng = np.random.default_rng(seed + 1)
    add_obstacles(t, 0.05, rng)
    seal_unreachable(t)
    return Workload(f"uniform{side}x{side}_{n // 1000000}M_v{v_m}", t,
                    place_uniform(t, n, seed + 2), v_m, seed=seed)


def config_batch(n_rep=256, seed=0, cells_lo=100 ** 2, cells_hi=2000 ** 2,
                 agents_lo=1000, agents_hi=100_000) -> list[Workload]:
    """n_rep independent replicates: cell count log-uniform in
    [cells_lo, cells_hi] with aspect 1..2, 10% rectangles, 1-4 exits, agents
    log-uniform in [agents_lo, agents_hi] capped at 0.3 per free cell, v_m
    uniform in 1..5, one seed per replicate."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_rep):
        cells = math.exp(rng.uniform(math.log(cells_lo), math.log(cells_hi)))
        aspect = rng.uniform(1.0, 2.0)
        W = max(16, int(round(math.sqrt(cells * aspect))))
        H = max(16, int(round(cells / W)))
        t = room(W, H)
        spread_exits(t, int(rng.integers(1, 5)), 4)
        add_obstacles(t, 0.10, np.random.default_rng(seed * 1000 + r + 1), protect=exit_apron(t))
        seal_unreachable(t)
        free = int((t == FREE).sum())
        n = int(math.exp(rng.uniform(math.log(agents_lo), math.log(agents_hi))))
        n = max(1, min(n, int(0.3 * free)))
        v = int(rng.integers(1, 6))
        rs = int(seed * 100003 + r)
        out.append(Workload(f"rep{r}_{W}x{H}_{n}_v{v}", t, place_uniform(t, n, rs), v, seed=rs))
    return out


def tiny_room(W=12, H=10, n=12, seed=0, v_m=2, walls=(), exits=(("bottom", 4, 2),)) -> Workload:
    """Small hand-sized rooms for brute-force checks."""
    t = room(W, H)
    for (x, y) in walls:
        t[y, x] = WALL
    for side, pos, width in exits:
        add_exit(t, side, pos, width)
    return Workload(f"tiny{W}x{H}", t, place_uniform(t, n, seed), v_m, seed=seed)


def config_fd_corridor(density: float, length=2000, width=20, seed=0, v_m=4) -> Workload:
    """Straight corridor for the fundamental diagram: `length` x `width`
    free cells between walls, closed at the left end, the whole right end an
    exit; agents uniform at `density` (fraction of the free cells)."""
    t = room(length + 2, width + 2)
    add_exit(t, "right", 1, width)
    free = int((t == FREE).sum())
    n = max(1, int(round(density * free)))
    rs = int(seed * 1009 + round(density * 1000))
    return Workload(f"corridor{length}x{width}_d{density:.2f}_v{v_m}", t,
                    place_uniform(t, n, rs), v_m, seed=rs)
