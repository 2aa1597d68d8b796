"""Fundamental diagram of the model in a straight corridor: flow and speed
against density at v_m = 4, a shape check of the remark in Sec. 2 that
v_m = 4 reproduces Weidmann's fundamental diagram (whose data is not used).

Measurement (open corridor, no periodic boundary): agents start uniformly at
density rho in a corridor `length` cells long and `width` wide, closed at
the left end, the whole right end an exit.  The flow through the cross-section
at mid-length is counted over a window of steps that ends well before either
front reaches it: the empty region that opens behind the agents at the closed
end, and the thinning that spreads back from the exit.  There the density
is still rho, so the window gives one point of the diagram per density.
Cells are 0.4 m wide and a step is one
simulated second (Sec. 2): density in persons per m^2 = rho / 0.16, flow in
persons per m and s = crossings per step / (width * 0.4).

Every density runs as one replicate of a single context (the batched form);
positions are read back after every step.

    python -m paper_0911_2900_gb300.fundamental      # JSON lines, one per density
"""
from __future__ import annotations

import json
import sys

import numpy as np

from . import workloads as wl

CELL_M = 0.4
DENSITIES = (0.02, 0.05, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9)


def crossings(prev_cells: np.ndarray, cells: np.ndarray, W: int, xm: int) -> int:
    """Agents (by id) that were left of column xm before a step and are at
    or right of it after it, or have left through the exit (which lies right
    of xm)."""
    was = prev_cells >= 0
    before = np.where(was, prev_cells % W, W) < xm
    now = np.where(cells >= 0, cells % W, W)  # gone: past every column
    return int((was & before & (now >= xm)).sum())


def window(length: int, v_m: int) -> tuple[int, int]:
    """Steps [first, last) whose flow at mid-length is unaffected by the
    fronts from both ends: half the time a front moving v_m cells per step
    needs to get there (in one step of the sequential movement a gap can be
    handed on along a few agents, so a front may run somewhat faster)."""
    last = (length // 2) // (2 * v_m)
    return min(10, last // 2), last


def point(rho_cells: float, width: int, n_steps: int, n_cross: int) -> dict:
    rho_m2 = rho_cells / (CELL_M * CELL_M)
    flow = n_cross / n_steps / (width * CELL_M)
    return {"density_cells": rho_cells, "density_per_m2": rho_m2,
            "flow_per_m_s": flow, "speed_m_s": flow / rho_m2 if rho_m2 > 0 else 0.0,
            "crossings": n_cross, "steps": n_steps}


def measure(densities=DENSITIES, length=2000, width=20, v_m=4, seed=0, steps=None,
            precision="fp32_recheck"):
    """Flow and speed at mid-length for each density, on the GPU."""
    from . import Context

    works = [wl.config_fd_corridor(d, length, width, seed, v_m) for d in densities]
    first, last = steps if steps is not None else window(length, v_m)
    ctx = Context(len(works), precision)
    for r, w in enumerate(works):
        ctx.init_grid(r, w.cell_type, w.k_S, w.v_m, w.seed)
    counts = np.array([len(w.cells) for w in works], np.int32)
    ctx.place_all(counts, np.concatenate([w.cells for w in works]))
    off = np.concatenate([[0], np.cumsum(counts)])
    Wg = works[0].cell_type.shape[1]
    xm = 1 + length // 2
    prev, _, _ = ctx.readback_all(counts)
    n_cross = np.zeros(len(works), np.int64)
    for t in range(last):
        ctx.step(1)
        cells, _, _ = ctx.readback_all(counts)
        if t >= first:
            for r in range(len(works)):
                n_cross[r] += crossings(prev[off[r]:off[r + 1]], cells[off[r]:off[r + 1]], Wg, xm)
        prev = cells
    ctx.close()
    free = [int((w.cell_type == wl.FREE).sum()) for w in works]
    return [dict(point(len(w.cells) / f, width, last - first, int(c)), workload=w.name)
            for w, f, c in zip(works, free, n_cross)]


def main(argv=None) -> int:
    for p in measure():
        print(json.dumps(p), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
