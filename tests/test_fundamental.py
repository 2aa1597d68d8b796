"""Fundamental-diagram shape check (Sec. 2: v_m = 4 is said to reproduce
Weidmann's fundamental diagram; his data is not available, so only the shape
is checked): the corridor workload, the crossing count, parity of the
corridor runs against the oracle, and flow and speed against density from
GPU runs."""
import os

import numpy as np
import pytest

from paper_0911_2900_gb300 import fundamental as fd
from paper_0911_2900_gb300 import workloads as wl


def test_corridor_workload():
    w = wl.config_fd_corridor(0.3, length=300, width=12, seed=2)
    t = w.cell_type
    assert t.shape == (14, 302)
    assert (t[1:-1, -1] == wl.EXIT).all() and (t[1:-1, 0] == wl.WALL).all()
    assert (t[0] == wl.WALL).all() and (t[-1] == wl.WALL).all()
    assert len(w.cells) == round(0.3 * 300 * 12)
    assert (t.ravel()[w.cells] == wl.FREE).all() and len(np.unique(w.cells)) == len(w.cells)


def test_crossings_count():
    W, xm = 20, 10
    prev = np.array([9 + 20, 5, 9, 12, -1, 3 * 20 + 9], np.int32)
    now = np.array([10 + 20, 9, -1, 15, -1, 3 * 20 + 9], np.int32)
    # agent 0 crosses, 1 stays left, 2 leaves through the exit (right of xm),
    # 3 was already right, 4 was gone, 5 stays on column 9
    assert fd.crossings(prev, now, W, xm) == 2


def test_window_stays_ahead_of_the_fronts():
    for length in (400, 1000, 2000):
        first, last = fd.window(length, 4)
        assert 0 <= first < last and last * 4 * 2 <= length // 2


@pytest.mark.gpu
@pytest.mark.parametrize("density", [0.15, 0.6])
def test_corridor_parity(orc, density):
    """The corridor at a low and a high density: GPU trajectories equal the
    oracle's for every agent and step, so the crossing counts are equal."""
    import paper_0911_2900_gb300 as fg

    w = wl.config_fd_corridor(density, length=240, width=10, seed=3)
    steps = 40
    ctx = fg.Context(1, "fp32_recheck")
    ctx.set_option("digests", 1)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    W = w.cell_type.shape[1]
    sim = orc.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed)
    sim.place(w.cells)
    prev_g = ctx.readback(0, len(w.cells))[0]
    prev_o = sim.cells_by_id()
    for t in range(steps):
        ctx.step(1)
        cg = ctx.readback(0, len(w.cells))[0]
        sim.run(t, 1, threads=os.cpu_count() or 1, digests=False)
        co = sim.cells_by_id()
        assert np.array_equal(cg, co), t
        assert fd.crossings(prev_g, cg, W, W // 2) == fd.crossings(prev_o, co, W, W // 2)
        prev_g, prev_o = cg, co


@pytest.mark.gpu
def test_fundamental_diagram_shape():
    """Flow rises with density from free walking, peaks at an intermediate
    density and falls towards the jam; speed falls with density."""
    pts = fd.measure(densities=(0.02, 0.1, 0.2, 0.3, 0.5, 0.7, 0.9), length=1000, width=20)
    flow = np.array([p["flow_per_m_s"] for p in pts])
    speed = np.array([p["speed_m_s"] for p in pts])
    dens = np.array([p["density_cells"] for p in pts])
    peak = int(np.argmax(flow))
    assert 0 < peak < len(pts) - 1, flow
    assert flow[-1] < 0.5 * flow[peak] and flow[0] < flow[peak]
    assert (np.diff(speed) < 0.05).all(), speed
    assert speed[0] > 2 * speed[-1] and abs(dens[3] - 0.3) < 0.01
