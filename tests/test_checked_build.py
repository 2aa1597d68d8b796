"""The debug build of the library (FASTGB_CHECKED=1): its kernels check every
index they derive from data -- agent and desired cells, candidate and path
cells, mover and re-check queue entries -- and record one out of range as a
device error instead of accessing memory.  On valid inputs it must give the
oracle's trajectories like the release build, with no error; its check
itself is exercised on an index that no access uses.  Runs in a subprocess,
since a process loads one of the two libraries."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import os, sys
import numpy as np
sys.path.insert(0, os.environ["ROOT"])
import oracle
import paper_0911_2900_gb300 as fg
from paper_0911_2900_gb300 import workloads as wl

assert fg.build_checked(), "the debug build is not the one loaded"
assert fg.selftest_bounds(10, 5) == (-4, 10)
assert fg.selftest_bounds(3, 5) == (0, -1)

def run(works, steps, precision="fp32_recheck", reach="l2", lanes=None):
    ctx = fg.Context(len(works), precision, reach)
    ctx.set_option("digests", 1)
    for v, l in (lanes or {}).items():
        ctx.set_option(f"lanes_v{v}", l)
    for r, w in enumerate(works):
        ctx.init_grid(r, w.cell_type, w.k_S, w.v_m, w.seed)
        ctx.place(r, w.cells)
    ctx.step(steps)
    for r, w in enumerate(works):
        cells, des, st = ctx.readback(r, len(w.cells))     # raises on a device error
        dc, dd = ctx.digests(r, steps)
        sim = oracle.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed,
                         reach={"l2": 0, "l2p": 1, "linf": 2}[reach])
        sim.place(w.cells)
        o = sim.run(0, steps, threads=os.cpu_count() or 1)
        assert np.array_equal(dd, o["dig_des"]) and np.array_equal(dc, o["dig_cell"]), w.name
        assert np.array_equal(cells, sim.cells_by_id()), w.name
    ctx.close()

run([wl.config_small_room()], 60)
run([wl.config_small_room(W=90, H=70, n=1500, seed=4, v_m=3)], 30, precision="fp64")
run([wl.config_small_room(W=90, H=70, n=1500, seed=4, v_m=5)], 30, reach="linf")
for lanes in (0, 4):
    run([wl.config_small_room(W=120, H=90, n=3001, seed=9, v_m=4)], 20, lanes={4: lanes})
run([wl.config_corridors(v_m=5)], 40)
run(wl.config_batch(n_rep=5, seed=11, cells_hi=250 ** 2, agents_hi=5000), 24)
print("checked build ok")
'''


def test_checked_build_gives_the_oracles_trajectories():
    env = dict(os.environ, FASTGB_CHECKED="1", ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout


def test_release_build_compiles_the_checks_away():
    import paper_0911_2900_gb300 as fg

    if os.environ.get("FASTGB_CHECKED", "0") == "1":
        pytest.skip("this process runs the debug build")
    assert not fg.build_checked()
    assert fg.selftest_bounds(10, 5) == (0, -1)
