"""Pins of the oracle's per-agent maximum speeds.  Sec. 2 notes that its
benchmark gave every agent the same maximum speed; the model itself lets the
agents' speeds differ, and each agent then plans over the reach set of its
own speed (the rest of the step does not depend on the speed).

* one speed given per agent, all equal, reproduces the single-speed run;
* with mixed speeds every agent's weights equal the brute-force enumeration
  (independent Python restatement) for its own speed, and the check tells
  its speed from the next one;
* over many steps with mixed speeds, no agent moves farther than its speed
  allows, no two agents share a cell and agents only leave through exits.
"""
import numpy as np
import pytest

from paper_0911_2900_gb300 import workloads as wl
from tests import refs
from tests.test_oracle_field_plan import _brute_probs, _scene


@pytest.mark.parametrize("v", [1, 3, 5])
def test_equal_speeds_reproduce_one_speed(orc, v):
    w = wl.config_small_room(W=40, H=30, n=300, seed=v, v_m=v)
    a = orc.Sim(w.cell_type, v=v, kS=w.k_S, seed=w.seed)
    a.place(w.cells)
    ra = a.run(0, 25)
    b = orc.Sim(w.cell_type, v=1 if v != 1 else 2, kS=w.k_S, seed=w.seed,
                speeds=np.full(len(w.cells), v, np.uint8))
    b.place(w.cells)
    rb = b.run(0, 25)
    assert np.array_equal(ra["dig_cell"], rb["dig_cell"])
    assert np.array_equal(ra["dig_des"], rb["dig_des"])
    assert np.array_equal(a.cells_by_id(), b.cells_by_id())


def test_each_agent_plans_with_its_own_speed(orc):
    told_apart = 0
    for seed in range(3):
        t, cells = _scene(seed, v=5)
        rng = np.random.default_rng(seed)
        speeds = rng.integers(1, 6, len(cells)).astype(np.uint8)
        sim = orc.Sim(t, v=5, kS=1.2, seed=seed + 5, speeds=speeds)
        sim.place(cells)
        H, W = t.shape
        occ2d = sim.occ.reshape(H, W).tolist()
        for i in range(len(cells)):
            c = int(cells[i])
            v = int(speeds[i])
            d, w, u = sim.plan_agent(i, t=3)
            want = _brute_probs(t, sim.S, occ2d, c % W, c // W, v, 1.2)
            assert len(w) == len(refs.reach_offsets(v))
            assert np.array_equal(w > 0, want > 0)
            np.testing.assert_allclose(w, want, rtol=1e-13, atol=0)
            # the desired cell lies in the agent's own reach set
            dx, dy = d % W - c % W, d // W - c // W
            assert (dx, dy) in refs.reach_offsets(v)
            if v < 5:
                other = _brute_probs(t, sim.S, occ2d, c % W, c // W, v + 1, 1.2)
                told_apart += int((other > 0).sum() != (want > 0).sum())
    assert told_apart > 0


def test_mixed_speeds_invariants(orc):
    w = wl.config_small_room(W=60, H=45, n=900, seed=11, v_m=5)
    n = len(w.cells)
    speeds = np.random.default_rng(3).integers(1, 6, n).astype(np.uint8)
    sim = orc.Sim(w.cell_type, v=5, kS=w.k_S, seed=w.seed, speeds=speeds)
    sim.place(w.cells)
    H, W = w.cell_type.shape
    exits = set(np.flatnonzero(w.cell_type.ravel() == 2).tolist())
    for step in range(40):
        before = sim.cells_by_id().copy()
        desired = sim.plan(step)
        left = sim.move(desired, step)
        after = sim.cells_by_id()
        live = after[after >= 0]
        assert len(np.unique(live)) == len(live)
        assert left == int(((before >= 0) & (after < 0)).sum())
        for i in np.flatnonzero(before >= 0):
            c0 = int(before[i])
            if after[i] >= 0:
                dx, dy = int(after[i]) % W - c0 % W, int(after[i]) // W - c0 // W
                assert max(abs(dx), abs(dy)) <= speeds[i]
            else:
                # it left through an exit on the path to a target in its reach
                tgt = int(desired[i])  # agent index i has id i here
                dx, dy = tgt % W - c0 % W, tgt // W - c0 // W
                assert (dx, dy) in refs.reach_offsets(int(speeds[i]))
                path = [(c0 // W + py) * W + c0 % W + px for px, py in refs.straight_path(dx, dy)]
                assert any(c in exits for c in path)


def test_speeds_are_checked(orc):
    w = wl.config_small_room(W=20, H=20, n=10, seed=1, v_m=2)
    with pytest.raises(ValueError):
        orc.Sim(w.cell_type, v=2, speeds=np.array([0, 1], np.uint8))
    with pytest.raises(ValueError):
        orc.Sim(w.cell_type, v=2, speeds=np.array([6], np.uint8))
    sim = orc.Sim(w.cell_type, v=2, speeds=np.full(5, 2, np.uint8))
    with pytest.raises(ValueError):
        sim.place(w.cells)  # ten agents, five speeds
