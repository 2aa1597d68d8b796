"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Desired cells and trajectories must be identical (bit-exact integers) for
every agent and step: the FP64 planning path replays the oracle's FP64
sequence, and the FP32 path re-evaluates in FP64 every draw that falls within
its error margin of a cumulative boundary.  Whole arrays are compared on
small grids; per-step digests (splitmix64 sums over (id, cell) and
(id, desired)) plus final arrays on the larger ones.
"""
import os

import numpy as np
import pytest

from paper_0911_2900_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

REACH_ORC = {"l2": 0, "l2p": 1, "linf": 2}


@pytest.fixture(scope="module")
def fg():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_0911_2900_gb300 as fg

    fg.load()
    return fg


def run_gpu(fg, works, steps, precision="fp32_recheck", reach="l2", digests=True, resort=8,
            graph=True, id_perm=None, start_step=0, lanes=None, tile_shift=None, chunks=None,
            graph_steps=None, tune=None, speeds=None):
    ctx = fg.Context(len(works), precision, reach)
    ctx.set_option("digests", 1 if digests else 0)
    ctx.set_option("resort_period", resort)
    ctx.set_option("use_graph", 1 if graph else 0)
    if graph_steps is not None:
        ctx.set_option("graph_steps", graph_steps)
    if tile_shift is not None:
        ctx.set_option("tile_shift", tile_shift)
    if lanes is not None:
        for v, g in lanes.items():
            ctx.set_option(f"lanes_v{v}", g)
    for r, w in enumerate(works):
        ctx.init_grid(r, w.cell_type, w.k_S, w.v_m, w.seed)
        if speeds is not None and speeds[r] is not None:
            ctx.set_speeds(r, speeds[r])
        if id_perm is None:
            ctx.place(r, w.cells, start_step=start_step)
        else:
            ctx.place(r, w.cells[id_perm], ids=id_perm.astype(np.int32), start_step=start_step)
    done = 0
    for n in (chunks or [steps]):
        if tune is not None and done == tune:
            ctx.tune_report = ctx.autotune(trials=2)
        ctx.step(n)
        done += n
    assert done == steps
    out = []
    for r, w in enumerate(works):
        cells, des, st = ctx.readback(r, len(w.cells))
        dc, dd = ctx.digests(r, steps) if digests else (None, None)
        out.append(dict(cells=cells, desired=des, stats=st, dig_cell=dc, dig_des=dd))
    return ctx, out


def run_oracle(orc, w, steps, reach="l2", t0=0, threads=None, speeds=None):
    sim = orc.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed, reach=REACH_ORC[reach],
                  speeds=speeds)
    sim.place(w.cells)
    r = sim.run(t0, steps, threads=threads or min(8, os.cpu_count() or 1))
    cells = sim.cells_by_id()
    return dict(cells=cells, desired=r["desired"], dig_cell=r["dig_cell"],
                dig_des=r["dig_des"], alive=r["alive"], sim=sim)


def assert_same(g, o, steps):
    assert len(g["dig_cell"]) == steps
    bad = np.flatnonzero(g["dig_des"] != o["dig_des"])
    assert len(bad) == 0, f"desired digests differ first at step {bad[0]}"
    bad = np.flatnonzero(g["dig_cell"] != o["dig_cell"])
    assert len(bad) == 0, f"cell digests differ first at step {bad[0]}"
    assert np.array_equal(g["cells"], o["cells"])
    alive = o["cells"] >= 0
    assert np.array_equal(g["desired"][alive], o["desired"][alive])
    assert g["stats"]["alive"] == int(alive.sum())


# --------------------------------------------------------------------------- self tests
def test_exp64_bitwise_equal_to_oracle(fg, orc):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-13, 13, 200_000), rng.uniform(-700, 700, 20_000),
                        np.array([0.0, -0.0, 1.0, -1.0, 0.5, -0.5])])
    y = fg.selftest_exp64(x)
    want = np.array([orc.exp64(float(v)) for v in x])
    assert np.array_equal(y.view(np.uint64), want.view(np.uint64))


def test_philox_bitwise_equal_to_oracle(fg, orc):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, (5000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (5000, 2), dtype=np.uint64).astype(np.uint32)
    out = fg.selftest_philox(ctr, key)
    for i in range(0, 5000, 7):
        assert out[i].tolist() == orc.philox(ctr[i], key[i]).tolist()


def test_ex2_error_within_margin_budget(fg):
    """The margin assumes the SFU 2^y has relative error <= 2^-21 on the
    weights' argument range; measure it exhaustively and demand a factor 2."""
    err = fg.selftest_ex2(-16.0, 16.0)
    assert err <= 2.0 ** -22, err


def test_bounded_barrier_reports_timeout(fg):
    assert fg.selftest_barrier_timeout(2_000_000) == -5


@pytest.mark.parametrize("per_sm", [1, 2])
def test_grid_barrier_sums_counts_exactly(fg, per_sm):
    """The movement rounds take the number of agents still waiting from the
    grid barrier's count sum; on a full grid every block must see the exact
    total at every barrier (both alternating words, 1000 barriers)."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert fg.selftest_barrier_sum(per_sm * sms, 512, 1000) == 0
    ns = fg.selftest_barrier_cost(per_sm * sms, 512, 1000)
    assert 0 < ns < 20_000, ns


# --------------------------------------------------------------------------- parity
@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck"])
def test_room200_2k_v4(fg, orc, precision):
    """The plain-method workload (200x200 room, one exit, 2,000 agents,
    v_m=4) for the paper's whole run of 396 steps (Sec. 2), in both
    precisions."""
    w = wl.config_small_room()
    steps = 396
    _, (g,) = run_gpu(fg, [w], steps, precision)
    o = run_oracle(orc, w, steps, threads=os.cpu_count() or 1)
    assert_same(g, o, steps)


@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck"])
@pytest.mark.parametrize("v", [1, 2, 3, 4, 5])
def test_corridors_40k_vsweep(fg, orc, v, precision):
    """The v_m sweep workload (1000x500 room and corridors, 40,000 agents)
    at every v_m for all 396 steps, in both precisions."""
    w = wl.config_corridors(v_m=v)
    steps = 396
    _, (g,) = run_gpu(fg, [w], steps, precision)
    o = run_oracle(orc, w, steps, threads=os.cpu_count() or 1)
    assert_same(g, o, steps)


@pytest.mark.parametrize("reach", ["l2p", "linf"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck"])
def test_reach_variants(fg, orc, reach, precision):
    w = wl.config_small_room(W=90, H=70, n=1500, seed=4, v_m=5 if reach == "linf" else 3)
    steps = 40
    _, (g,) = run_gpu(fg, [w], steps, precision, reach=reach)
    o = run_oracle(orc, w, steps, reach=reach)
    assert_same(g, o, steps)


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("v", [1, 4, 5])
def test_lanes_per_agent_variants(fg, orc, lanes, v):
    """Every planning variant (tiled, one thread, 2/4/8 lanes per agent) at
    the smallest reach set, the benchmark's and the largest (two mask words)."""
    w = wl.config_small_room(W=120, H=90, n=3001, seed=5 + v, v_m=v)
    steps = 25
    _, (g,) = run_gpu(fg, [w], steps, "fp32_recheck", lanes={v: lanes})
    o = run_oracle(orc, w, steps)
    assert_same(g, o, steps)


def test_caller_floor_field(fg, orc):
    """A caller's static floor field (fast_grid_desc.static_field): the
    library's own field passed back gives the same trajectories, and a field
    computed around a wall that is not in the grid (agents are steered
    around it but may cross it) gives the oracle's trajectories with the same
    field."""
    t = wl.room(90, 70)
    wl.add_exit(t, "bottom", 40, 4)
    wl.add_exit(t, "left", 20, 3)
    cells = wl.place_uniform(t, 2500, 5)
    tv = t.copy()
    tv[35, 10:80] = wl.WALL
    _, _, vS = orc.floor_field(tv)
    vS[35, 10:80] = 500.0 + 3 * np.sqrt(2.0)
    S0 = fg.floor_field(t)[0]
    steps = 60
    for field in (S0, vS):
        w = wl.Workload("field", t, cells, 4, seed=77)
        ctx = fg.Context(1, "fp32_recheck")
        ctx.set_option("digests", 1)
        ctx.init_grid(0, t, w.k_S, w.v_m, w.seed, static_field=field)
        ctx.place(0, cells)
        ctx.step(steps)
        c, d, st = ctx.readback(0, len(cells))
        dc, dd = ctx.digests(0, steps)
        sim = orc.Sim(t, v=4, kS=w.k_S, seed=w.seed, S=field)
        sim.place(cells)
        r = sim.run(0, steps, threads=os.cpu_count() or 1)
        o = dict(cells=sim.cells_by_id(), desired=r["desired"], dig_cell=r["dig_cell"],
                 dig_des=r["dig_des"])
        assert_same(dict(cells=c, desired=d, stats=st, dig_cell=dc, dig_des=dd), o, steps)
    with pytest.raises(fg.FastError):
        bad = S0.copy()
        bad[10, 10] += 1e-9
        fg.Context(1, "fp32_recheck").init_grid(0, t, 1.2, 4, 0, static_field=bad)


@pytest.mark.parametrize("k_S", [0.0, 0.35, 5.0])
def test_coupling_strengths(fg, orc, k_S):
    """k_S = 0 (every admissible candidate equally likely: FP32 weights are
    exactly 1), a weak coupling, and a strong one (weights spread over many
    binades)."""
    w0 = wl.config_small_room(W=80, H=70, n=1500, seed=31, v_m=3)
    w = wl.Workload(w0.name, w0.cell_type, w0.cells, w0.v_m, seed=w0.seed, k_S=k_S)
    steps = 30
    _, (g,) = run_gpu(fg, [w], steps, "fp32_recheck")
    o = run_oracle(orc, w, steps)
    assert_same(g, o, steps)


def test_storage_order_graph_and_resort_do_not_matter(fg, orc):
    w = wl.config_small_room(W=100, H=100, n=2500, seed=6, v_m=4)
    steps = 30
    o = run_oracle(orc, w, steps)
    perm = np.random.default_rng(3).permutation(len(w.cells))
    for kw in (dict(), dict(id_perm=perm), dict(graph=False), dict(resort=0), dict(resort=1),
               dict(tile_shift=2)):
        _, (g,) = run_gpu(fg, [w], steps, "fp32_recheck", **kw)
        assert_same(g, o, steps)


def test_step_loop_graph_modes(fg, orc):
    """The step loop as one captured graph per call, one graph per step,
    direct launches, and calls that start at every phase of the re-sort
    period all give the oracle's trajectories."""
    w = wl.config_small_room(W=90, H=70, n=1800, seed=12, v_m=3)
    steps = 29
    o = run_oracle(orc, w, steps)
    for kw in (dict(), dict(graph_steps=1), dict(graph=False),
               dict(chunks=[3, 5, 1, 7, 2, 11]), dict(chunks=[1] * 29, graph_steps=0),
               dict(chunks=[13, 13, 3])):
        _, (g,) = run_gpu(fg, [w], steps, "fp32_recheck", **kw)
        assert_same(g, o, steps)


@pytest.mark.parametrize("reserve,tag", [(0, 240), (254, None), (96, None), (96, 200)])
def test_claim_tag_cleanups(fg, orc, reserve, tag):
    """Movement claims whose tags run out within a step (cleared by the
    rounds kernel), before every step, or every few steps: same
    trajectories."""
    w = wl.config_small_room(W=70, H=70, n=2200, seed=21, v_m=5)
    steps = 20
    o = run_oracle(orc, w, steps)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.set_option("digests", 1)
    ctx.set_option("claim_reserve", reserve)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    for i in range(steps):
        if tag is not None:
            ctx.set_option("claim_tag", tag)
        ctx.step(1)
    cells, des, st = ctx.readback(0, len(w.cells))
    dc, dd = ctx.digests(0, steps)
    assert_same(dict(cells=cells, desired=des, stats=st, dig_cell=dc, dig_des=dd), o, steps)


def test_dense_room_and_batch(fg, orc):
    """A room four fifths full (long priority chains in the movement rounds)
    next to a batch of replicates in one context: the oracle's trajectories
    for every replicate."""
    t2 = wl.room(40, 32)
    wl.add_exit(t2, "left", 12, 3)
    wl.add_exit(t2, "top", 20, 2)
    free = np.flatnonzero(t2.ravel() == wl.FREE)
    cells = np.sort(np.random.default_rng(9).choice(free, int(0.8 * len(free)), replace=False))
    dense = wl.Workload("dense", t2, cells.astype(np.int32), 5, seed=12)
    works = [dense] + wl.config_batch(n_rep=3, seed=17, cells_hi=200 ** 2, agents_hi=4000)
    steps = 40
    _, gs = run_gpu(fg, works, steps, "fp32_recheck")
    for w, g in zip(works, gs):
        assert_same(g, run_oracle(orc, w, steps), steps)


def test_autotune_changes_speed_not_results(fg, orc):
    """Tuning in the middle of a run (re-sort bucket side and the planning
    variant of every v_m present) leaves the trajectories bit-exact."""
    works = wl.config_batch(n_rep=5, seed=11, cells_hi=250 ** 2, agents_hi=5000)
    steps = 24
    ctx, gs = run_gpu(fg, works, steps, "fp32_recheck", chunks=[10, 14], tune=10)
    rep = ctx.tune_report
    assert rep["tile_shift"] in (3, 4, 5, 6)
    for w in works:
        assert rep["lanes"][w.v_m - 1] in (0, 1, 2, 4, 8)
        assert len(rep["lanes_us"][w.v_m]) == 5
    for w, g in zip(works, gs):
        assert_same(g, run_oracle(orc, w, steps), steps)


def test_autotune_cache_roundtrip(fg, tmp_path):
    w = wl.config_small_room(W=60, H=60, n=500, seed=2, v_m=2)
    cache = str(tmp_path / "tune.json")
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    first = ctx.autotune(trials=1, cache=cache, key="room60")
    second = ctx.autotune(trials=1, cache=cache, key="room60")
    assert not first["cached"] and second["cached"]
    assert second["lanes"] == first["lanes"] and second["tile_shift"] == first["tile_shift"]
    with pytest.raises(fg.FastError):
        ctx.autotune(trials=0)


def test_place_all_and_readback_all_match_per_replicate_calls(fg, orc):
    """Placing and reading every replicate in one call gives the same
    trajectories as the per-replicate calls (and the oracle); a bad cell in
    one replicate empties only the replicates that failed."""
    works = wl.config_batch(n_rep=4, seed=5, cells_hi=200 ** 2, agents_hi=3000)
    steps = 12
    ctx = fg.Context(len(works), "fp32_recheck")
    for r, w in enumerate(works):
        ctx.init_grid(r, w.cell_type, w.k_S, w.v_m, w.seed)
    counts = np.array([len(w.cells) for w in works], np.int32)
    ctx.place_all(counts, np.concatenate([w.cells for w in works]))
    ctx.step(6)
    cells, des, alive = ctx.readback_all(counts)
    ctx.place_all(counts, cells, start_step=6)       # the read-back state, placed again
    ctx.step(6)
    cells, des, alive = ctx.readback_all(counts)
    off = np.concatenate([[0], np.cumsum(counts)])
    for r, w in enumerate(works):
        o = run_oracle(orc, w, steps)
        assert np.array_equal(cells[off[r]:off[r + 1]], o["cells"])
        assert alive[r] == int((o["cells"] >= 0).sum())
    bad = cells.copy()
    bad[off[2]] = 0                                    # a wall (the top-left corner)
    with pytest.raises(fg.FastError):
        ctx.place_all(counts, bad, start_step=12)
    _, _, alive = ctx.readback_all(counts)
    assert alive[2] == 0 and alive[0] == int((cells[off[0]:off[1]] >= 0).sum())


def test_allocation_failure_is_reported_and_recoverable(fg, orc):
    """The allocator refuses device memory (a 64 MB limit on the context,
    below what a 3000x3000 grid needs: its records fit, its line-of-sight
    masks do not): fast_init_grid returns FAST_ENOMEM, the replicate is left
    without a grid (placing agents is refused), and the same context then
    runs a small grid exactly as the oracle does."""
    ctx = fg.Context(1, "fp32_recheck", memory_limit=64 << 20)
    big = wl.room(3000, 3000)
    wl.add_exit(big, "bottom", 1500, 4)
    with pytest.raises(fg.FastError) as e:
        ctx.init_grid(0, big, 1.2, 4, 0)
    assert e.value.code == -3
    with pytest.raises(fg.FastError) as e:
        ctx.place(0, np.array([3001 + 5], np.int32))
    assert e.value.code == -2
    w = wl.config_small_room(W=60, H=50, n=500, seed=1, v_m=4)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    steps = 5
    ctx.step(steps)
    cells, _, st = ctx.readback(0, len(w.cells))
    assert st["step"] == steps
    assert np.array_equal(cells, run_oracle(orc, w, steps)["cells"])
    ctx.close()


def test_seeded_uniform_placement(fg, orc):
    """fast_place_agents without cells places ids 0..n-1 on distinct free
    cells from which an exit can be reached, drawn from the grid's seed: the
    same grid, seed and count give the same cells, another seed others; a
    walled-in pocket of free cells gets no agent; more agents than such cells
    are refused; and the run from the drawn cells equals the oracle's."""
    t = wl.room(80, 60)
    wl.add_exit(t, "bottom", 40, 4)
    t[20:31, 20] = wl.WALL  # a closed pocket of 9x9 free cells
    t[20:31, 30] = wl.WALL
    t[20, 20:31] = wl.WALL
    t[30, 20:31] = wl.WALL
    pocket = np.zeros(t.shape, bool)
    pocket[21:30, 21:30] = True
    eligible = ((t == wl.FREE) & ~pocket).ravel()
    n_el = int(eligible.sum())
    n = int(0.9 * n_el)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, t, 1.2, 4, 123)
    ctx.place_uniform(0, n)
    cells, _, _ = ctx.readback(0, n)
    assert (cells >= 0).all() and len(np.unique(cells)) == n
    assert eligible[cells].all()
    ctx.place_uniform(0, n)
    assert np.array_equal(ctx.readback(0, n)[0], cells)
    other = fg.Context(1, "fp32_recheck")
    other.init_grid(0, t, 1.2, 4, 124)
    other.place_uniform(0, n)
    assert not np.array_equal(other.readback(0, n)[0], cells)
    other.close()
    with pytest.raises(fg.FastError) as e:
        ctx.place_uniform(0, n_el + 1)
    assert e.value.code == -1
    ctx.place_uniform(0, n)
    steps = 15
    ctx.step(steps)
    got = ctx.readback(0, n)[0]
    sim = orc.Sim(t, v=4, kS=1.2, seed=123)
    sim.place(cells)
    sim.run(0, steps, threads=os.cpu_count() or 1, digests=False)
    want = np.full(n, -1, np.int32)
    o = sim.cells_by_id()
    want[:len(o)] = o
    assert np.array_equal(got, want)
    ctx.close()


def test_place_all_mixed_replicates(fg, orc):
    """One batched placement that leaves one replicate as it is (count -1),
    places another's read-back state again with some agents moved, removed
    and brought back (same ids: each agent goes back to its id's storage
    slot), and gives a third fewer agents (stored by id, then sorted): every
    replicate then follows the oracle from its own state."""
    works = wl.config_batch(n_rep=3, seed=9, cells_hi=150 ** 2, agents_hi=2000)
    ctx = fg.Context(len(works), "fp32_recheck")
    for r, w in enumerate(works):
        ctx.init_grid(r, w.cell_type, w.k_S, w.v_m, w.seed)
    counts = np.array([len(w.cells) for w in works], np.int32)
    ctx.place_all(counts, np.concatenate([w.cells for w in works]))
    ctx.step(10)
    cells, _, _ = ctx.readback_all(counts)
    t = ctx.readback(0, 0)[2]["step"]
    off = np.concatenate([[0], np.cumsum(counts)])
    state = [cells[off[r]:off[r + 1]].copy() for r in range(3)]
    rng = np.random.default_rng(4)
    s1 = state[1]
    present, left = np.flatnonzero(s1 >= 0), np.flatnonzero(s1 < 0)
    assert len(left) > 0
    moved = rng.choice(present, 30, replace=False)
    removed = rng.choice(np.setdiff1d(present, moved), 20, replace=False)
    back = rng.choice(left, min(10, len(left)), replace=False)
    free = np.flatnonzero(works[1].cell_type.ravel() == wl.FREE)
    to = rng.choice(np.setdiff1d(free, s1[present]), len(moved) + len(back), replace=False)
    s1[moved] = to[:len(moved)]
    s1[back] = to[len(moved):]
    s1[removed] = -1
    state[2] = state[2][:len(state[2]) - 50]
    new_counts = np.array([-1, len(s1), len(state[2])], np.int32)
    ctx.place_all(new_counts, np.concatenate([s1, state[2]]), start_step=t)
    steps = 4
    ctx.step(steps)
    read_counts = np.array([len(state[0]), len(s1), len(state[2])], np.int32)
    got, _, alive = ctx.readback_all(read_counts)
    roff = np.concatenate([[0], np.cumsum(read_counts)])
    for r, w in enumerate(works):
        ids = np.flatnonzero(state[r] >= 0).astype(np.int32)
        sim = orc.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed)
        sim.place(state[r][ids], ids=ids)
        sim.run(t, steps, threads=os.cpu_count() or 1, digests=False)
        want = np.full(read_counts[r], -1, np.int32)
        o = sim.cells_by_id()
        want[:len(o)] = o
        assert np.array_equal(got[roff[r]:roff[r + 1]], want), r
        assert alive[r] == int((want >= 0).sum()), r
    ctx.close()


def test_batched_replicates(fg, orc):
    works = wl.config_batch(n_rep=6, seed=3, cells_hi=300 ** 2, agents_hi=6000)
    steps = 30
    _, gs = run_gpu(fg, works, steps, "fp32_recheck")
    for w, g in zip(works, gs):
        assert_same(g, run_oracle(orc, w, steps), steps)


def test_resume_is_bit_exact(fg, orc):
    w = wl.config_small_room(W=80, H=80, n=1200, seed=8, v_m=4)
    ctx, (g20,) = run_gpu(fg, [w], 20, "fp32_recheck", digests=False)
    ctx1, (g10,) = run_gpu(fg, [w], 10, "fp32_recheck", digests=False)
    alive = np.flatnonzero(g10["cells"] >= 0).astype(np.int32)
    ctx2 = fg.Context(1, "fp32_recheck")
    ctx2.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx2.place(0, g10["cells"][alive], ids=alive, start_step=10)
    ctx2.step(10)
    cells, _, st = ctx2.readback(0, len(w.cells))
    assert np.array_equal(cells, g20["cells"])
    # the cells-by-id array as read back (-1: left) placed again as it is
    ctx3 = fg.Context(1, "fp32_recheck")
    ctx3.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx3.place(0, g10["cells"], start_step=10)
    ctx3.step(10)
    cells3, _, st3 = ctx3.readback(0, len(w.cells))
    assert np.array_equal(cells3, g20["cells"])
    assert st3["alive"] == st["alive"]


def test_edge_cases(fg, orc):
    # no agents at all
    t = wl.room(30, 20)
    wl.add_exit(t, "bottom", 10, 4)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, t, 1.2, 4, 0)
    ctx.place(0, np.zeros(0, np.int32))
    ctx.step(3)
    cells, des, st = ctx.readback(0, 0)
    assert st["alive"] == 0
    # one agent next to the exit leaves
    w = wl.Workload("one", t, np.array([18 * 30 + 11], np.int32), 4, seed=2)
    _, (g,) = run_gpu(fg, [w], 5, "fp32_recheck")
    o = run_oracle(orc, w, 5)
    assert_same(g, o, 5)
    # a packed room (every free cell taken but a few): rounds with long chains
    t2 = wl.room(24, 24)
    wl.add_exit(t2, "left", 10, 3)
    free = np.flatnonzero(t2.ravel() == wl.FREE)
    cells = np.sort(np.random.default_rng(0).choice(free, len(free) - 9, replace=False))
    w2 = wl.Workload("packed", t2, cells.astype(np.int32), 5, seed=4)
    _, (g2,) = run_gpu(fg, [w2], 60, "fp32_recheck")
    assert_same(g2, run_oracle(orc, w2, 60), 60)
    # k_S = 0 (uniform choice)
    w3 = wl.config_small_room(W=50, H=40, n=300, seed=2, v_m=3)
    w3.k_S = 0.0
    _, (g3,) = run_gpu(fg, [w3], 20, "fp32_recheck")
    assert_same(g3, run_oracle(orc, w3, 20), 20)


def test_invalid_inputs_are_rejected(fg):
    t = wl.room(20, 20)
    wl.add_exit(t, "top", 5, 2)
    ctx = fg.Context(1, "fp32_recheck")
    with pytest.raises(fg.FastError):
        ctx.place(0, [25])                      # grid not set
    with pytest.raises(fg.FastError):
        ctx.init_grid(0, t, 1.2, 6, 0)          # v_m out of range
    with pytest.raises(fg.FastError):
        ctx.init_grid(0, wl.room(20, 20), 1.2, 4, 0)   # no exit
    ctx.init_grid(0, t, 1.2, 4, 0)
    for bad in ([0], [5], [25, 25], [20 * 20]):  # wall, exit, duplicate, outside
        with pytest.raises(fg.FastError):
            ctx.place(0, bad)
    with pytest.raises(fg.FastError):
        ctx.place(0, [25, 26], ids=[3, 3])     # duplicate ids
    with pytest.raises(fg.FastError):
        ctx.place(0, [25], ids=[1 << 24])      # id too large
    _, _, st = ctx.readback(0, 0)
    assert st["alive"] == 0                    # a rejected placement leaves no agents
    ctx.place(0, [25, 47])
    ctx.step(2)
    ctx.readback(0)


# --------------------------------------------------------------------------- full size
def oracle_batch(orc, works, steps):
    """The oracle on every replicate, several replicates at a time on host
    threads (the C oracle releases the interpreter lock; no process fork)."""
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(lambda w: run_oracle(orc, w, steps, threads=1), works))


def test_batched_form_full_size(fg, orc):
    """All 256 replicates of the batched form (grids 100^2..2000^2 cells,
    1e3..1e5 agents, v_m 1..5) in one context, autotuned, the step loop as
    one graph launch as the benchmark runs it: every replicate's per-step
    desired and cell digests and its final positions and desired cells equal
    the oracle's, run from the same start, for the configuration's 396
    steps."""
    works = wl.config_batch()
    steps = 396
    ctx = fg.Context(len(works), "fp32_recheck")
    ctx.set_option("digests", 1)
    for r, w in enumerate(works):
        ctx.init_grid(r, w.cell_type, w.k_S, w.v_m, w.seed)
        ctx.place(r, w.cells)
    ctx.autotune(trials=2)
    ctx.step(steps)
    outs = oracle_batch(orc, works, steps)
    for r, (w, o) in enumerate(zip(works, outs)):
        cells, des, st = ctx.readback(r, len(w.cells))
        dc, dd = ctx.digests(r, steps)
        assert_same(dict(cells=cells, desired=des, stats=st, dig_cell=dc, dig_des=dd), o, steps)
        assert st["alive"] + st["exited"] == len(w.cells)


def test_precision_form_full_length(fg, orc):
    """4000x4000, 1M clustered agents, v_m=4, FP32 + FP64 re-check, autotuned
    as the benchmark runs it, for the paper's whole run of 396 steps from the
    workload's own start: per-step digests of desired cells and positions,
    and the final arrays, equal the oracle's for every agent and step.  The
    FP32-only draws of the first step flip only inside the margin."""
    w = wl.config_precision()
    steps = 396
    ctx = fg.Context(1, "fp32_recheck")
    ctx.set_option("digests", 1)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    ctx.autotune(trials=2)
    rep = ctx.precision_report()
    assert rep["flips_unflagged"] == 0 and rep["flips_after_recheck"] == 0
    assert rep["flagged"] < 0.01 * rep["agents"]
    ctx.step(steps)
    cells, des, st = ctx.readback(0, len(w.cells))
    # the read-back's stats carry the report's diagnostics
    assert st["diag_flips"] == rep["flips"] and st["diag_max_abs_dp"] == rep["max_abs_dp"]
    dc, dd = ctx.digests(0, steps)
    o = run_oracle(orc, w, steps, threads=os.cpu_count() or 1)
    assert_same(dict(cells=cells, desired=des, stats=st, dig_cell=dc, dig_des=dd), o, steps)


def test_stats_carry_the_precision_report(fg):
    """fast_readback's stats give the last precision report's FP32-only
    flip count and largest |p32 - p64| (zero before any report)."""
    w = wl.config_small_room(W=120, H=90, n=4000, seed=8, v_m=5)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    ctx.step(3)
    st = ctx.readback(0, 0)[2]
    assert st["diag_flips"] == 0 and st["diag_max_abs_dp"] == 0.0
    rep = ctx.precision_report()
    st = ctx.readback(0, 0)[2]
    assert st["diag_flips"] == rep["flips"]
    assert st["diag_max_abs_dp"] == rep["max_abs_dp"] > 0.0
    ctx.close()


def test_recheck_mid_length_queue(fg, orc):
    """The FP64 re-check takes 2, 4 or 8 queued agents per block by the
    queue's length (2 up to one agent per 8 blocks of its 16-per-SM grid, 4 up
    to one per 2 blocks); the corridors and precision workloads take 2 and 8.
    A quarter-size clustered workload (2000x2000, 250k agents) queues a
    length in between: its 12 steps from the start equal the oracle's."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = wl.config_precision(side=2000, n=250_000)
    steps = 12
    ctx, (g,) = run_gpu(fg, [w], steps, "fp32_recheck")
    per_step = g["stats"]["rechecked"] / steps
    assert 2 * sms < per_step <= 8 * sms, per_step
    assert_same(g, run_oracle(orc, w, steps, threads=os.cpu_count() or 1), steps)
    ctx.close()


def test_placing_the_read_back_state_again(fg, orc):
    """Placing a replicate again with implicit ids and the same count keeps
    each agent in its id's storage slot (ids without one are added after the
    others) and skips the sort before the next step.  Run as the end-to-end
    loop does (place what was read back, step, read back), and with the
    read-back state changed before it is placed again (agents moved to other
    free cells, some removed, agents that had left brought back), the cells
    equal the oracle's sequential run from the same state."""
    w = wl.config_small_room(W=120, H=90, n=3000, seed=7, v_m=4)
    n = len(w.cells)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    ctx.step(12)  # sorts, and drops agents that left, on the way
    cells, _, st = ctx.readback(0, n)
    t = st["step"]
    free = np.flatnonzero(w.cell_type.ravel() == wl.FREE)
    rng = np.random.default_rng(3)
    for case in range(4):
        new = cells.copy()
        if case >= 2:
            present = np.flatnonzero(new >= 0)
            left = np.flatnonzero(new < 0)
            assert len(left) > 0
            moved = rng.choice(present, 40, replace=False)
            removed = rng.choice(np.setdiff1d(present, moved), 25, replace=False)
            back = rng.choice(left, min(20, len(left)), replace=False)
            open_cells = np.setdiff1d(free, new[present])
            to = rng.choice(open_cells, len(moved) + len(back), replace=False)
            new[moved] = to[:len(moved)]
            new[back] = to[len(moved):]
            new[removed] = -1
        ids = np.flatnonzero(new >= 0).astype(np.int32)
        sim = orc.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed)
        sim.place(new[ids], ids=ids)
        for k in range(3):  # one step at a time, read back in between
            ctx.place(0, new, start_step=t)
            ctx.step(1)
            new, _, st = ctx.readback(0, n)
            sim.run(t, 1, threads=os.cpu_count() or 1, digests=False)
            want = np.full(n, -1, np.int32)
            o = sim.cells_by_id()
            want[:len(o)] = o
            assert np.array_equal(new, want), (case, k)
            assert st["step"] == t + 1
            t += 1
        cells = new
    ctx.close()


def test_stress_form_from_start(fg, orc):
    """16384x16384, 10M uniform agents, v_m=5, FP32 + FP64 re-check, spatial
    re-sort every 8 steps: 24 steps from the workload's own start (three
    re-sorts) with per-step digests and the final arrays equal to the
    oracle's; the FP32-only draws of the first step flip only inside the
    margin."""
    w = wl.config_stress()
    steps = 24
    ctx = fg.Context(1, "fp32_recheck")
    ctx.set_option("digests", 1)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    rep = ctx.precision_report()
    assert rep["flips_unflagged"] == 0 and rep["flips_after_recheck"] == 0
    assert rep["flagged"] < 0.02 * rep["agents"]
    ctx.step(steps)
    cells, des, st = ctx.readback(0, len(w.cells))
    dc, dd = ctx.digests(0, steps)
    ctx.close()
    o = run_oracle(orc, w, steps, threads=os.cpu_count() or 1)
    assert_same(dict(cells=cells, desired=des, stats=st, dig_cell=dc, dig_des=dd), o, steps)
    assert st["alive"] + st["exited"] == len(w.cells)


# --------------------------------------------------------------------------- speeds per agent
def _speeds(n, seed, lo=1, hi=5):
    return np.random.default_rng(seed).integers(lo, hi + 1, n).astype(np.uint8)


@pytest.mark.parametrize("precision,lanes", [("fp64", None), ("fp32_recheck", 0),
                                             ("fp32_recheck", 1), ("fp32_recheck", 2),
                                             ("fp32_recheck", 4), ("fp32_recheck", 8)])
def test_per_agent_speeds(fg, orc, precision, lanes):
    """Agents of one replicate with maximum speeds 1..5 of their own: each
    speed's planning launch plans only its agents, over its reach set and
    line-of-sight mask; the re-sort keeps the speed classes apart; the FP64
    re-check uses each agent's speed.  Bit-equal to the oracle."""
    w = wl.config_small_room(W=80, H=60, n=1500, seed=21, v_m=3)
    sp = _speeds(len(w.cells), 5)
    lanes_by_v = None if lanes is None else {v: lanes for v in range(1, 6)}
    steps = 60
    _, (g,) = run_gpu(fg, [w], steps, precision, speeds=[sp], lanes=lanes_by_v)
    o = run_oracle(orc, w, steps, speeds=sp)
    assert_same(g, o, steps)


def test_per_agent_speeds_batched_with_uniform_replicates(fg, orc):
    """A batch mixing replicates with speeds per agent and replicates with one
    speed: every replicate joins the planning launch of each speed it has."""
    ws = [wl.config_small_room(W=50 + 10 * i, H=40, n=500 + 100 * i, seed=30 + i, v_m=1 + i)
          for i in range(4)]
    sps = [_speeds(len(ws[0].cells), 7, 2, 4), None, _speeds(len(ws[2].cells), 8), None]
    steps = 40
    _, gs = run_gpu(fg, ws, steps, "fp32_recheck", speeds=sps)
    for w, sp, g in zip(ws, sps, gs):
        assert_same(g, run_oracle(orc, w, steps, speeds=sp), steps)


def test_speeds_equal_to_v_m_change_nothing(fg, orc):
    w = wl.config_small_room(W=60, H=50, n=800, seed=41, v_m=4)
    steps = 30
    _, (a,) = run_gpu(fg, [w], steps)
    _, (b,) = run_gpu(fg, [w], steps, speeds=[np.full(len(w.cells), 4, np.uint8)])
    assert np.array_equal(a["dig_cell"], b["dig_cell"])
    assert np.array_equal(a["dig_des"], b["dig_des"])
    assert np.array_equal(a["cells"], b["cells"])


def test_speeds_are_checked_by_the_library(fg):
    w = wl.config_small_room(W=30, H=30, n=50, seed=2, v_m=2)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    with pytest.raises(fg.FastError):
        ctx.set_speeds(0, np.array([1, 0, 3], np.uint8))  # speed 0
    with pytest.raises(fg.FastError):
        ctx.set_speeds(0, np.array([6], np.uint8))  # speed 6
    ctx.set_speeds(0, np.full(10, 3, np.uint8))  # fewer ids than agents
    with pytest.raises(fg.FastError):
        ctx.place(0, w.cells)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)  # drops the speeds
    ctx.set_speeds(0, np.full(len(w.cells), 3, np.uint8))
    ctx.place(0, w.cells)
    with pytest.raises(fg.FastError):
        ctx.set_speeds(0, np.full(len(w.cells), 2, np.uint8))  # agents already placed
    ctx.step(3)
    ctx.close()
