"""The allocation-free planning pass (fast_plan_noalloc) against the regular
one and against the FP64 oracle.

fast_plan_noalloc serves callers that cannot allocate device memory when
they plan (for instance while they capture a CUDA graph on their stream); its
only scratch is a fixed array inside the library.  It must give exactly the
desired cells of a regular planning pass (fast_plan_only + fast_readback) and
of the oracle, call after call, although every call reuses the same array,
including the draws that the FP64 re-check settles.  This file is collected
last on purpose.
"""
import os

import numpy as np
import pytest

from paper_0911_2900_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_0911_2900_gb300 as fg

    return fg


def oracle_plan(orc, w, reach, t):
    """The oracle's desired cells (by id) at step t, run from the start."""
    sim = orc.Sim(w.cell_type, v=w.v_m, kS=w.k_S, seed=w.seed, reach={"l2": 0, "linf": 2}[reach])
    sim.place(w.cells)
    if t:
        sim.run(0, t, threads=os.cpu_count() or 1, digests=False)
    des = sim.plan(t, threads=os.cpu_count() or 1)
    out = np.full(len(w.cells), -1, np.int32)
    out[sim.id] = np.where(sim.cell >= 0, des, -1)
    return out


@pytest.mark.parametrize("reach", ["l2", "linf"])
@pytest.mark.parametrize("v", [1, 4, 5])
def test_plan_noalloc_matches_regular_planning_and_oracle(fg, orc, v, reach):
    import torch

    w = wl.config_corridors(v_m=v)
    n = len(w.cells)
    ctx = fg.Context(1, "fp32_recheck", reach)
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    ctx.step(2)
    rechecked_calls = 0
    for call in range(2):   # two calls in a row share the fixed scratch array
        _, _, st0 = ctx.readback(0, 0)
        ctx.plan_only(1)
        cells, want, st = ctx.readback(0, n)
        rechecked_calls += st["rechecked"] > st0["rechecked"]
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        ctx.plan_noalloc(0, st["step"], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        present = cells >= 0
        assert present.sum() > 0
        assert np.array_equal(got[present], want[present]), f"call {call}"
        assert (got[~present] == -7).all()
        assert np.array_equal(got[present], oracle_plan(orc, w, reach, st["step"])[present])
        # an output shorter than the largest id: only ids below its length
        # are written, the rest of the buffer is left alone
        half = n // 2
        out.fill_(-7)
        ctx.plan_noalloc(0, st["step"], out[:half])
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        lo = present.copy()
        lo[half:] = False
        assert np.array_equal(got[lo], want[lo])
        assert (got[half:] == -7).all() and (got[:half][~present[:half]] == -7).all()
        ctx.step(1)
    # the planned steps did send draws to the FP64 re-check (its scratch path)
    assert rechecked_calls > 0
    ctx.close()


def test_plan_noalloc_rejects_more_slots_than_its_scratch(fg):
    """The fixed scratch holds 2^20 agent slots: a replicate with one more is
    refused with FAST_EINVAL (nothing is queued)."""
    import torch

    t = wl.room(1100, 1100)
    wl.add_exit(t, "bottom", 500, 4)
    free = np.flatnonzero(t.ravel() == wl.FREE)
    n = (1 << 20) + 1
    cells = np.random.default_rng(0).choice(free, n, replace=False).astype(np.int32)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, t, 1.2, 1, 0)
    ctx.place(0, cells)
    ctx.plan_only(1)
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FastError) as e:
        ctx.plan_noalloc(0, 0, out)
    assert e.value.code == -1
    torch.cuda.synchronize()
    assert int((out != -7).sum()) == 0
    ctx.close()


def test_plan_noalloc_refuses_speeds_per_agent(fg):
    """A replicate whose agents have speeds of their own is refused with
    FAST_EINVAL before anything is queued; the output stays untouched."""
    import torch

    w = wl.config_small_room(W=40, H=30, n=200, seed=3, v_m=3)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.set_speeds(0, np.full(len(w.cells), 2, np.uint8))
    ctx.place(0, w.cells)
    ctx.plan_only(1)
    out = torch.full((len(w.cells),), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FastError) as e:
        ctx.plan_noalloc(0, 0, out)
    assert e.value.code == -1
    torch.cuda.synchronize()
    assert int((out != -7).sum()) == 0
    ctx.close()
