"""The allocation-free planning pass (fast_plan_noalloc) against the regular one.

fast_plan_noalloc serves callers that cannot allocate device memory when
they plan (for instance while they capture a CUDA graph on their stream); its
only scratch is a fixed array inside the library.  It must give exactly the
desired cells of a regular planning pass (fast_plan_only + fast_readback),
call after call, although every call reuses the same array.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_0911_2900_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_plan_noalloc_matches_regular_planning_two_calls():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_0911_2900_gb300 as fg

    w = wl.config_corridors(v_m=4)
    n = len(w.cells)
    ctx = fg.Context(1, "fp32_recheck")
    ctx.init_grid(0, w.cell_type, w.k_S, w.v_m, w.seed)
    ctx.place(0, w.cells)
    ctx.step(2)
    for call in range(2):
        ctx.plan_only(1)
        cells, want, st = ctx.readback(0, n)
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        ctx.plan_noalloc(0, st["step"], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        present = cells >= 0
        assert present.sum() > 0
        assert np.array_equal(got[present], want[present]), f"call {call}"
        assert (got[~present] == -7).all()
        ctx.step(1)
    ctx.close()
