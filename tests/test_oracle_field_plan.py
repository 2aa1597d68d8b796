"""Pins of the oracle's floor field and planning rule.

Floor field: closed-form octile distances on empty rooms, the minimum over
several exits, exhaustive relaxation with exact comparisons on small walled
grids.  Planning: brute-force enumeration of the admissible candidates and
their probabilities (independent Python restatement, libm exp), a chi-square
test of the draws, and the special cases k_S = 0 (uniform) and large k_S
(argmin of the floor field).
"""
import math

import numpy as np
import pytest

from paper_0911_2900_gb300 import workloads as wl
from tests import refs

SQ2 = math.sqrt(2.0)


def test_floor_field_closed_form_single_exit(orc):
    t = wl.room(23, 17)
    ex = (0, 9)               # exit cell on the left wall
    t[ex[1], ex[0]] = wl.EXIT
    a, b, S = orc.floor_field(t)
    for y in range(1, 16):
        for x in range(1, 22):
            oa, ob = refs.octile(x - ex[0], y - ex[1])
            assert (a[y, x], b[y, x]) == (oa, ob)
            assert S[y, x] == float(oa) + float(ob) * SQ2
    # walls are unreachable
    assert a[0, 0] == -1 and math.isinf(S[0, 0])


def test_floor_field_min_over_exits(orc):
    t = wl.room(30, 20)
    exits = [(0, 5), (29, 14), (12, 19)]
    for x, y in exits:
        t[y, x] = wl.EXIT
    a, b, _ = orc.floor_field(t)
    for y in range(1, 19):
        for x in range(1, 29):
            best = None
            for ex, ey in exits:
                d = refs.octile(x - ex, y - ey)
                if best is None or refs.less_ab(d, best):
                    best = d
            assert (a[y, x], b[y, x]) == best


@pytest.mark.parametrize("seed", range(6))
def test_floor_field_vs_relaxation_on_walled_grids(orc, seed):
    rng = np.random.default_rng(seed)
    W, H = int(rng.integers(6, 14)), int(rng.integers(6, 12))
    t = wl.room(W, H)
    t[1:-1, 1:-1][rng.random((H - 2, W - 2)) < 0.25] = wl.WALL
    t[0, int(rng.integers(1, W - 1))] = wl.EXIT
    t[H - 1, int(rng.integers(1, W - 1))] = wl.EXIT
    a, b, S = orc.floor_field(t)
    ref = refs.bellman_ford_field(t.tolist())
    for y in range(H):
        for x in range(W):
            if ref[y][x] is None:
                assert a[y, x] == -1 and math.isinf(S[y, x])
            else:
                assert (a[y, x], b[y, x]) == ref[y][x]


def _brute_probs(t, S, occ2d, x0, y0, v, kS, metric="l2"):
    cands = refs.candidates(t.tolist(), occ2d, x0, y0, v, metric)
    K = len(refs.reach_offsets(v, metric))
    w = np.zeros(K)
    for k, dx, dy in cands:
        w[k] = math.exp(-kS * (S[y0 + dy, x0 + dx] - S[y0, x0]))
    return w


def _scene(seed, W=14, H=12, n=25, v=3):
    rng = np.random.default_rng(seed)
    t = wl.room(W, H)
    t[1:-1, 1:-1][rng.random((H - 2, W - 2)) < 0.12] = wl.WALL
    wl.add_exit(t, "bottom", W // 2 - 1, 2)
    wl.add_exit(t, "left", H // 2, 2)
    wl.seal_unreachable(t)
    cells = wl.place_uniform(t, n, seed)
    return t, cells


@pytest.mark.parametrize("v,metric", [(1, "l2"), (2, "l2"), (3, "l2"), (4, "l2"), (5, "l2"),
                                      (3, "l2p"), (2, "linf")])
def test_planning_weights_match_brute_force(orc, v, metric):
    reach = {"l2": orc.REACH_L2, "l2p": orc.REACH_L2P, "linf": orc.REACH_LINF}[metric]
    for seed in range(3):
        t, cells = _scene(seed, v=v)
        sim = orc.Sim(t, v=v, kS=1.2, seed=seed + 5, reach=reach)
        sim.place(cells)
        H, W = t.shape
        occ2d = sim.occ.reshape(H, W).tolist()
        for i in range(len(cells)):
            c = int(cells[i])
            d, w, u = sim.plan_agent(i, t=3)
            want = _brute_probs(t, sim.S, occ2d, c % W, c // W, v, 1.2, metric)
            # the admissible set is exact (integers), the weights agree to rounding
            assert np.array_equal(w > 0, want > 0)
            np.testing.assert_allclose(w, want, rtol=1e-13, atol=0)
            # u is the 53-bit uniform of the planning stream
            assert u == refs.uniform53(seed + 5, i, 3)
            # the choice is the inverse-CDF draw of the brute-force probabilities
            cum = np.cumsum(want) / want.sum()
            k = int(np.searchsorted(cum, u, side="right"))
            off = refs.reach_offsets(v, metric)[k]
            if abs(cum[k] - u) > 1e-12 and (k == 0 or abs(cum[k - 1] - u) > 1e-12):
                assert d == c + off[1] * W + off[0]


@pytest.mark.parametrize("v", [1, 2, 3, 4, 5])
def test_planning_chi_square(orc, v):
    """The draws of one agent over many steps follow the brute-force
    probabilities (the planning stream is keyed by the step index)."""
    from scipy import stats

    t, cells = _scene(100 + v, W=16, H=16, n=30, v=v)
    sim = orc.Sim(t, v=v, kS=1.2, seed=77)
    sim.place(cells)
    H, W = t.shape
    occ2d = sim.occ.reshape(H, W).tolist()
    i = 4
    c = int(cells[i])
    w = _brute_probs(t, sim.S, occ2d, c % W, c // W, v, 1.2)
    p = w / w.sum()
    offs = refs.reach_offsets(v)
    idx = {c + dy * W + dx: k for k, (dx, dy) in enumerate(offs)}
    n_draw = 200_000
    counts = np.zeros(len(offs))
    for tt in range(n_draw):
        d, _, _ = sim.plan_agent(i, tt)
        counts[idx[d]] += 1
    nz = p > 0
    assert counts[~nz].sum() == 0
    chi2 = (((counts[nz] - n_draw * p[nz]) ** 2) / (n_draw * p[nz])).sum()
    pval = stats.chi2.sf(chi2, nz.sum() - 1)
    assert pval > 1e-3, (chi2, pval)


def test_planning_kS_zero_is_uniform(orc):
    """k_S = 0: every admissible candidate has weight exactly 1, so the choice
    is candidate floor(u * K_free) unless u * K_free rounds onto an integer."""
    t, cells = _scene(9, v=3)
    sim = orc.Sim(t, v=3, kS=0.0, seed=123)
    sim.place(cells)
    H, W = t.shape
    occ2d = sim.occ.reshape(H, W).tolist()
    for i in range(len(cells)):
        c = int(cells[i])
        cands = refs.candidates(t.tolist(), occ2d, c % W, c // W, 3)
        for tt in range(20):
            d, w, u = sim.plan_agent(i, tt)
            assert set(np.flatnonzero(w)) == {k for k, _, _ in cands}
            assert all(x == 1.0 for x in w[w > 0])
            j = int(math.floor(u * len(cands)))
            if u * len(cands) != j:
                _, dx, dy = cands[j]
                assert d == c + dy * W + dx


def test_planning_large_kS_picks_argmin(orc):
    """k_S large: the weight of the candidate nearest to the exit dominates
    (ratio exp(-k_S * gap) per other candidate), so the draw lands on it."""
    t = wl.room(20, 20)
    wl.add_exit(t, "bottom", 9, 2)
    rng = np.random.default_rng(5)
    cells = wl.place_uniform(t, 15, 5)
    sim = orc.Sim(t, v=3, kS=60.0, seed=9)
    sim.place(cells)
    H, W = t.shape
    occ2d = sim.occ.reshape(H, W).tolist()
    for i in range(len(cells)):
        c = int(cells[i])
        cands = refs.candidates(t.tolist(), occ2d, c % W, c // W, 3)
        Ss = sorted((sim.S[c // W + dy, c % W + dx], (dx, dy)) for _, dx, dy in cands)
        best, second = Ss[0], Ss[1]
        if second[0] - best[0] < 0.3:
            continue   # near tie: no dominance claim
        for tt in range(10):
            d, _, _ = sim.plan_agent(i, tt)
            assert d == c + best[1][1] * W + best[1][0]


def test_single_agent_open_field_closed_form(orc):
    """One agent far from walls: every reach offset is a candidate and its
    weight is exp(-k_S * (octile(target) - octile(start))) in closed form."""
    t = wl.room(41, 41)
    t[40, 20] = wl.EXIT
    sim = orc.Sim(t, v=4, kS=1.2, seed=1)
    c = 15 * 41 + 20
    sim.place([c])
    d, w, u = sim.plan_agent(0, 0)
    a0, b0 = refs.octile(0, 40 - 15)
    for k, (dx, dy) in enumerate(refs.reach_offsets(4)):
        a1, b1 = refs.octile(dx, 40 - (15 + dy))
        want = math.exp(-1.2 * ((a1 + b1 * SQ2) - (a0 + b0 * SQ2)))
        assert w[k] == pytest.approx(want, rel=1e-13)
