"""Independent pure-Python references used only to pin the C oracle.

Each function restates a definition directly (exact rationals, integer
arithmetic, Python's own libm exp) without the oracle's code paths, so that a
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand) shows up as a disagreement.
"""
from __future__ import annotations

import math
from fractions import Fraction

M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32-10 from Salmon et al. (SC'11): S-box of two 32x32->64
    multiplications, Feistel-like permutation, Weyl key schedule."""
    c = [int(x) & M32 for x in ctr]
    k = [int(x) & M32 for x in key]
    for rnd in range(10):
        if rnd:
            k = [(k[0] + 0x9E3779B9) & M32, (k[1] + 0xBB67AE85) & M32]
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & M32, p1 & M32,
             ((p0 >> 32) ^ c[3] ^ k[1]) & M32, p0 & M32]
    return c


def uniform53(seed, agent_id, t):
    r = philox4x32_10([agent_id, t, 0, 0], [seed & M32, seed >> 32])
    return ((r[0] >> 5) * 2 ** 26 + (r[1] >> 6)) / 2.0 ** 53


def fmix32(h):
    """MurmurHash3 32-bit finalizer (A. Appleby)."""
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    h ^= h >> 16
    return h


def move_priority(seed, agent_id, t):
    """Four-round Feistel network on the 12-bit halves of the 24-bit id, round
    function fmix32(R ^ k_i) & 0xFFF, keys = Philox(seed; (0, t, 2, 0))."""
    k = philox4x32_10([0, t, 2, 0], [seed & M32, seed >> 32])
    L, R = (agent_id >> 12) & 0xFFF, agent_id & 0xFFF
    for i in range(4):
        L, R = R, L ^ (fmix32(R ^ k[i]) & 0xFFF)
    return (L << 12) | R


def reach_offsets(v, metric="l2"):
    out = []
    for dy in range(-v, v + 1):
        for dx in range(-v, v + 1):
            if metric == "l2":
                ok = dx * dx + dy * dy <= v * v
            elif metric == "l2p":
                ok = dx * dx + dy * dy <= v * v + v
            else:
                ok = max(abs(dx), abs(dy)) <= v
            if ok:
                out.append((dx, dy))
    return out


def round_half_away(q: Fraction) -> int:
    """Nearest integer, ties away from zero, from an exact rational."""
    if q >= 0:
        return math.floor(q + Fraction(1, 2))
    return -math.floor(-q + Fraction(1, 2))


def straight_path(dx, dy):
    L = max(abs(dx), abs(dy))
    return [(round_half_away(Fraction(s * dx, L)), round_half_away(Fraction(s * dy, L)))
            for s in range(1, L + 1)]


def octile(dx, dy):
    """Exact 8-neighbour distance in an empty plane, as (a, b): a + b*sqrt2."""
    ax, ay = abs(dx), abs(dy)
    return max(ax, ay) - min(ax, ay), min(ax, ay)


def less_ab(p, q):
    """(a1 + b1 sqrt2) < (a2 + b2 sqrt2), exactly."""
    da, db = p[0] - q[0], p[1] - q[1]
    # sign of da + db*sqrt2
    if da >= 0 and db >= 0:
        return False
    if da <= 0 and db <= 0:
        return (da, db) != (0, 0)
    if da > 0:        # db < 0: negative iff 2 db^2 > da^2
        return 2 * db * db > da * da
    return da * da > 2 * db * db   # da < 0 < db


def bellman_ford_field(t):
    """Exact floor field by repeated relaxation until nothing changes.
    t: 2-D list/array of cell types (0 free, 1 wall, 2 exit)."""
    H, W = len(t), len(t[0])
    INF = None
    d = [[INF] * W for _ in range(H)]
    for y in range(H):
        for x in range(W):
            if t[y][x] == 2:
                d[y][x] = (0, 0)
    changed = True
    while changed:
        changed = False
        for y in range(H):
            for x in range(W):
                if t[y][x] == 1:
                    continue
                for ny in range(y - 1, y + 2):
                    for nx in range(x - 1, x + 2):
                        if (nx, ny) == (x, y) or not (0 <= nx < W and 0 <= ny < H):
                            continue
                        if d[ny][nx] is None:
                            continue
                        step = (0, 1) if (nx != x and ny != y) else (1, 0)
                        cand = (d[ny][nx][0] + step[0], d[ny][nx][1] + step[1])
                        if d[y][x] is None or less_ab(cand, d[y][x]):
                            d[y][x] = cand
                            changed = True
    return d


def candidates(t, occ, x0, y0, v, metric="l2"):
    """Admissible candidates of an agent at (x0, y0): list of (k, dx, dy)."""
    H, W = len(t), len(t[0])
    out = []
    for k, (dx, dy) in enumerate(reach_offsets(v, metric)):
        x, y = x0 + dx, y0 + dy
        if not (0 <= x < W and 0 <= y < H):
            continue
        if (dx, dy) != (0, 0):
            if occ[y][x] != -1:
                continue
            if any(t[y0 + py][x0 + px] == 1 for px, py in straight_path(dx, dy)):
                continue
        out.append((k, dx, dy))
    return out
