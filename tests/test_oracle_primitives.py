"""Pins of the oracle's primitives: Philox4x32-10, exp64, reach sets, paths.

Each check compares the oracle with something other than itself: published
known-answer vectors, an independent build of PyTorch's Philox engine,
correctly rounded exponentials from Python's decimal module, lattice-point
counts, and exact rational path rasterisation.
"""
import math
import os
import shutil
import subprocess
from decimal import Decimal, getcontext

import numpy as np
import pytest

from tests import refs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[:4], v[4:6], v[6:]))
    return rows


def test_philox_known_answers(orc):
    for ctr, key, want in _kat():
        assert orc.philox(ctr, key).tolist() == want
        assert refs.philox4x32_10(ctr, key) == want


def test_philox_matches_python_reference_random(orc):
    rng = np.random.default_rng(7)
    for _ in range(300):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).tolist()
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).tolist()
        assert orc.philox(ctr, key).tolist() == refs.philox4x32_10(ctr, key)


def _torch_header_dir():
    try:
        import torch.utils.cpp_extension as ce
    except Exception:
        return None
    for p in ce.include_paths():
        if os.path.exists(os.path.join(p, "ATen", "core", "PhiloxRNGEngine.h")):
            return p
    return None


def test_philox_matches_pytorch_engine(orc, tmp_path):
    """Builds a tiny program against PyTorch's installed Philox engine header
    (library code, run, not copied) and compares 1000 blocks."""
    inc = _torch_header_dir()
    gxx = shutil.which("g++")
    if inc is None or gxx is None:
        pytest.skip("PyTorch headers or g++ not available")
    src = tmp_path / "ph.cpp"
    src.write_text(
        "#include <ATen/core/PhiloxRNGEngine.h>\n#include <cstdio>\n#include <cstdint>\n"
        "int main(){ unsigned long long seed, sub, off;\n"
        " while (scanf(\"%llu %llu %llu\", &seed, &sub, &off) == 3) {\n"
        "  at::philox_engine e(seed, sub, off);\n"
        "  unsigned a=e(), b=e(), c=e(), d=e(); printf(\"%u %u %u %u\\n\", a, b, c, d); }\n"
        " return 0; }\n")
    exe = tmp_path / "ph"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("could not build against PyTorch's Philox header: " + r.stderr[-300:])
    rng = np.random.default_rng(11)
    cases = [(int(rng.integers(0, 2 ** 63)), int(rng.integers(0, 2 ** 63)),
              int(rng.integers(0, 2 ** 63))) for _ in range(1000)]
    inp = "".join(f"{s} {u} {o}\n" for s, u, o in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    got = [list(map(int, l.split())) for l in out.strip().splitlines()]
    for (seed, sub, off), want in zip(cases, got):
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert orc.philox(ctr, key).tolist() == want


def _exp_correctly_rounded(x: float) -> float:
    getcontext().prec = 60
    return float(Decimal(x).exp())


def _ulp_diff(a: float, b: float) -> int:
    ia = np.array([a], np.float64).view(np.int64)[0]
    ib = np.array([b], np.float64).view(np.int64)[0]
    return abs(int(ia) - int(ib))


def test_exp64_within_one_ulp_of_correctly_rounded(orc):
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-13.0, 13.0, 4000), rng.uniform(-0.5, 0.5, 1000),
                         rng.uniform(-700, 700, 500),
                         np.array([0.0, -0.0, 1.0, -1.0, math.log(2), -math.log(2), 12.0,
                                   -12.0, 0.5 * math.log(2), -0.5 * math.log(2)])])
    worst = 0
    for x in xs:
        worst = max(worst, _ulp_diff(orc.exp64(float(x)), _exp_correctly_rounded(float(x))))
    assert worst <= 1, worst


def test_exp64_special_values(orc):
    assert orc.exp64(0.0) == 1.0
    assert orc.exp64(-0.0) == 1.0
    for n in range(-20, 21):
        # exp(n ln2) = 2^n up to the rounding of n*ln2 (one ulp of the argument)
        y = orc.exp64(n * math.log(2))
        assert abs(y / 2.0 ** n - 1.0) < 1e-14
    # monotone on a fine grid of the weights' argument range
    xs = np.linspace(-12.0, 12.0, 20001)
    ys = [orc.exp64(float(x)) for x in xs]
    assert all(b > a for a, b in zip(ys, ys[1:]))


def test_reach_counts_match_lattice_point_counts(orc):
    table = {}
    with open(os.path.join(GOLD, "reach_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            table[name] = list(map(int, vals))
    for reach, name, metric in ((orc.REACH_L2, "L2", "l2"), (orc.REACH_L2P, "L2P", "l2p"),
                                (orc.REACH_LINF, "LINF", "linf")):
        for v in range(1, 6):
            dx, dy = orc.offsets(v, reach)
            assert len(dx) == table[name][v - 1]
            assert list(zip(dx.tolist(), dy.tolist())) == refs.reach_offsets(v, metric)


def test_paths_match_exact_rational_rounding(orc):
    for dy in range(-5, 6):
        for dx in range(-5, 6):
            if dx == 0 and dy == 0:
                assert orc.path(0, 0) == []
                continue
            p = orc.path(dx, dy)
            assert p == refs.straight_path(dx, dy)
            # every step is a Moore move and the path ends on the target
            prev = (0, 0)
            for q in p:
                assert max(abs(q[0] - prev[0]), abs(q[1] - prev[1])) == 1
                prev = q
            assert p[-1] == (dx, dy)
            # point symmetry of rounding half away from zero
            assert orc.path(-dx, -dy) == [(-a, -b) for a, b in p]


def test_paths_hand_drawn(orc):
    # hand-drawn rasterisations (L = max(|dx|,|dy|), round half away from 0)
    assert orc.path(4, 1) == [(1, 0), (2, 1), (3, 1), (4, 1)]
    assert orc.path(2, 1) == [(1, 1), (2, 1)]
    assert orc.path(0, -3) == [(0, -1), (0, -2), (0, -3)]
    assert orc.path(-3, 2) == [(-1, 1), (-2, 1), (-3, 2)]
    assert orc.path(3, 3) == [(1, 1), (2, 2), (3, 3)]
