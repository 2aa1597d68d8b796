"""FP64 CPU oracle of the F.A.S.T. time step (planning + sequential movement).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It is
independent of the CUDA library: it shares no source, header, helper or table
with ``paper_0911_2900_gb300`` and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, no fast-math, no FMA
contraction); this module only builds it with gcc and marshals numpy arrays.
Paper: T. Kretz, "Computation Speed of the F.A.S.T. Model" -- Sec. 1 (parallel
planning from read-only common data, sequential movement), Sec. 2 (k_S = 1.2,
k_other = 0, one v_m for all agents, the OpenMP planning loop).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FREE, WALL, EXIT = 0, 1, 2
REACH_L2, REACH_L2P, REACH_LINF = 0, 1, 2
MAXK = 121


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class World(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("v", C.c_int32), ("reach", C.c_int32),
                ("kS", C.c_double), ("seed", C.c_uint64),
                ("type", C.c_void_p), ("S", C.c_void_p), ("speed", C.c_void_p)]


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i32, i64, u64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            sig = {
                "orc_philox4x32_10": (None, [vp, vp, vp]),
                "orc_exp64": (d, [d]),
                "orc_offsets": (i32, [i32, i32, vp, vp]),
                "orc_path": (i32, [i32, i32, vp, vp]),
                "orc_floor_field": (i64, [i32, i32, vp, vp, vp, vp]),
                "orc_build_occ": (i32, [vp, i32, vp, vp]),
                "orc_plan_agent": (i32, [vp, vp, i32, i32, i32, vp, vp]),
                "orc_plan_all": (None, [vp, vp, i32, vp, vp, i32, vp, i32]),
                "orc_move_priority": (C.c_uint32, [u64, i32, i32]),
                "orc_move": (i32, [vp, vp, i32, vp, vp, vp, i32]),
                "orc_digest": (u64, [i32, vp, vp]),
                "orc_run": (i32, [vp, vp, i32, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# --------------------------------------------------------------------------- primitives
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def exp64(x: float) -> float:
    return lib().orc_exp64(float(x))


def offsets(v: int, reach: int = REACH_L2):
    dx = np.zeros(MAXK, np.int32)
    dy = np.zeros(MAXK, np.int32)
    K = lib().orc_offsets(v, reach, _p(dx), _p(dy))
    return dx[:K].copy(), dy[:K].copy()


def path(dx: int, dy: int):
    px = np.zeros(8, np.int32)
    py = np.zeros(8, np.int32)
    L = lib().orc_path(dx, dy, _p(px), _p(py))
    return list(zip(px[:L].tolist(), py[:L].tolist()))


def floor_field(cell_type: np.ndarray):
    """Exact Dijkstra floor field: returns (a, b, S) arrays shaped like cell_type."""
    t = np.ascontiguousarray(cell_type, dtype=np.uint8)
    H, W = t.shape
    a = np.empty((H, W), np.int32)
    b = np.empty((H, W), np.int32)
    S = np.empty((H, W), np.float64)
    r = lib().orc_floor_field(W, H, _p(t), _p(a), _p(b), _p(S))
    if r < 0:
        raise MemoryError("oracle floor field: allocation failed")
    return a, b, S


def move_priority(seed: int, agent_id: int, t: int) -> int:
    return int(lib().orc_move_priority(seed, agent_id, t))


def digest(ids: np.ndarray, vals: np.ndarray) -> int:
    i = np.ascontiguousarray(ids, np.int32)
    v = np.ascontiguousarray(vals, np.int32)
    return int(lib().orc_digest(len(i), _p(i), _p(v)))


# --------------------------------------------------------------------------- simulation
class Sim:
    """One replicate: grid, floor field, agents (id, cell) and occupancy."""

    def __init__(self, cell_type, v, kS=1.2, seed=0, reach=REACH_L2, S=None, speeds=None):
        """speeds: optional maximum speed of each agent id (1..5); v is then
        only a default that no agent uses."""
        self.type = np.ascontiguousarray(cell_type, dtype=np.uint8)
        self.H, self.W = self.type.shape
        if S is None:
            _, _, S = floor_field(self.type)
        self.S = np.ascontiguousarray(S, dtype=np.float64)
        self.speeds = None
        if speeds is not None:
            self.speeds = np.ascontiguousarray(speeds, dtype=np.uint8).copy()
            if self.speeds.size and (self.speeds.min() < 1 or self.speeds.max() > 5):
                raise ValueError("speeds must be in 1..5")
        self.world = World(self.W, self.H, v, reach, float(kS), int(seed),
                           self.type.ctypes.data, self.S.ctypes.data,
                           self.speeds.ctypes.data if self.speeds is not None else None)
        self.occ = np.empty(self.W * self.H, np.int32)
        self.id = np.zeros(0, np.int32)
        self.cell = np.zeros(0, np.int32)

    def place(self, cells, ids=None):
        self.cell = np.ascontiguousarray(cells, dtype=np.int32).copy()
        n = len(self.cell)
        self.id = (np.arange(n, dtype=np.int32) if ids is None
                   else np.ascontiguousarray(ids, dtype=np.int32).copy())
        if self.speeds is not None and n and int(self.id.max()) >= len(self.speeds):
            raise ValueError("speeds does not cover every agent id")
        if lib().orc_build_occ(C.byref(self.world), n, _p(self.cell), _p(self.occ)) != 0:
            raise ValueError("invalid placement (wall/exit/duplicate/outside)")

    def plan_agent(self, i: int, t: int):
        """Returns (desired cell, weights[K], u) of agent index i at step t."""
        v = self.world.v if self.speeds is None else int(self.speeds[self.id[i]])
        K = len(offsets(v, self.world.reach)[0])
        w = np.zeros(MAXK, np.float64)
        u = C.c_double(0.0)
        d = lib().orc_plan_agent(C.byref(self.world), _p(self.occ), int(self.cell[i]),
                                 int(self.id[i]), int(t), _p(w), C.byref(u))
        return d, w[:K].copy(), u.value

    def plan(self, t: int, threads: int = 1) -> np.ndarray:
        out = np.empty(len(self.id), np.int32)
        lib().orc_plan_all(C.byref(self.world), _p(self.occ), len(self.id), _p(self.id),
                           _p(self.cell), int(t), _p(out), int(threads))
        return out

    def move(self, desired: np.ndarray, t: int) -> int:
        d = np.ascontiguousarray(desired, np.int32)
        return int(lib().orc_move(C.byref(self.world), _p(self.occ), len(self.id), _p(self.id),
                                  _p(self.cell), _p(d), int(t)))

    def run(self, t0: int, n_steps: int, threads: int = 1, digests: bool = True):
        n = len(self.id)
        des = np.empty(n, np.int32)
        dc = np.zeros(n_steps, np.uint64) if digests else None
        dd = np.zeros(n_steps, np.uint64) if digests else None
        al = np.zeros(n_steps, np.int32)
        ps, ms = C.c_double(0.0), C.c_double(0.0)
        left = lib().orc_run(C.byref(self.world), _p(self.occ), n, _p(self.id), _p(self.cell),
                             int(t0), int(n_steps), int(threads), _p(des), _p(dc), _p(dd),
                             _p(al), C.byref(ps), C.byref(ms))
        return dict(left=int(left), desired=des, dig_cell=dc, dig_des=dd, alive=al,
                    plan_s=ps.value, move_s=ms.value)

    def cells_by_id(self) -> np.ndarray:
        out = np.full(int(self.id.max()) + 1 if len(self.id) else 0, -1, np.int32)
        out[self.id] = self.cell
        return out
