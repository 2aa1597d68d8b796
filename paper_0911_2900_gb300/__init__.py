"""Python binding of libfastgb, the GB300 implementation of the F.A.S.T. time step.

Argument marshalling only: every step of the planning and movement phases runs
in the CUDA kernels of ``csrc/`` behind the C ABI of ``include/fastgb.h``.  There
is no CPU fallback: if the shared library cannot be loaded (not built, or no
CUDA device), the calls raise.

PyTorch is used only as the device allocator and to supply the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Context", "FastError", "load", "PRECISION", "REACH", "OPT"]

PRECISION = {"fp64": 0, "fp32_recheck": 1, "fp32_norecheck": 2}
REACH = {"l2": 0, "l2p": 1, "linf": 2}
OPT = {"resort_period": 1, "digests": 2, "lanes_v1": 3, "lanes_v2": 4, "lanes_v3": 5,
       "lanes_v4": 6, "lanes_v5": 7, "barrier_ns": 10, "use_graph": 11, "move_blocks": 12,
       "tile_shift": 13, "graph_steps": 14, "claim_reserve": 15, "claim_tag": 16}
ERRORS = {0: "FAST_OK", -1: "FAST_EINVAL", -2: "FAST_ESTATE", -3: "FAST_ENOMEM",
          -4: "FAST_ECUDA", -5: "FAST_ETIMEOUT"}


class FastError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("cell_type", C.c_void_p),
                ("k_S", C.c_double), ("v_m", C.c_int32), ("seed", C.c_uint64),
                ("static_field", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("steps_run", C.c_int64), ("alive", C.c_int32),
                ("exited", C.c_int32), ("agent_steps", C.c_int64), ("rechecked", C.c_int64),
                ("move_rounds", C.c_int64), ("max_rounds", C.c_int32), ("last_rounds", C.c_int32),
                ("kernel_launches", C.c_int64), ("tile_fallbacks", C.c_int64),
                ("movers", C.c_int64), ("footprint_cells", C.c_int64),
                ("diag_flips", C.c_int64), ("diag_max_abs_dp", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PrecisionReport(C.Structure):
    _fields_ = [("agents", C.c_int64), ("flagged", C.c_int64), ("flips", C.c_int64),
                ("flips_unflagged", C.c_int64), ("max_abs_dp", C.c_double), ("margin", C.c_double),
                ("flips_after_recheck", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneReport(C.Structure):
    _fields_ = [("tile_shift", C.c_int32), ("lanes", C.c_int32 * 5), ("shift_us", C.c_float * 4),
                ("lanes_us", (C.c_float * 5) * 5)]

    def as_dict(self):
        return {"tile_shift": self.tile_shift, "lanes": list(self.lanes),
                "shift_us": {3 + i: float(self.shift_us[i]) for i in range(4)},
                "lanes_us": {v + 1: {l: float(self.lanes_us[v][j])
                                     for j, l in enumerate((0, 1, 2, 4, 8))
                                     if self.lanes_us[v][j] > 0}
                             for v in range(5) if self.lanes[v] >= 0}}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()

EXPORTS = {
    "fast_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "fast_init_grid": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "fast_place_agents": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_int32]),
    "fast_set_speeds": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "fast_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "fast_plan_only": (C.c_int, [C.c_void_p, C.c_int32]),
    "fast_readback": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "fast_get_digests": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "fast_phase_times": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fast_precision_report_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fast_move_profile": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "fast_reach_union": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "fast_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "fast_selftest_l2_read": (C.c_int, [C.c_int64, C.c_int32, C.c_void_p]),
    "fast_build_checked": (C.c_int, []),
    "fast_selftest_bounds": (C.c_int, [C.c_int64, C.c_int64, C.c_void_p]),
    "fast_floor_field": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "fast_plan_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "fast_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "fast_place_all": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fast_readback_all": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "fast_last_error": (C.c_char_p, [C.c_void_p]),
    "fast_destroy": (None, [C.c_void_p]),
    "fast_selftest_exp64": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "fast_selftest_philox": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "fast_selftest_ex2": (C.c_int, [C.c_float, C.c_float, C.c_void_p]),
    "fast_selftest_barrier_timeout": (C.c_int, [C.c_int64]),
    "fast_selftest_barrier_cost": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "fast_selftest_barrier_sum": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Loads libfastgb.so (building it first if it is missing or stale); with
    the environment variable FASTGB_CHECKED=1 the debug build, whose kernels
    check the indices they derive from data (an index out of range becomes a
    device error instead of a memory access)."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("FASTGB_CHECKED", "0") == "1"
            path = _build.LIB_CHECKED if checked else _build.LIB
            if build_if_missing:
                _build.build(checked=checked)
            if not os.path.exists(path):
                raise FastError(-4, f"{os.path.basename(path)} not built ({path})")
            lib = C.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, kept alive by pointer;
    with `limit` (bytes), a request that would take the context's live total
    above it is refused, as an out-of-memory one is (the library then reports
    FAST_ENOMEM)."""

    def __init__(self, device, limit=None):
        import torch

        self.torch = torch
        self.device = device
        self.limit = limit
        self.live = {}
        self.total = 0
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, _user):
        if self.limit is not None and self.total + int(nbytes) > self.limit:
            return None
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory: the library reports FAST_ENOMEM
            return None
        p = t.data_ptr()
        self.live[p] = t
        self.total += t.numel()
        return p

    def _free(self, ptr, _user):
        t = self.live.pop(ptr, None)
        if t is not None:
            self.total -= t.numel()


class Context:
    """One fast_ctx: n replicates stepped together on one CUDA stream."""

    def __init__(self, n_replicates: int = 1, precision: str = "fp32_recheck",
                 reach: str = "l2", stream=None, device=None, torch_memory: bool = True,
                 memory_limit: int | None = None):
        import torch

        if not torch.cuda.is_available():
            raise FastError(-4, "no CUDA device: libfastgb runs on the GPU only")
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        if memory_limit is not None and not torch_memory:
            raise ValueError("memory_limit needs torch_memory=True (the limit is the allocator's)")
        self._alloc = _TorchAllocator(self.device, memory_limit) if torch_memory else None
        h = C.c_void_p()
        rc = self.lib.fast_create(
            C.byref(h), n_replicates, PRECISION[precision], REACH[reach],
            C.c_void_p(self.stream.cuda_stream),
            C.cast(self._alloc.alloc_cb, C.c_void_p) if self._alloc else None,
            C.cast(self._alloc.free_cb, C.c_void_p) if self._alloc else None, None)
        if rc != 0:
            raise FastError(rc, "fast_create failed")
        self.h = h
        self.n_rep = n_replicates
        self.precision = precision
        self.reach = reach
        self.id_bound = [0] * n_replicates

    # -- helpers ---------------------------------------------------------------
    def _check(self, rc, what):
        if rc < 0:
            msg = self.lib.fast_last_error(self.h)
            raise FastError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.fast_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API ---------------------------------------------------------------------
    def init_grid(self, rep: int, cell_type: np.ndarray, k_S: float = 1.2, v_m: int = 4,
                  seed: int = 0, static_field=None):
        """static_field: optional float64 array shaped like cell_type, the
        caller's floor field (see fast_grid_desc); None: the library computes
        the 8-neighbour distance to the exits."""
        t = np.ascontiguousarray(cell_type, dtype=np.uint8)
        H, W = t.shape
        S = None
        if static_field is not None:
            S = np.ascontiguousarray(static_field, dtype=np.float64)
            if S.shape != t.shape:
                raise ValueError("static_field must have the shape of cell_type")
        g = GridDesc(W, H, t.ctypes.data, float(k_S), int(v_m), int(seed),
                     S.ctypes.data if S is not None else None)
        self._check(self.lib.fast_init_grid(self.h, rep, C.byref(g)), "fast_init_grid")

    def set_speeds(self, rep: int, speed_by_id) -> None:
        """Maximum speed (1..5) of every agent id of replicate rep; call after
        init_grid and before the first place.  An empty array returns to the
        grid's v_m for every agent."""
        sp = np.ascontiguousarray(speed_by_id, dtype=np.uint8)
        self._check(self.lib.fast_set_speeds(self.h, rep, len(sp), _ptr(sp)), "fast_set_speeds")

    def place(self, rep: int, cells, ids=None, start_step: int = 0):
        c = np.ascontiguousarray(cells, dtype=np.int32)
        i = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        self._check(self.lib.fast_place_agents(self.h, rep, len(c), _ptr(c), _ptr(i),
                                               int(start_step)), "fast_place_agents")
        self.id_bound[rep] = (int(i.max()) + 1 if len(c) else 0) if i is not None else len(c)

    def place_uniform(self, rep: int, n: int, start_step: int = 0):
        """Ids 0..n-1 on n distinct free, reachable cells drawn uniformly,
        from the grid's seed (fast_place_agents with no cells)."""
        self._check(self.lib.fast_place_agents(self.h, rep, int(n), None, None, int(start_step)),
                    "fast_place_agents")
        self.id_bound[rep] = int(n)

    def place_all(self, counts, cells_by_id, start_step: int = 0):
        """Every replicate at once: counts[r] ids of replicate r (-1: leave it),
        cells_by_id the concatenation of the replicates' cells-by-id arrays."""
        n = np.ascontiguousarray(counts, dtype=np.int32)
        c = np.ascontiguousarray(cells_by_id, dtype=np.int32)
        self._check(self.lib.fast_place_all(self.h, _ptr(n), _ptr(c), int(start_step)),
                    "fast_place_all")
        for r, k in enumerate(n):
            if k >= 0:
                self.id_bound[r] = int(k)

    def readback_all(self, counts, cells_out=None, desired_out=None):
        """(cells_by_id, desired_by_id, alive per replicate), concatenated by
        replicate with counts[r] ids each."""
        n = np.ascontiguousarray(counts, dtype=np.int32)
        total = int(n.sum())
        cells = np.empty(total, np.int32) if cells_out is None else cells_out
        des = np.empty(total, np.int32) if desired_out is None else desired_out
        alive = np.zeros(len(n), np.int32)
        self._check(self.lib.fast_readback_all(self.h, _ptr(n), _ptr(cells), _ptr(des),
                                               _ptr(alive)), "fast_readback_all")
        return cells, des, alive

    def step(self, n: int = 1):
        self._check(self.lib.fast_step(self.h, int(n)), "fast_step")

    def plan_only(self, n: int = 1):
        self._check(self.lib.fast_plan_only(self.h, int(n)), "fast_plan_only")

    def readback(self, rep: int = 0, id_bound: int | None = None, cells_out=None,
                 desired_out=None):
        """Returns (cells_by_id, desired_by_id, stats dict); -1 = not present."""
        b = self.id_bound[rep] if id_bound is None else int(id_bound)
        cells = np.empty(b, np.int32) if cells_out is None else cells_out
        des = np.empty(b, np.int32) if desired_out is None else desired_out
        st = Stats()
        self._check(self.lib.fast_readback(self.h, rep, b, _ptr(cells), _ptr(des), C.byref(st)),
                    "fast_readback")
        return cells, des, st.as_dict()

    def digests(self, rep: int, max_steps: int):
        a = np.zeros(max_steps, np.uint64)
        b = np.zeros(max_steps, np.uint64)
        n = self._check(self.lib.fast_get_digests(self.h, rep, max_steps, _ptr(a), _ptr(b)),
                        "fast_get_digests")
        return a[:n], b[:n]

    def phase_times(self):
        """(planning kernels, FP64 re-check, movement footprints, movement rounds,
        bookkeeping) of the last step, ms."""
        ms = (C.c_float * 5)()
        self._check(self.lib.fast_phase_times(self.h, ms), "fast_phase_times")
        return tuple(ms)

    def move_profile(self):
        """(waiting agents after each round's claims, round durations in us) of the last step."""
        n_wait = np.zeros(140, np.uint32)
        t_ns = np.zeros(140, np.uint64)
        r = self._check(self.lib.fast_move_profile(self.h, 137, _ptr(n_wait), _ptr(t_ns)),
                        "fast_move_profile")
        m = min(r, 64)
        self.last_move_phases = t_ns[65:73].astype(np.float64).copy()
        self.last_move_block_max = t_ns[73:73 + m].astype(np.int64).copy()
        return n_wait[:m].copy(), np.diff(t_ns[:m + 1].astype(np.float64)) / 1e3

    def precision_report(self):
        r = PrecisionReport()
        self._check(self.lib.fast_precision_report_run(self.h, C.byref(r)),
                    "fast_precision_report_run")
        return r.as_dict()

    def reach_union(self, rep: int = 0) -> int:
        v = C.c_int64()
        self._check(self.lib.fast_reach_union(self.h, rep, C.byref(v)), "fast_reach_union")
        return v.value

    def plan_noalloc(self, rep: int, step: int, out_by_id) -> None:
        """Allocation-free planning pass into `out_by_id` (a contiguous int32
        tensor on this context's CUDA device, indexed by agent id); queued on
        the context's stream.  The library writes through the raw pointer and
        cannot check what it points to, so the tensor is checked here."""
        import torch

        if not isinstance(out_by_id, torch.Tensor):
            raise ValueError("out_by_id must be a torch tensor")
        if out_by_id.dtype != torch.int32:
            raise ValueError(f"out_by_id must be int32, not {out_by_id.dtype}")
        if not out_by_id.is_contiguous():
            raise ValueError("out_by_id must be contiguous")
        if not out_by_id.is_cuda or out_by_id.device != torch.device(self.device):
            raise ValueError(f"out_by_id must be on {self.device}, not {out_by_id.device}")
        self._check(self.lib.fast_plan_noalloc(self.h, rep, int(step), int(out_by_id.numel()),
                                               C.c_void_p(out_by_id.data_ptr())),
                    "fast_plan_noalloc")

    def autotune(self, trials: int = 5, cache: str | None = None, key: str | None = None):
        """Runs the library's autotuner (fast_autotune) and returns its report
        as a dict.  With `cache` (a JSON file path) and `key` (a caller's
        description of the workload), a choice stored under that key and this
        GPU's name is applied instead of tuning again, and a new one is
        stored."""
        import json

        full_key = None
        if cache is not None and key is not None:
            import torch

            full_key = f"{torch.cuda.get_device_name(self.device)}|{key}"
            try:
                with open(cache) as f:
                    stored = json.load(f).get(full_key)
            except (OSError, ValueError):
                stored = None
            if stored is not None:
                self.set_option("tile_shift", stored["tile_shift"])
                for v, l in enumerate(stored["lanes"]):
                    if l >= 0:
                        self.set_option(f"lanes_v{v + 1}", l)
                return dict(stored, cached=True)
        rep = TuneReport()
        self._check(self.lib.fast_autotune(self.h, int(trials), C.byref(rep)), "fast_autotune")
        out = rep.as_dict()
        if full_key is not None:
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
            table[full_key] = out
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, default=str)
            os.replace(tmp, cache)
        return dict(out, cached=False)

    def set_option(self, name: str, value: int):
        self._check(self.lib.fast_set_option(self.h, OPT[name], int(value)), "fast_set_option")


def floor_field(cell_type, static_field=None):
    """The static floor field fast_init_grid uses for this grid (host only,
    no GPU): (S, a, b) shaped like cell_type, S = fl(a + fl(b*sqrt2)), +inf
    and -1 at walls and cells no exit is reached from.  With static_field,
    the caller's field checked and decomposed into its step counts (a
    FastError names the first cell of the wrong form)."""
    t = np.ascontiguousarray(cell_type, dtype=np.uint8)
    H, W = t.shape
    S = np.empty((H, W), np.float64)
    a = np.empty((H, W), np.int32)
    b = np.empty((H, W), np.int32)
    src = None
    if static_field is not None:
        src = np.ascontiguousarray(static_field, dtype=np.float64)
        if src.shape != t.shape:
            raise ValueError("static_field must have the shape of cell_type")
    bad = C.c_int64(-1)
    rc = load().fast_floor_field(W, H, _ptr(t), _ptr(src), _ptr(S), _ptr(a), _ptr(b),
                                          C.byref(bad))
    if rc:
        raise FastError(rc, f"fast_floor_field: cell {bad.value}")
    return S, a, b


# -- self tests of the device arithmetic ------------------------------------------
def selftest_exp64(x: np.ndarray) -> np.ndarray:
    lib = load()
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty_like(x)
    rc = lib.fast_selftest_exp64(_ptr(x), _ptr(y), len(x))
    if rc:
        raise FastError(rc, "fast_selftest_exp64")
    return y


def selftest_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    lib = load()
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.empty_like(c)
    rc = lib.fast_selftest_philox(_ptr(c), _ptr(k), _ptr(out), len(c))
    if rc:
        raise FastError(rc, "fast_selftest_philox")
    return out


def selftest_ex2(lo: float, hi: float) -> float:
    lib = load()
    v = C.c_double()
    rc = lib.fast_selftest_ex2(C.c_float(lo), C.c_float(hi), C.byref(v))
    if rc:
        raise FastError(rc, "fast_selftest_ex2")
    return v.value


def build_checked() -> bool:
    """True when the loaded library is the debug build with index checks."""
    return load().fast_build_checked() == 1


def selftest_bounds(index: int, n: int):
    """(return code, index recorded) of one index check of the debug build
    on the GPU: FAST_ECUDA and the index when it is outside [0, n); in the
    release build the checks are compiled away (FAST_OK, -1)."""
    v = C.c_int64(-1)
    rc = load().fast_selftest_bounds(int(index), int(n), C.byref(v))
    return rc, v.value


def selftest_l2_read(nbytes: int = 32 << 20, iters: int = 50) -> float:
    """L2 read bandwidth in GB/s (a buffer of nbytes read iters times)."""
    v = C.c_double()
    rc = load().fast_selftest_l2_read(int(nbytes), int(iters), C.byref(v))
    if rc:
        raise FastError(rc, "fast_selftest_l2_read")
    return v.value


def selftest_barrier_cost(blocks: int, threads: int, iters: int = 1000) -> float:
    """Average ns per grid barrier of the library's cooperative kernels."""
    v = C.c_double()
    rc = load().fast_selftest_barrier_cost(int(blocks), int(threads), int(iters), C.byref(v))
    if rc:
        raise FastError(rc, "fast_selftest_barrier_cost")
    return v.value


def selftest_barrier_sum(blocks: int, threads: int, iters: int = 1000) -> int:
    """(block, barrier) pairs whose count sum at the grid barrier was wrong."""
    v = C.c_int64()
    rc = load().fast_selftest_barrier_sum(int(blocks), int(threads), int(iters), C.byref(v))
    if rc:
        raise FastError(rc, "fast_selftest_barrier_sum")
    return v.value


def selftest_barrier_timeout(limit_ns: int = 1_000_000) -> int:
    return load().fast_selftest_barrier_timeout(int(limit_ns))
