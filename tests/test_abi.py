"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/fastgb.h declares; the binding refuses to run
without a GPU instead of falling back to the CPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastgb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fast_[a-z0-9_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    from paper_0911_2900_gb300 import build

    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fast_create", "fast_init_grid", "fast_place_agents", "fast_step",
                 "fast_readback", "fast_last_error", "fast_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_0911_2900_gb300 as fg

    assert set(declared_functions()) <= set(fg.EXPORTS), \
        set(declared_functions()) - set(fg.EXPORTS)


def test_create_without_gpu_fails_loudly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p(123)
    lib.fast_create.restype = C.c_int
    rc = lib.fast_create(C.byref(h), 1, 1, 0, None, None, None, None)
    assert rc == -4          # FAST_ECUDA
    assert not h.value


def test_binding_refuses_cpu(lib):
    import torch

    import paper_0911_2900_gb300 as fg

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fg.FastError):
        fg.Context(1)


def test_create_rejects_bad_arguments(lib):
    h = C.c_void_p()
    lib.fast_create.restype = C.c_int
    assert lib.fast_create(C.byref(h), 0, 1, 0, None, None, None, None) == -1
    assert lib.fast_create(C.byref(h), 1, 7, 0, None, None, None, None) == -1
    assert lib.fast_create(C.byref(h), 1, 1, 9, None, None, None, None) == -1
    assert lib.fast_create(C.byref(h), 300, 1, 0, None, None, None, None) == -1


def test_plan_noalloc_checks_the_output_tensor():
    """The allocation-free pass writes by agent id through a raw device
    pointer, which the C side cannot check: the binding refuses a tensor of
    another dtype, a non-contiguous view and one that is not on the
    context's CUDA device, before any call into the library (no GPU needed:
    the refusals come first)."""
    import torch

    import paper_0911_2900_gb300 as fg

    class NoLib:
        def __getattr__(self, name):
            raise AssertionError(f"the library was called ({name})")

    ctx = object.__new__(fg.Context)
    ctx.lib, ctx.h, ctx.device = NoLib(), None, torch.device("cuda", 0)
    with pytest.raises(ValueError, match="torch tensor"):
        ctx.plan_noalloc(0, 0, [0, 1, 2])
    with pytest.raises(ValueError, match="int32"):
        ctx.plan_noalloc(0, 0, torch.zeros(8, dtype=torch.int64))
    with pytest.raises(ValueError, match="int32"):
        ctx.plan_noalloc(0, 0, torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError, match="contiguous"):
        ctx.plan_noalloc(0, 0, torch.zeros(16, dtype=torch.int32)[::2])
    with pytest.raises(ValueError, match="must be on"):
        ctx.plan_noalloc(0, 0, torch.zeros(8, dtype=torch.int32))
    with pytest.raises(ValueError, match="must be on"):
        ctx.plan_noalloc(0, 0, torch.zeros(8, dtype=torch.int32, device="meta"))


def test_checked_build_exports_the_same_boundary():
    """The debug build (index checks in the kernels) is a drop-in for the
    release library: the same declared symbols, and each reports which build
    it is (a host-only call)."""
    from paper_0911_2900_gb300 import build

    rel = C.CDLL(build.build())
    chk = C.CDLL(build.build(checked=True))
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, missing
    rel.fast_build_checked.restype = chk.fast_build_checked.restype = C.c_int
    assert rel.fast_build_checked() == 0 and chk.fast_build_checked() == 1


def test_memory_limit_accounting():
    """The binding's allocator refuses a request that would take the live
    total above the context's memory limit (the library then reports
    FAST_ENOMEM), and counts freed memory back; CPU tensors stand in for
    device memory here (no kernel runs)."""
    import ctypes as C

    from paper_0911_2900_gb300 import _TorchAllocator

    a = _TorchAllocator("cpu", limit=1000)
    p1 = a._alloc(600, None)
    assert p1 and a.total == 600
    assert a._alloc(500, None) is None and a.total == 600
    p2 = a._alloc(400, None)
    assert p2 and a.total == 1000
    a._free(p1, None)
    assert a.total == 400
    assert a._alloc(500, None) and a.total == 900
    a._free(C.c_void_p(12345).value, None)  # an unknown pointer is ignored
    assert a.total == 900
    unlimited = _TorchAllocator("cpu")
    assert unlimited._alloc(1 << 20, None) and unlimited.total == 1 << 20
