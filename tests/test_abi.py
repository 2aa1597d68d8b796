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
