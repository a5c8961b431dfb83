"""CPU checks of the C-ABI library: it builds, loads, and exports every
entry point that include/leg.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1106_0463_gb300 import build as B
    return B.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "leg.h")).read()
    return re.findall(r"LEG_API\s+[\w\s\*]*?\b(leg_\w+)\s*\(", text)


def test_header_declares_the_boundary():
    names = set(_declared())
    for must in ("leg_plan_create", "leg_plan_destroy", "leg_forward", "leg_backward", "leg_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols(libpath):
    import paper_1106_0463_gb300 as leg
    assert sorted(leg.declared_symbols()) == sorted(_declared())
    assert os.path.samefile(leg.library_path(), libpath)


def test_null_plan_is_rejected_without_a_gpu(libpath):
    # argument validation happens before any CUDA call
    lib = ctypes.CDLL(libpath)
    lib.leg_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)] + [ctypes.c_int] * 5
    lib.leg_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    assert lib.leg_plan_create(ctypes.byref(h), 64, 100, 33, 0, 0) == 1      # M not a power of two
    assert b"power of two" in lib.leg_last_error()
    assert lib.leg_plan_create(ctypes.byref(h), 200, 256, 33, 0, 0) == 1     # N > M/2
    assert lib.leg_plan_create(ctypes.byref(h), 64, 256, 1, 0, 0) == 1       # K < 2
    assert lib.leg_plan_create(ctypes.byref(h), 64, 256, 33, 0, 9) == 1      # dtype
    assert lib.leg_plan_create(None, 64, 256, 33, 0, 0) == 1


def test_every_handle_entry_point_rejects_null_without_a_gpu(libpath):
    """Each entry point that takes a plan or a ragged batch checks the handle
    before it touches the device: a NULL handle is LEG_ERR_INVALID_ARG (1)."""
    lib = ctypes.CDLL(libpath)
    vp, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    calls = {
        "leg_plan_reserve": ([vp, i], (None, 4)),
        "leg_plan_info": ([vp] + [vp] * 7, (None,) + (None,) * 7),
        "leg_forward": ([vp, vp, vp, i, vp], (None, None, None, 4, None)),
        "leg_forward_profiled": ([vp, vp, vp, i, vp, vp], (None, None, None, 4, None, None)),
        "leg_forward_batches": ([vp, vp, vp, i, i, vp], (None, None, None, 4, 2, None)),
        "leg_forward_batches_profiled": ([vp, vp, vp, i, i, vp, vp], (None, None, None, 4, 2, None, None)),
        "leg_backward": ([vp, vp, vp, i, vp], (None, None, None, 4, None)),
        "leg_plain_forward": ([vp, i, vp, i, vp, vp], (None, 0, None, 4, None, None)),
        "leg_plain_forward_cheb": ([vp, vp, i, i, vp, vp], (None, None, 8, 4, None, None)),
        "leg_plan_status": ([vp, i], (None, 0)),
        "leg_plan_set_wait_limit": ([vp, ll], (None, 1000)),
        "leg_plan_set_tile": ([vp, i], (None, 0)),
        "leg_plan_set_host_overlap": ([vp, i], (None, 1)),
        "leg_plan_tile_info": ([vp, i, vp, vp, vp], (None, 4, None, None, None)),
        "leg_plan_autotune": ([vp, vp, vp, i, vp, vp, vp], (None, None, None, 4, None, None, None)),
        "leg_forward_host": ([vp, vp, vp, i, vp], (None, None, None, 4, None)),
        "leg_forward_host_batches": ([vp, vp, vp, i, i, vp], (None, None, None, 4, 2, None)),
        "leg_forward_noalloc": ([vp, vp, vp, i, vp], (None, None, None, 4, None)),
        "leg_forward_ragged": ([vp, vp, vp, vp], (None, None, None, None)),
        "leg_ragged_status": ([vp, i], (None, 0)),
    }
    assert set(calls) <= set(_declared())
    for name, (argtypes, args) in calls.items():
        fn = getattr(lib, name)
        fn.argtypes = argtypes
        fn.restype = ctypes.c_int
        assert fn(*args) == 1, name
