"""Host-only checks of the C ABI: the library builds, loads, exports every
symbol declared in include/pa_nufft.h, and rejects invalid arguments before
touching the device.  No compute call is made (no GPU here)."""
import ctypes
import os
import re
from ctypes import byref, c_void_p

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_02946_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pa_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pa_plan_create", "pa_reconstruct", "pa_reconstruct_adjoint", "pa_plan_destroy",
                     "pa_position_grad", "pa_batch_create", "pa_batch_run", "pa_batch_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib._name)
    for name in declared_functions():
        assert hasattr(raw, name), name


def test_version_and_empty_error(lib):
    assert b"sm_103a" in lib.pa_version()
    assert lib.pa_last_error() is not None


def _create(lib, **kw):
    from paper_1501_02946_gb300._lib import PaGrid
    args = dict(M=4, xy=np.zeros((4, 2)), w=None, nt=16, dt=1e-8, c=1500.0,
                grid=PaGrid(8, 8, 8, 1e-4, 1e-4, 1e-4), sigma=2, width=8, flags=0)
    args.update(kw)
    ptr = c_void_p()
    xy = args["xy"]
    rc = lib.pa_plan_create(byref(ptr), args["M"], None if xy is None else xy.ctypes.data_as(c_void_p),
                            None if args["w"] is None else args["w"].ctypes.data_as(c_void_p),
                            args["nt"], args["dt"], args["c"],
                            None if args["grid"] is None else byref(args["grid"]),
                            args["sigma"], args["width"], args["flags"], None)
    return rc, ptr


@pytest.mark.parametrize("bad", [
    dict(M=0), dict(xy=None), dict(grid=None), dict(nt=1), dict(dt=0.0), dict(dt=float("nan")),
    dict(c=-1.0), dict(sigma=1), dict(sigma=5), dict(width=7), dict(width=10), dict(flags=4),
    dict(xy=np.array([[0.0, float("nan")]] * 4)), dict(w=np.array([1.0, 1.0, -1.0, 1.0])),
])
def test_invalid_arguments_rejected(lib, bad):
    rc, ptr = _create(lib, **bad)
    assert rc == 1
    assert ptr.value is None
    assert len(lib.pa_last_error()) > 0


def test_unsupported_sizes_rejected(lib):
    from paper_1501_02946_gb300._lib import PaGrid
    rc, _ = _create(lib, grid=PaGrid(11, 8, 8, 1e-4, 1e-4, 1e-4))   # 11 is not 7-smooth
    assert rc == 2
    rc, _ = _create(lib, grid=PaGrid(8, 4, 8, 1e-4, 1e-4, 1e-4))    # sigma*ny < 2*width
    assert rc == 2
    rc, _ = _create(lib, nt=13)
    assert rc == 2


def test_null_plan_calls_are_errors(lib):
    assert lib.pa_reconstruct(None, None, None, None) == 1
    assert lib.pa_reconstruct_adjoint(None, None, None, None) == 1
    assert lib.pa_position_grad(None, None, None, None, None, None) == 1
    assert lib.pa_plan_destroy(None) == 0
    assert lib.pa_batch_destroy(None) == 0
    assert lib.pa_profile_enable(None, 1) == 1
    assert lib.pa_profile_select(None, 1) == 1
