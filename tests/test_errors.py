"""Argument validation of the C ABI: every rejected call returns its error code before
any CUDA call, so these run on the host (no GPU)."""
import ctypes

import pytest

from paper_2304_08159_gb300 import wl


@pytest.fixture(scope="module")
def lib():
    return wl.load()


def create(dims, nu=0.01, U=(1.0, 0.0, 0.0), body=None, opts=None):
    rc, h = wl.wl_create(dims, nu, U[: len(dims)], body, opts)
    assert not h.value, "a rejected create must not return a handle"
    return rc


def test_bad_grids(lib):
    assert create((1, 8)) == wl.WL_EINVAL          # a side shorter than 2
    assert create((0, 8)) == wl.WL_EINVAL          # an empty grid
    assert create((8, -4)) == wl.WL_EINVAL
    for ndim in (1, 4):  # 1-D and 4-D, straight through the C ABI
        d = (ctypes.c_int * 4)(8, 8, 8, 8)
        u = (ctypes.c_double * 4)(1.0, 0.0, 0.0, 0.0)
        h = ctypes.c_void_p()
        assert lib.wl_create(d, ndim, 0.01, u, None, None, ctypes.byref(h)) == wl.WL_EINVAL
        assert not h.value
    assert create((1 << 21, 4)) == wl.WL_EINVAL    # side too long


def test_bad_physics_and_options(lib):
    assert create((16, 8), nu=float("nan")) == wl.WL_EINVAL
    assert create((16, 8), nu=-1.0) == wl.WL_EINVAL
    assert create((16, 8), U=(float("inf"), 0.0)) == wl.WL_EINVAL
    for field, bad in (("tol", 0.0), ("max_vcycles", -1), ("post", 0), ("eps", 0.0), ("dt_cap", 0.0),
                       ("precision", 2)):
        o = wl.wl_default_opts()
        setattr(o, field, bad)
        assert create((16, 8), opts=o) == wl.WL_EINVAL, field


def test_bad_bodies(lib):
    torus = wl.make_body({"kind": wl.WL_BODY_TORUS, "center": (8, 8), "radius": 4, "radius2": 1})
    assert create((16, 16), body=torus) == wl.WL_EINVAL  # a torus needs 3-D
    b = wl.make_body({"kind": 7, "center": (8, 8), "radius": 4})
    assert create((16, 16), body=b) == wl.WL_EINVAL


def test_caller_workspace_too_small_or_misaligned(lib):
    dims = (32, 16)
    o = wl.wl_default_opts()
    need = wl.wl_workspace_bytes(dims, o)
    assert need > 0
    # never dereferenced: the size and alignment checks come first
    o.workspace = ctypes.c_void_p(1 << 20)
    o.workspace_bytes = need - 1
    assert create(dims, opts=o) == wl.WL_ENOMEM
    o.workspace = ctypes.c_void_p((1 << 20) + 16)
    o.workspace_bytes = need
    assert create(dims, opts=o) == wl.WL_ENOMEM


def test_wait_probe_rejects_bad_limits(lib):
    assert wl.wl_wait_probe(0.0)[0] == wl.WL_EINVAL
    assert wl.wl_wait_probe(-1.0)[0] == wl.WL_EINVAL
    assert wl.wl_wait_probe(11.0)[0] == wl.WL_EINVAL
