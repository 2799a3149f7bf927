"""The C ABI library: builds, loads, exports every declared symbol, and
rejects bad arguments on the host (no GPU needed for any of this)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2104_06718_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load_library()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ld_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ld_bound" in names and "ld_intermediate_bounds" in names and "ld_bound_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.EXPORTED) <= set(names)


def test_status_strings_and_defaults(lib):
    assert lib.ld_status_str(0) == b"ok"
    assert lib.ld_status_str(6).startswith(b"non-finite")
    o = binding.Opts()
    lib.ld_opts_default(C.byref(o))
    assert abs(o.alpha0 - 1e-2) < 1e-9 and abs(o.alpha_end - 1e-4) < 1e-9
    assert abs(o.beta1 - 0.9) < 1e-7 and abs(o.beta2 - 0.999) < 1e-7
    assert o.init == binding.LD_INIT_CROWN and o.fp64_final == 1


def _desc(kind, cin, h, w, cout, k, s, p, W, b):
    d = binding.LayerDesc()
    d.kind, d.cin, d.h, d.w, d.cout, d.kh, d.kw, d.stride, d.pad = kind, cin, h, w, cout, k, k, s, p
    d.W, d.b = W.ctypes.data, b.ctypes.data
    return d


def test_create_rejects_bad_shapes_on_host(lib):
    W1 = np.zeros((4, 3), np.float32)
    b1 = np.zeros(4, np.float32)
    W2 = np.zeros((1, 5), np.float32)   # does not chain: 4 outputs feed 5 inputs
    b2 = np.zeros(1, np.float32)
    arr = (binding.LayerDesc * 2)(_desc(0, 3, 1, 1, 4, 1, 1, 0, W1, b1), _desc(0, 5, 1, 1, 1, 1, 1, 0, W2, b2))
    h = C.c_void_p()
    assert lib.ld_net_create(arr, 2, None, C.byref(h), None) == binding.LD_ERR_SHAPE
    # last layer with several outputs needs a margin vector
    W2 = np.zeros((3, 4), np.float32)
    b2 = np.zeros(3, np.float32)
    arr = (binding.LayerDesc * 2)(_desc(0, 3, 1, 1, 4, 1, 1, 0, W1, b1), _desc(0, 4, 1, 1, 3, 1, 1, 0, W2, b2))
    assert lib.ld_net_create(arr, 2, None, C.byref(h), None) == binding.LD_ERR_SHAPE
    # conv whose output plane is empty
    Wc = np.zeros((2, 1, 5, 5), np.float32)
    bc = np.zeros(2, np.float32)
    arr = (binding.LayerDesc * 2)(_desc(1, 1, 3, 3, 2, 5, 1, 0, Wc, bc), _desc(0, 4, 1, 1, 1, 1, 1, 0, W1, b1))
    assert lib.ld_net_create(arr, 2, None, C.byref(h), None) == binding.LD_ERR_SHAPE
    # last layer must be FC
    arr = (binding.LayerDesc * 2)(_desc(0, 3, 1, 1, 4, 1, 1, 0, W1, b1), _desc(1, 1, 2, 2, 1, 1, 1, 0, Wc, bc))
    assert lib.ld_net_create(arr, 2, None, C.byref(h), None) in (binding.LD_ERR_SHAPE,)
    assert lib.ld_net_create(None, 2, None, C.byref(h), None) == binding.LD_ERR_ARG
    assert lib.ld_net_create(arr, 1, None, C.byref(h), None) == binding.LD_ERR_ARG


def test_calls_reject_null_handle_on_host(lib):
    o = binding.Opts()
    lib.ld_opts_default(C.byref(o))
    assert lib.ld_bound(None, None, None, None, None, 1, None, None, 1, 1, C.byref(o), None, None, None, None, None) == binding.LD_ERR_ARG
    assert lib.ld_intermediate_bounds(None, None, None, 1, None, None, None, None) == binding.LD_ERR_ARG
    assert lib.ld_bound_backward(None, *([None] * 4), 1, None, None, 1, *([None] * 9)) == binding.LD_ERR_ARG
    assert lib.ld_dual_supergradient(None, *([None] * 4), 1, None, None, 1, *([None] * 5)) == binding.LD_ERR_ARG
    assert lib.ld_bound_ball(None, *([None] * 4), 1, None, None, 1, 1, C.byref(o), *([None] * 5)) == binding.LD_ERR_ARG
    assert lib.ld_bound_trace(None, *([None] * 4), 1, None, None, 1, 1, C.byref(o), *([None] * 6)) == binding.LD_ERR_ARG
    assert lib.ld_intermediate_bounds_ball(None, None, None, 1, None, None, None, None) == binding.LD_ERR_ARG
    assert lib.ld_net_destroy(None) == binding.LD_ERR_ARG
    assert lib.ld_net_reserve(None, 4) == binding.LD_ERR_ARG


def test_allocation_failure_injection_on_host(lib):
    """The failure-injection hook makes the library's first device allocation
    fail on the host, before any CUDA allocator call: ld_net_create reports
    the injected code (no GPU is needed to reach it)."""
    W1 = np.ones((4, 3), np.float32)
    b1 = np.zeros(4, np.float32)
    W2 = np.ones((1, 4), np.float32)
    b2 = np.zeros(1, np.float32)
    arr = (binding.LayerDesc * 2)(_desc(0, 3, 1, 1, 4, 1, 1, 0, W1, b1), _desc(0, 4, 1, 1, 1, 1, 1, 0, W2, b2))
    h = C.c_void_p()
    try:
        assert lib.ld_test_inject_alloc_failure(0, binding.LD_ERR_NOMEM) == binding.LD_OK
        assert lib.ld_net_create(arr, 2, None, C.byref(h), None) == binding.LD_ERR_NOMEM
        assert not h.value
        assert lib.ld_test_inject_alloc_failure(0, binding.LD_ERR_CUDA) == binding.LD_OK
        assert lib.ld_net_create(arr, 2, None, C.byref(h), None) == binding.LD_ERR_CUDA
        assert lib.ld_test_inject_alloc_failure(0, binding.LD_ERR_ARG) == binding.LD_ERR_ARG
    finally:
        lib.ld_test_inject_alloc_failure(-1, 0)
