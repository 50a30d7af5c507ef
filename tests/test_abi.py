"""The C-ABI library loads and exports every entry point include/*.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(ns_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def _lib_path():
    from paper_1511_06959_gb300 import build
    if not os.path.exists(build.OUT):
        build.build()
    return build.OUT


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["ns_primal_step", "ns_adjoint_step", "ns_objective", "ns_growth_sigma1",
                     "ns_add_adjoint_viscosity"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1511_06959_gb300 import api
    assert sorted(api.EXPORTED) == sorted(n for n in _declared() if n in api.EXPORTED)
    undeclared_in_binding = [n for n in _declared() if n not in api.EXPORTED and
                             not n.endswith("_noalloc")]
    assert not undeclared_in_binding, undeclared_in_binding


def test_error_strings_without_gpu():
    from paper_1511_06959_gb300 import api
    lib = api.load_library(_lib_path())
    assert lib.ns_error_string(api.NS_ERR_ARG) == b"invalid argument"
    assert lib.ns_error_string(0) == b"ok"


def test_create_rejects_bad_params_without_gpu():
    """Argument validation happens before any CUDA call, so it runs on CPU."""
    from paper_1511_06959_gb300 import api
    lib = api.load_library(_lib_path())
    p = api.NsParams(0, 4, 4, 1, 0.1, 0.1, 0.1, 1.4, 0.0, 0.72, 0.0, 0, 0, 1.0)
    ctx = ctypes.c_void_p()
    assert lib.ns_create(ctypes.byref(p), None, ctypes.byref(ctx)) == api.NS_ERR_ARG
    p.nx = 4
    p.precision = 7
    assert lib.ns_create(ctypes.byref(p), None, ctypes.byref(ctx)) == api.NS_ERR_ARG
    assert lib.ns_primal_step(None, None, None, None) == api.NS_ERR_ARG
    assert lib.ns_last_error(None) == api.NS_ERR_ARG


def test_host_arena_must_be_contiguous_host_memory():
    """The snapshot arena of a host-tier sweep is host memory: the binding refuses a
    non-contiguous tensor before any call (a CUDA tensor is refused the same way)."""
    torch = pytest.importorskip("torch")
    from paper_1511_06959_gb300 import api
    assert api._host_ptr(None) is None
    t = torch.empty(64, dtype=torch.uint8)
    assert api._host_ptr(t).value == t.data_ptr()
    with pytest.raises(ValueError):
        api._host_ptr(torch.empty((8, 8), dtype=torch.uint8).t())


def test_size_and_plane_checks_without_gpu():
    """ns_create and ns_objective_noalloc refuse grids beyond the kernels' 32-bit plane
    indexing and objective planes whose index arithmetic could overflow, before any CUDA
    call."""
    from paper_1511_06959_gb300 import api
    lib = api.load_library(_lib_path())
    f = lib.ns_objective_noalloc
    f.argtypes = [ctypes.POINTER(api.NsParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(256)
    big = api.NsParams(1 << 16, 1 << 16, 1, 1, 0.1, 0.1, 0.1, 1.4, 0.0, 0.72, 0.0, 0, 6, 1.0)
    assert lib.ns_create(ctypes.byref(big), None, ctypes.byref(ctx)) == api.NS_ERR_ARG
    assert f(ctypes.byref(big), None, dummy, 1.0, dummy, None) == api.NS_ERR_ARG
    far = api.NsParams(8, 4, 2, 1, 0.1, 0.1, 0.1, 1.4, 0.0, 0.72, 0.0, 0, 1 << 30, 1.0)
    assert lib.ns_create(ctypes.byref(far), None, ctypes.byref(ctx)) == api.NS_ERR_ARG
    assert f(ctypes.byref(far), None, dummy, 1.0, dummy, None) == api.NS_ERR_ARG
    far.plane_i = -(1 << 30)
    assert f(ctypes.byref(far), None, dummy, 1.0, dummy, None) == api.NS_ERR_ARG


def test_binding_refuses_undersized_tensors_before_any_call():
    """The binding checks that every tensor holds the elements the library will touch
    through its raw pointer (here on CPU tensors: the size check comes first)."""
    torch = pytest.importorskip("torch")
    from paper_1511_06959_gb300 import api
    with pytest.raises(ValueError, match="elements"):
        api._sized(torch.empty(7, dtype=torch.float64), torch.float64, 8, "field")
    assert api._sized(None, torch.float64, 8, "field") is None
