"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/mg.h declares, and rejects
bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1104_1703_gb300 import binding as B
from paper_1104_1703_gb300 import build as Bd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_create_hierarchy", "mg_set_rhs", "mg_set_dirichlet", "mg_set_dirichlet_from_coarse",
                     "mg_vcycle", "mg_solve", "mg_destroy_hierarchy", "mg_get_solution", "mg_set_solution"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(Bd.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert set(B.SIGNATURES) == set(declared_functions())


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(Bd.ARCH)
    assert os.path.getsize(Bd.build()) > 0


def test_default_options_are_the_papers():
    o = B.mg_default_options()
    assert (o.n_pre, o.n_post, o.n_cycles, o.coarse_sweeps, o.hold_solves, o.eta, o.order) == (2, 2, 1, 50, 10,
                                                                                                0.5, 0)


def test_appended_option_defaults_and_ranges():
    """The options appended after the paper's (precision and kernel
    choices): their defaults, and every out-of-range value refused on the
    host before any device work."""
    o = B.mg_default_options()
    assert (o.precision, o.inner_cycles, o.use_graphs, o.coarse_cluster, o.smoother_pass) == (0, 1, 1, 0, 0)
    assert (o.fp64_sum, o.fine_segments, o.coarse_matrix) == (1, 3, 1)
    lib = B.lib()
    out = ctypes.c_void_p(123)
    mask = np.ones((4, 4, 4), np.int8)
    p = mask.ctypes.data_as(ctypes.c_void_p)
    for field, value in [("fine_segments", -1), ("fine_segments", 4), ("coarse_matrix", 2), ("coarse_matrix", -1),
                         ("fp64_sum", 2), ("inner_cycles", 0), ("inner_cycles", 17), ("smoother_pass", 2),
                         ("n_cycles", 0), ("n_cycles", 5)]:
        bad = B.mg_default_options()
        setattr(bad, field, value)
        assert lib.mg_create_hierarchy(p, 0, 4, 4, 4, 0.25, ctypes.byref(bad), None, ctypes.byref(out)) == \
            B.MG_ERR_INVALID_ARG, (field, value)
        assert "invalid options" in B.mg_last_error()


def test_invalid_arguments_rejected_on_host():
    lib = B.lib()
    out = ctypes.c_void_p(123)
    mask = np.ones((4, 4, 4), np.int8)
    p = mask.ctypes.data_as(ctypes.c_void_p)
    assert lib.mg_create_hierarchy(None, 0, 4, 4, 4, 0.25, None, None, ctypes.byref(out)) == B.MG_ERR_INVALID_ARG
    assert out.value is None
    assert lib.mg_create_hierarchy(p, 0, 0, 4, 4, 0.25, None, None, ctypes.byref(out)) == B.MG_ERR_INVALID_ARG
    assert lib.mg_create_hierarchy(p, 0, 4, 4, 4, -1.0, None, None, ctypes.byref(out)) == B.MG_ERR_INVALID_ARG
    assert lib.mg_create_hierarchy(p, 0, 4, 4, 4, float("nan"), None, None, ctypes.byref(out)) == \
        B.MG_ERR_INVALID_ARG
    assert lib.mg_create_hierarchy(p, 0, 4096, 4, 4, 0.25, None, None, ctypes.byref(out)) == B.MG_ERR_INVALID_ARG
    bad = B.mg_default_options()
    bad.eta = -1
    assert lib.mg_create_hierarchy(p, 0, 4, 4, 4, 0.25, ctypes.byref(bad), None, ctypes.byref(out)) == \
        B.MG_ERR_INVALID_ARG
    assert "invalid options" in B.mg_last_error()
    assert lib.mg_solve(None, 1e-8, 10, None) == B.MG_ERR_INVALID_ARG
    assert lib.mg_set_rhs(None, p, 0) == B.MG_ERR_INVALID_ARG
    assert lib.mg_destroy_hierarchy(None) == B.MG_OK
    assert B.mg_status_string(B.MG_ERR_DIVERGED) == "diverged"


def test_binding_marshalling_rejects_bad_shapes():
    with pytest.raises(ValueError):
        B._in(np.zeros((3, 3)), np.float64, (3, 3, 3), "x")
    p, where, keep = B._in(np.zeros((2, 3, 4), np.float32), np.float64, (2, 3, 4), "x")
    assert where == B.MG_MEM_HOST and keep.dtype == np.float64
