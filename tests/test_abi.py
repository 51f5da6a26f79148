"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every entry point that include/pgb.h declares, and argument errors
are reported without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pgb.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(pgb_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpgb():
    from paper_1506_03745_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pgb_create", "pgb_mesh_load", "pgb_tree_build", "pgb_matvec", "pgb_solve", "pgb_energy"):
        assert n in names


def test_every_declared_symbol_is_exported(libpgb):
    for n in _declared():
        assert hasattr(libpgb, n), n


def test_binding_covers_every_symbol():
    import paper_1506_03745_gb300._lib as L
    for n in _declared():
        assert n in L._SIGS, n


def test_argument_errors_need_no_device(libpgb):
    import paper_1506_03745_gb300._lib as L
    lib = L.lib()
    p = L.pgb_params()
    assert lib.pgb_default_params(ctypes.byref(p)) == 0
    assert (p.K, p.K_near, p.n_edge, p.P, p.theta, p.leaf_size) == (7, 19, 9, 6, 0.5, 32)
    assert (p.p2p_item, p.m2p_item, p.precond, p.graphs, p.lanes, p.overlap) == (64, 64, 0, 2, 4, 0)
    assert (p.batch, p.residual) == (1, 1)
    for f, v in (("p2p_item", 5000), ("m2p_item", -1), ("precond", 2), ("graphs", 3), ("lanes", 17), ("overlap", 2),
                 ("batch", 65), ("batch", -1), ("residual", 2)):
        q = L.pgb_params()
        lib.pgb_default_params(ctypes.byref(q))
        setattr(q, f, v)
        h0 = ctypes.c_void_p()
        assert lib.pgb_create(ctypes.byref(h0), ctypes.byref(q), None) == L.PGB_EINVAL
    bad = L.pgb_params(K=5, K_near=19, n_edge=9, P=6, theta=0.5, leaf_size=32, group_size=32)
    h = ctypes.c_void_p()
    assert lib.pgb_create(ctypes.byref(h), ctypes.byref(bad), None) == L.PGB_EINVAL
    assert lib.pgb_create(None, None, None) == L.PGB_EINVAL
    assert lib.pgb_destroy(None) == L.PGB_EINVAL
    assert lib.pgb_matvec(None, None, None, 0) == L.PGB_EINVAL
    assert lib.pgb_last_error(None) == b"null context"


def test_math_check_argument_errors(libpgb):
    import paper_1506_03745_gb300._lib as L
    lib = L.lib()
    assert lib.pgb_math_check(None, -1, None) == L.PGB_EINVAL
    assert lib.pgb_math_check(None, 4, None) == L.PGB_EINVAL
    assert lib.pgb_math_check(None, 0, None) == L.PGB_OK


def test_alloc_count_needs_no_device(libpgb):
    import paper_1506_03745_gb300._lib as L
    lib = L.lib()
    assert lib.pgb_alloc_count(None) == L.PGB_EINVAL
    assert L.pgb_alloc_count() >= 0
