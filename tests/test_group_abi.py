"""The grouped-solve entry points (include/ldgmg.h) on the CPU: argument
checks that return before any device work (no GPU needed).  The solves
themselves are tested in test_gpu_group.py."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


def test_group_argument_checks(lib):
    L = lib._lib
    g = ctypes.c_void_p()
    assert L.ldgmg_group_create(ctypes.byref(g)) == lib.OK and g.value
    assert L.ldgmg_group_create(None) == lib.EINVAL
    vp = ctypes.c_void_p
    # nothing to solve
    assert L.ldgmg_solve_group(g, 0, None, None, None, None, None, None, None, None) == lib.OK
    # bad counts and null arrays
    assert L.ldgmg_solve_group(g, -1, None, None, None, None, None, None, None, None) == lib.EINVAL
    assert L.ldgmg_solve_group(g, (1 << 20) + 1, None, None, None, None, None, None, None, None) == lib.EINVAL
    assert L.ldgmg_solve_group(g, 1, None, None, None, None, None, None, None, None) == lib.EINVAL
    assert L.ldgmg_solve_group(None, 1, None, None, None, None, None, None, None, None) == lib.EINVAL
    # a null hierarchy / vector of one problem
    hs = (vp * 1)(None)
    bs = (vp * 1)(None)
    xs = (vp * 1)(None)
    tol = (ctypes.c_double * 1)(1e-10)
    assert L.ldgmg_solve_group(g, 1, hs, bs, xs, tol, None, None, None, None) == lib.EINVAL
    assert b"null" in L.ldgmg_last_error()
    c = ctypes.c_int(-1)
    assert L.ldgmg_group_cluster(None, ctypes.byref(c)) == lib.EINVAL
    L.ldgmg_group_free(g)
    L.ldgmg_group_free(None)


def test_server_group_options(lib):
    with pytest.raises(lib.LdgmgError):
        lib.Server(workers=1, simulate=True, group_max=-1)
    s = lib.Server(workers=1, simulate=True, group_dofs=1 << 14, group_max=1)
    st = s.stats()
    assert st["group_calls"] == 0 and st["group_requests"] == 0
    s.close()
