"""CPU checks of the C-ABI library without a GPU.

  * the shared library loads and exports every function declared in include/*.h;
  * the library's host-side setup (assembly, operator coarsening, block-Jacobi
    inverse blocks, balanced SAI) matches the oracle entry by entry.
"""
import os
import re

import numpy as np
import pytest

from oracle import ldg
from oracle import multigrid as mg
from paper_2412_12506_gb300.inputs import circle_mu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    so = os.path.join(ROOT, "paper_2412_12506_gb300", "libldgmg.so")
    if not os.path.exists(so):
        from paper_2412_12506_gb300 import build
        build.build()
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(ldgmg_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    declared = _declared_functions()
    assert len(declared) >= 20
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(so, n)]
    assert not missing, missing
    assert set(lib.EXPORTED) <= declared


def _dense(rp, col, vals):
    from bsr_dense import bsr_to_dense
    return bsr_to_dense(rp, col, vals)


def _pattern(rp, col, N):
    P = np.zeros((N, N), dtype=bool)
    for i in range(N):
        P[i, col[rp[i]:rp[i + 1]]] = True
    return P


CASES = [
    (2, 4, 1, None), (2, 8, 2, None), (2, 6, 3, None), (2, 2, 2, None), (2, 1, 1, None),
    (3, 4, 1, None), (3, 2, 2, None), (2, 8, 2, "circle"), (2, 6, 1, "circle"),
]


@pytest.mark.parametrize("d,n,p,mu_kind", CASES)
def test_host_operators_match_oracle(lib, d, n, p, mu_kind):
    mu = circle_mu(d, n, seed=2, mu_in=1e4) if mu_kind else None
    H = lib.HostHierarchy(d, n, p, mu, smoother="jacobi")
    levels = mg.build_levels(d, n, p, mu)
    assert H.nlevels == len(levels)
    for l, lv in enumerate(levels):
        rp, col, vals = H.export(l, lib.MAT_A)
        A = _dense(rp, col, vals)
        Ao = lv.A.dense()
        scale = np.abs(Ao).max()
        assert np.abs(A - Ao).max() <= 1e-12 * scale, (l, np.abs(A - Ao).max() / scale)
        assert np.array_equal(_pattern(rp, col, lv.N), lv.A.pat.toarray().astype(bool))


@pytest.mark.parametrize("d,n,p,mu_kind", [(2, 8, 2, None), (2, 6, 3, "circle"), (3, 4, 1, None)])
def test_host_jacobi_blocks_match_oracle(lib, d, n, p, mu_kind):
    mu = circle_mu(d, n, seed=2, mu_in=1e4) if mu_kind else None
    H = lib.HostHierarchy(d, n, p, mu, smoother="jacobi")
    levels = mg.build_levels(d, n, p, mu)
    for l, lv in enumerate(levels[:-1]):
        jac = mg.Jacobi(lv.A)
        _, _, vals = H.export(l, lib.MAT_D)
        for i in range(lv.N):
            ref = jac.Dinv[i]
            assert np.abs(vals[i] - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("d,n,p,mu_kind,ell", [(2, 8, 2, None, 1), (2, 6, 1, "circle", 1),
                                               (2, 8, 1, None, 0), (2, 8, 1, None, 2), (3, 4, 1, None, 1),
                                               (2, 4, 2, None, 1)])
def test_host_sai_matches_oracle(lib, d, n, p, mu_kind, ell):
    mu = circle_mu(d, n, seed=1, mu_in=1e4) if mu_kind else None
    H = lib.HostHierarchy(d, n, p, mu, smoother="sai", sai_level=ell)
    levels = mg.build_levels(d, n, p, mu)
    for l, lv in enumerate(levels[:-1]):
        sai = mg.SAI(lv.A, ell)
        Bo = sai.B.dense()
        rp, col, vals = H.export(l, lib.MAT_B)
        B = _dense(rp, col, vals)
        scale = np.abs(Bo).max()
        assert np.abs(B - Bo).max() <= 1e-9 * scale, (l, np.abs(B - Bo).max() / scale)
        assert np.array_equal(_pattern(rp, col, lv.N), sai.B.pat.toarray().astype(bool))
        rpt, colt, valst = H.export(l, lib.MAT_BT)
        assert np.array_equal(_dense(rpt, colt, valst), B.T)


def test_host_pools_are_small_on_uniform_meshes(lib):
    """On a uniform periodic mesh every row of A holds the same 2d+1 distinct
    blocks, so setup work does not grow with N."""
    for n in (8, 32):
        H = lib.HostHierarchy(2, n, 2, smoother="sai")
        assert H.info(0)["distinct_A"] == 5
    H = lib.HostHierarchy(3, 8, 1, smoother="sai")
    assert H.info(0)["distinct_A"] == 7


def test_host_rejects_bad_arguments(lib):
    with pytest.raises(lib.LdgmgError) as e:
        lib.HostHierarchy(4, 4, 1)
    assert e.value.status == lib.EINVAL
    with pytest.raises(lib.LdgmgError):
        lib.HostHierarchy(2, 4, 1, mu=np.full(16, -1.0))
    with pytest.raises(lib.LdgmgError):
        lib.HostHierarchy(2, 4, 1, mu=np.full(16, np.nan))


STOKES_CASES = [(2, 4, 1, 0, None), (2, 4, 2, 1, None), (2, 8, 2, 0, "circle"), (2, 6, 2, 1, "circle"),
                (3, 2, 1, 0, None), (3, 4, 1, 1, None)]


@pytest.mark.parametrize("d,n,p,gamma,mu_kind", STOKES_CASES)
def test_host_stokes_operators_match_oracle(lib, d, n, p, gamma, mu_kind):
    """Sec. 3.1 assembly and per-field coarsening: every level of the library's
    Stokes hierarchy equals the oracle's, entry by entry and block pattern."""
    from oracle import stokes as st
    mu = circle_mu(d, n, seed=2, mu_in=1e3) if mu_kind else None
    H = lib.HostHierarchy(d, n, p, mu, stokes=gamma, smoother="jacobi")
    levels = st.build_stokes_levels(d, n, p, mu, gamma=gamma)
    assert H.nlevels == len(levels)
    for l, lv in enumerate(levels):
        rp, col, vals = H.export(l, lib.MAT_A)
        assert vals.shape[1] == (d + 1) * (p + 1) ** d
        A = _dense(rp, col, vals)
        Ao = lv.A.dense()
        scale = np.abs(Ao).max()
        assert np.abs(A - Ao).max() <= 1e-12 * scale, (l, np.abs(A - Ao).max() / scale)
        assert np.array_equal(_pattern(rp, col, lv.op.N), lv.A.pat.toarray().astype(bool))


@pytest.mark.parametrize("d,n,p,gamma,mu_kind", [(2, 8, 2, 0, None), (2, 4, 2, 1, None), (2, 8, 1, 1, "circle"),
                                                 (3, 4, 1, 0, None)])
def test_host_stokes_sai_matches_oracle(lib, d, n, p, gamma, mu_kind):
    """Balanced Stokes SAI (Sec. 3.3, zeta of Table tab:zeta) equals the oracle's."""
    from oracle import stokes as st
    mu = circle_mu(d, n, seed=1, mu_in=1e3) if mu_kind else None
    H = lib.HostHierarchy(d, n, p, mu, stokes=gamma, smoother="sai")
    levels = st.build_stokes_levels(d, n, p, mu, gamma=gamma)
    zeta = st.ZETA[(gamma, d)][p - 1]
    for l, lv in enumerate(levels[:-1]):
        alpha = st.stokes_alpha(lv.A, d, lv.op.bs, zeta)
        sai = mg.SAI(lv.A, 1, alpha=alpha)
        Bo = sai.B.dense()
        rp, col, vals = H.export(l, lib.MAT_B)
        B = _dense(rp, col, vals)
        scale = np.abs(Bo).max()
        assert np.abs(B - Bo).max() <= 1e-9 * scale, (l, np.abs(B - Bo).max() / scale)
        assert np.array_equal(_pattern(rp, col, lv.op.N), sai.B.pat.toarray().astype(bool))
        rpt, colt, valst = H.export(l, lib.MAT_BT)
        assert np.array_equal(_dense(rpt, colt, valst), B.T)


def test_host_stokes_jacobi_blocks_match_oracle(lib):
    from oracle import stokes as st
    H = lib.HostHierarchy(2, 8, 2, None, stokes=1, smoother="jacobi")
    levels = st.build_stokes_levels(2, 8, 2, gamma=1)
    for l, lv in enumerate(levels[:-1]):
        jac = mg.Jacobi(lv.A)
        _, _, vals = H.export(l, lib.MAT_D)
        for i in range(lv.op.N):
            ref = jac.Dinv[i]
            assert np.abs(vals[i] - ref).max() <= 1e-9 * np.abs(ref).max()


def test_host_stokes_rejects_bad_arguments(lib):
    with pytest.raises(lib.LdgmgError):
        lib.HostHierarchy(2, 4, 1, stokes=2)
    with pytest.raises(lib.LdgmgError):
        lib.HostHierarchy(2, 4, 1, stokes=0, taup=-1.0)


@pytest.mark.parametrize("d,n,p,stokes", [(2, 8, 2, None), (3, 4, 1, None), (2, 8, 1, 1), (2, 8, 2, 0)])
def test_host_gauss_seidel_colours_and_blocks_match_oracle(lib, d, n, p, stokes):
    """Sec. 2.3.2: the library's greedy colouring and inverse blocks equal the oracle's."""
    from oracle import stokes as st
    if stokes is None:
        levels = mg.build_levels(d, n, p)
    else:
        levels = st.build_stokes_levels(d, n, p, gamma=stokes)
    H = lib.HostHierarchy(d, n, p, stokes=stokes, smoother="gs")
    for l, lv in enumerate(levels[:-1]):
        gs = mg.GaussSeidel(lv.A)
        col, nc = H.colours(l)
        assert nc == gs.ncolours and np.array_equal(col, gs.colour)
        _, _, vals = H.export(l, lib.MAT_D)
        for i in range(lv.A.nblocks):
            assert np.abs(vals[i] - gs.Dinv[i]).max() <= 1e-9 * np.abs(gs.Dinv[i]).max()
