"""Pins for the oracle's hierarchy, smoothers, V-cycle and CG (Sec. 2.2-2.4).

Checks against: the coarse operator assembled directly (Sec. 2.2 equivalence
claim), exact identities (R I = Id), Table tab:sizes (golden fixture), the
normal equations and an independent SVD least-squares solve, dense linear
algebra on tiny meshes, the symmetry the paper states for the B1/BT pairing
(Sec. 2.4), and exact-arithmetic properties of CG.
"""
import json
import os

import numpy as np
import pytest

from oracle import krylov, ldg
from oracle import multigrid as mg
from paper_2412_12506_gb300.inputs import circle_mu, square_mu


# ----------------------------------------------------------------------------
# transfer operators and operator coarsening
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,p", [(2, 4, 2), (3, 2, 1)])
def test_restriction_of_injection_is_identity(d, n, p):
    I = mg.injection(d, n, p)
    fine = ldg.assemble(d, n, p)
    coarse = ldg.assemble(d, n // 2, p)
    R = np.linalg.inv(coarse.M.dense()) @ I.dense().T @ fine.M.dense()
    assert np.allclose(R @ I.dense(), np.eye(R.shape[0]), atol=1e-13)


@pytest.mark.parametrize("d,n,p", [(2, 8, 1), (2, 8, 3), (3, 4, 2), (2, 4, 2)])
def test_coarsening_equals_rediscretisation(d, n, p):
    """Sec. 2.2: operator coarsening and coarse re-discretisation coincide (mu == 1)."""
    levels = mg.build_levels(d, n, p)
    for lv in levels[1:]:
        direct = ldg.assemble(d, lv.n, p)
        Ac, Ad = lv.A.dense(), direct.A.dense()
        assert np.abs(Ac - Ad).max() <= 1e-12 * np.abs(Ad).max()
        assert (lv.A.pat != direct.A.pat).nnz == 0


def test_coarse_interface_operators_spsd_with_constant_kernel():
    d, n, p = 2, 8, 2
    levels = mg.build_levels(d, n, p, circle_mu(d, n, seed=2, mu_in=1e4))
    for lv in levels:
        A = lv.A.dense()
        s = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-12 * s
        lam = np.linalg.eigvalsh(A)
        assert lam[0] >= -1e-10 * lam[-1]
        c = ldg.constant_vector(d, p, lv.N)
        assert np.abs(A @ c).max() <= 1e-10 * s


def test_hierarchy_sizes():
    assert [lv.n for lv in mg.build_levels(2, 16, 1)] == [16, 8, 4, 2, 1]
    assert [lv.n for lv in mg.build_levels(2, 12, 1)] == [12, 6, 3]


# ----------------------------------------------------------------------------
# block Jacobi (Eq. Jsmooth)
# ----------------------------------------------------------------------------

def test_jacobi_inverse_blocks_and_sweep():
    d, n, p = 2, 4, 2
    A = ldg.assemble(d, n, p).A
    jac = mg.Jacobi(A, 0.8)
    b = A.b
    for i in range(A.nblocks):
        assert np.allclose(jac.Dinv[i] @ A.block(i, i), np.eye(b), atol=1e-12)
    rng = np.random.default_rng(0)
    x, rhs = rng.standard_normal(A.mat.shape[0]), rng.standard_normal(A.mat.shape[0])
    # the same update written as x + w D^{-1} (b - A x)
    Dinv = np.zeros((A.mat.shape[0],) * 2)
    for i in range(A.nblocks):
        Dinv[i * b:(i + 1) * b, i * b:(i + 1) * b] = np.linalg.inv(A.block(i, i))
    ref = x + 0.8 * Dinv @ (rhs - A.dense() @ x)
    assert np.allclose(jac.sweep(x, rhs), ref, atol=1e-12)


# ----------------------------------------------------------------------------
# balanced block SAI (Sec. 2.3.3)
# ----------------------------------------------------------------------------

def _golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "tab_sizes.json")) as f:
        return json.load(f)["poisson"]


@pytest.mark.parametrize("d,n,ell", [(2, 8, 0), (2, 8, 1), (2, 8, 2), (3, 5, 0), (3, 5, 1),
                                     (3, 7, 2)])
def test_sai_stencil_sizes_match_table(d, n, ell):
    g = _golden()[str(d)]
    A = ldg.assemble(d, n, 1).A
    Pc = mg.pattern_power(A.pat, ell).tocsc()
    Ac = A.pat.tocsc()
    for i in (0, A.nblocks // 2, A.nblocks - 1):
        S, R = mg.sai_sets(A, ell, i, Pc, Ac)
        assert [len(R), len(S)] == g["stencil"][str(ell)]
        assert len(A.row_pattern(i)) + len(S) == g["cost"][str(ell)]


@pytest.mark.parametrize("mu_kind", ["one", "circle"])
def test_sai_columns_solve_their_least_squares(mu_kind):
    d, n, p = 2, 6, 1
    mu = None if mu_kind == "one" else circle_mu(d, n, seed=1, mu_in=1e4)
    A = ldg.assemble(d, n, p, mu).A
    sai = mg.SAI(A, 1)
    b = A.b
    # balancing: every diagonal block of diag(alpha) A diag(alpha) has unit Frobenius norm
    for i in range(A.nblocks):
        blk = sai.alpha_el[i] ** 2 * A.block(i, i)
        assert abs(np.linalg.norm(blk, "fro") - 1.0) < 1e-12
    At = np.diag(sai.alpha) @ A.dense() @ np.diag(sai.alpha)
    Bt = np.diag(1 / sai.alpha) @ sai.B.dense() @ np.diag(1 / sai.alpha)
    for i in (0, 7, A.nblocks - 1):
        S, R = mg.sai_sets(A, 1, i)
        rows = np.concatenate([np.arange(r * b, (r + 1) * b) for r in R])
        cols = np.concatenate([np.arange(k * b, (k + 1) * b) for k in S])
        M = At[np.ix_(rows, cols)]
        E = np.eye(A.mat.shape[0])[np.ix_(rows, np.arange(i * b, (i + 1) * b))]
        X = Bt[np.ix_(cols, np.arange(i * b, (i + 1) * b))]
        # normal equations of the least-squares problem
        assert np.abs(M.T @ (M @ X - E)).max() < 1e-11
        # independent SVD-based solve
        Xs = np.linalg.lstsq(M, E, rcond=None)[0]
        assert np.allclose(X, Xs, atol=1e-10)
        # B has no entries outside S(i) in column i
        others = np.setdiff1d(np.arange(A.mat.shape[0]), cols)
        assert np.abs(Bt[np.ix_(others, np.arange(i * b, (i + 1) * b))]).max() == 0.0


def test_sai_balancing_is_neutral_for_constant_mu_and_translation_invariant():
    d, n, p = 2, 6, 2
    A = ldg.assemble(d, n, p).A
    B1 = mg.SAI(A, 1, balance=True).B.dense()
    B0 = mg.SAI(A, 1, balance=False).B.dense()
    assert np.abs(B1 - B0).max() <= 1e-10 * np.abs(B0).max()
    sai = mg.SAI(A, 1)
    ref = sai.column(0)
    mesh = ldg.Mesh(d, n)
    for i in (5, 14, 35):
        ci = mesh.coords(i)
        col = sai.column(i)
        for (k, _), blk in ref.items():
            ck = mesh.coords(k)
            shifted = mesh.index(tuple(ck[a] + ci[a] for a in range(d)))
            assert np.allclose(col[(shifted, i)], blk, atol=1e-11)


# ----------------------------------------------------------------------------
# V-cycle (Algorithm 1) and bottom solve
# ----------------------------------------------------------------------------

def _dense_V(V, size):
    return np.column_stack([V(e) for e in np.eye(size)])


@pytest.mark.parametrize("smoother,pre,post,sym", [("jacobi", "B1", "B1", True),
                                                   ("sai", "B1", "BT", True),
                                                   ("sai", "BT", "B1", True),
                                                   ("sai", "B1", "B1", False)])
def test_vcycle_symmetry(smoother, pre, post, sym):
    """Sec. 2.4: Jacobi and opposite SAI forms give a symmetric V; equal forms do not."""
    d, n, p = 2, 4, 1
    levels = mg.build_levels(d, n, p)
    V = mg.VCycle(levels, smoother, 2, 2, pre=pre, post=post)
    Vd = _dense_V(V, levels[0].A.mat.shape[0])
    asym = np.abs(Vd - Vd.T).max() / np.abs(Vd).max()
    if sym:
        assert asym < 1e-12
        # positive semi-definite on the range of A
        c = ldg.constant_vector(d, p, levels[0].N)
        P = np.eye(len(c)) - np.outer(c, c) / (c @ c)
        lam = np.linalg.eigvalsh(P @ Vd @ P)
        assert lam[0] > -1e-12 * lam[-1]
    else:
        assert asym > 1e-6


def test_single_level_vcycle_is_pseudo_inverse():
    levels = mg.build_levels(2, 3, 2)           # odd n: the finest level is the bottom
    assert len(levels) == 1
    V = mg.VCycle(levels, "jacobi")
    Vd = _dense_V(V, levels[0].A.mat.shape[0])
    assert np.allclose(Vd, np.linalg.pinv(levels[0].A.dense(), rcond=1e-12), atol=1e-10)


@pytest.mark.parametrize("smoother", ["jacobi", "sai"])
def test_two_level_error_propagation(smoother):
    """x_out = V b from x0 = 0 with 1 pre- and 1 post-sweep, written out densely."""
    d, n, p = 2, 6, 1                            # 6 -> 3: two levels
    levels = mg.build_levels(d, n, p)
    assert [lv.n for lv in levels] == [6, 3]
    V = mg.VCycle(levels, smoother, 1, 1, omega=0.8)
    A = levels[0].A.dense()
    I = levels[0].I.dense()
    Ac_pinv = np.linalg.pinv(levels[1].A.dense(), rcond=1e-12)
    size = A.shape[0]
    if smoother == "jacobi":
        Dinv = np.zeros_like(A)
        b = levels[0].b
        for i in range(levels[0].N):
            sl = slice(i * b, (i + 1) * b)
            Dinv[sl, sl] = np.linalg.inv(A[sl, sl])
        Spre = Spost = 0.8 * Dinv                # x <- x + S (b - A x)
    else:
        Bd = levels[0].smoother.B.dense()
        Spre, Spost = Bd, Bd.T
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal(size)
    x = Spre @ rhs
    x = x + I @ (Ac_pinv @ (I.T @ (rhs - A @ x)))
    x = x + Spost @ (rhs - A @ x)
    assert np.allclose(V(rhs), x, atol=1e-11 * np.abs(x).max())


# ----------------------------------------------------------------------------
# CG and eta
# ----------------------------------------------------------------------------

def test_cg_exact_arithmetic_property():
    """Unpreconditioned CG on a matrix with m distinct eigenvalues stops in m steps."""
    A = np.diag(np.repeat([1.0, 2.0, 5.0, 9.0], 6))
    rng = np.random.default_rng(0)
    b = rng.standard_normal(24)
    x, k, _ = krylov.pcg(A, lambda r: r.copy(), b, tol=1e-12)
    assert k == 4
    assert np.allclose(A @ x, b, atol=1e-10)
    x, k, _ = krylov.pcg(A, lambda r: r.copy(), b, tol=1e-12, flexible=True)
    assert k == 4


def test_eta_of_geometric_sequence():
    hist = [10.0 * 0.1 ** (k / 0.7) for k in range(8)]
    assert abs(krylov.eta(hist) - 0.7) < 1e-12


@pytest.mark.parametrize("smoother,nu", [("jacobi", 2), ("sai", 3)])
def test_pcg_matches_dense_solve(smoother, nu):
    d, n, p = 2, 4, 2
    levels = mg.build_levels(d, n, p)
    V = mg.VCycle(levels, smoother, nu, nu)
    A = levels[0].A
    rhs = ldg.project_out_constant(np.random.default_rng(7).standard_normal(A.mat.shape[0]), d, p, A.nblocks)
    x, k, _ = krylov.pcg(A.mat, V, rhs, tol=1e-12)
    xd = np.linalg.pinv(A.dense(), rcond=1e-12) @ rhs
    x = ldg.project_out_constant(x, d, p, A.nblocks)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_sai_fwd_rev_is_fast_and_mesh_independent():
    """Sec. 2.4.1 (vi) and the abstract: good combinations need about 4-8
    iterations per 1e10 residual reduction, independently of the mesh size;
    BT pre / B1 post is the bad pairing (Sec. 2.4.1, second bullet)."""
    d, p = 2, 2
    iters = []
    for n in (8, 16, 32):
        levels = mg.build_levels(d, n, p)
        V = mg.VCycle(levels, "sai", 3, 3)
        A = levels[0].A
        rhs = ldg.project_out_constant(np.random.default_rng(n).standard_normal(A.mat.shape[0]),
                                       d, p, A.nblocks)
        _, k, _ = krylov.pcg(A.mat, V, rhs)
        iters.append(k)
    assert max(iters) - min(iters) <= 1
    assert 4 <= min(iters) and max(iters) <= 8
    levels = mg.build_levels(d, 16, p)
    Vbad = mg.VCycle(levels, "sai", 3, 3, pre="BT", post="B1")
    A = levels[0].A
    rhs = ldg.project_out_constant(np.random.default_rng(16).standard_normal(A.mat.shape[0]), d, p, A.nblocks)
    _, kbad, _ = krylov.pcg(A.mat, Vbad, rhs)
    assert kbad > iters[1]


def test_interface_contrast_independence():
    """Sec. 2.4.3: on the inclusion (1/4, 3/4)^d the iteration counts are
    essentially the same for viscosity ratios 1e-4 ... 1e4 (and as for mu == 1)."""
    d, n, p = 2, 16, 1
    ks = []
    for contrast in (1.0, 1e2, 1e4, 1e-4):
        mu = square_mu(d, n, mu_in=contrast)
        levels = mg.build_levels(d, n, p, mu)
        V = mg.VCycle(levels, "sai", 3, 3)
        A = levels[0].A
        rhs = ldg.project_out_constant(np.random.default_rng(1).standard_normal(A.mat.shape[0]), d, p, A.nblocks)
        _, k, _ = krylov.pcg(A.mat, V, rhs)
        ks.append(k)
    assert max(ks) - min(ks) <= 2 and max(ks) <= 12, ks


# ---------------------------------------------------------------------------
# multi-coloured block Gauss-Seidel (Sec. 2.3.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,p", [(2, 8, 1), (2, 6, 2), (3, 4, 1), (2, 2, 1)])
def test_colouring_is_red_black_on_the_block_stencil(d, n, p):
    """Sec. 2.3.2: on Cartesian grids with one-sided fluxes the colouring of the
    block pattern is the red-black colouring of the 5 / 7-point stencil."""
    A = ldg.assemble(d, n, p).A
    col = mg.greedy_colouring(A.pat)
    assert col.max() == 1
    P = A.pat.tocoo()
    assert all(col[i] != col[j] for i, j in zip(P.row, P.col) if i != j)
    mesh = ldg.Mesh(d, n)
    parity = np.array([sum(mesh.coords(e)) % 2 for e in range(mesh.N)])
    assert np.array_equal(col, parity)


def _block_parts(A, order):
    """Dense A permuted to `order` (block level) and split into D, strict lower L, strict upper U."""
    b = A.b
    perm = np.concatenate([np.arange(i * b, (i + 1) * b) for i in order])
    Ad = A.dense()[np.ix_(perm, perm)]
    N = len(order)
    D = np.zeros_like(Ad)
    L = np.zeros_like(Ad)
    for I in range(N):
        for J in range(N):
            blk = Ad[I * b:(I + 1) * b, J * b:(J + 1) * b]
            if I == J:
                D[I * b:(I + 1) * b, J * b:(J + 1) * b] = blk
            elif J < I:
                L[I * b:(I + 1) * b, J * b:(J + 1) * b] = blk
    return perm, D, L, Ad - D - L


@pytest.mark.parametrize("mu_kind", [None, "circle"])
def test_gauss_seidel_sweep_is_block_triangular_solve(mu_kind):
    """A forward multi-coloured sweep equals textbook block Gauss-Seidel in the
    colour-sorted element order, x' = (D + L)^{-1} (b - U x); the backward sweep
    equals (D + U)^{-1} (b - L x) (Sec. 2.3.2, Sec. 2.4 pairings)."""
    d, n, p = 2, 6, 2
    mu = None if mu_kind is None else circle_mu(d, n, seed=1, mu_in=1e3)
    A = ldg.assemble(d, n, p, mu).A
    gs = mg.GaussSeidel(A)
    order = np.argsort(gs.colour, kind="stable")
    perm, D, L, U = _block_parts(A, order)
    rng = np.random.default_rng(0)
    x, rhs = rng.standard_normal(A.mat.shape[0]), rng.standard_normal(A.mat.shape[0])
    fwd = np.empty_like(x)
    fwd[perm] = np.linalg.solve(D + L, rhs[perm] - U @ x[perm])
    bwd = np.empty_like(x)
    bwd[perm] = np.linalg.solve(D + U, rhs[perm] - L @ x[perm])
    assert np.abs(gs.sweep(x, rhs, "B1") - fwd).max() <= 1e-11 * np.abs(fwd).max()
    assert np.abs(gs.sweep(x, rhs, "BT") - bwd).max() <= 1e-11 * np.abs(bwd).max()


def test_gauss_seidel_vcycle_symmetry_and_pairing_speed():
    """Forward pre / backward post gives a symmetric V-cycle (CG-usable); the
    forward / forward pairing is asymmetric and, with GMRES, needs fewer
    iterations (Sec. 2.4.1: GS with same-order sweeps is usually fastest)."""
    d, n, p = 2, 4, 1
    levels = mg.build_levels(d, n, p)
    sym = mg.VCycle(levels, "gs", 2, 2, pre="B1", post="BT")
    asym = mg.VCycle(levels, "gs", 2, 2, pre="B1", post="B1")
    size = levels[0].A.mat.shape[0]
    c = ldg.constant_vector(d, p, levels[0].N)
    Pc = np.eye(size) - np.outer(c, c) / (c @ c)
    Vs = Pc @ np.column_stack([sym(Pc @ e) for e in np.eye(size)])
    Va = Pc @ np.column_stack([asym(Pc @ e) for e in np.eye(size)])
    assert np.abs(Vs - Vs.T).max() <= 1e-11 * np.abs(Vs).max()
    assert np.abs(Va - Va.T).max() > 1e-3 * np.abs(Va).max()
    from oracle import stokes as st
    for d, n, p in ((2, 16, 2), (2, 16, 3)):
        levels = mg.build_levels(d, n, p)
        A = levels[0].A
        rhs = ldg.project_out_constant(np.random.default_rng(0).standard_normal(A.mat.shape[0]), d, p, A.nblocks)
        _, k_oi, _ = st.gmres(A.mat, mg.VCycle(levels, "gs", 3, 3, pre="B1", post="BT"), rhs, tol=1e-10)
        _, k_oo, _ = st.gmres(A.mat, mg.VCycle(levels, "gs", 3, 3, pre="B1", post="B1"), rhs, tol=1e-10)
        assert k_oo < k_oi, (k_oo, k_oi)


@pytest.mark.parametrize("d,n,p", [(2, 16, 2), (2, 16, 1), (3, 8, 1)])
@pytest.mark.parametrize("mu_in,mu_out", [(1e4, 1.0), (1.0, 1e4)])
def test_coarsening_equals_rediscretisation_across_aligned_jump(d, n, p, mu_in, mu_out):
    """Sec. 2.2 option (ii) with a coefficient jump.  The inclusion (1/4, 3/4)^d
    of Sec. 2.4.3 stays a union of whole elements on every level with n >= 4,
    so an injected coarse function has no jump on the fine faces inside a coarse
    element and the same upwind side on the others.  The coarsened G, M_mu and
    E are then exactly those assembled on the coarse mesh with the coarse
    element coefficients, and so is A.  Dropping mu from M_mu,c (I^T M I) or
    the 1/2 of E_c makes this fail by O(1)."""
    levels = mg.build_levels(d, n, p, square_mu(d, n, mu_in, mu_out))
    checked = 0
    for lv in levels[1:]:
        if lv.n < 4:
            continue
        direct = ldg.assemble(d, lv.n, p, square_mu(d, lv.n, mu_in, mu_out))
        Ac, Ad = lv.A.dense(), direct.A.dense()
        assert np.abs(Ac - Ad).max() <= 1e-12 * np.abs(Ad).max()
        assert (lv.A.pat != direct.A.pat).nnz == 0
        checked += 1
    assert checked == len([k for k in range(1, 8) if n >> k >= 4])
