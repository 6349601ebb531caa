"""Pins of the Stokes oracle (oracle/stokes.py) against what the paper and the
mathematics fix: Table tab:sizes, the five-step construction of Sec. 3.1, the
kernel of the periodic problem, operator coarsening, the balancing norms of
Sec. 3.3, convergence order on a manufactured solution, GMRES's minimal-
residual property, V-cycle symmetry and the multigrid speed eta of Sec. 3.4."""
import json
import os

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import krylov, ldg
from oracle import multigrid as mg
from oracle import stokes as st


def _golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "tab_sizes.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("d,n,ell", [(2, 8, 0), (2, 8, 1), (2, 8, 2), (3, 5, 0), (3, 5, 1), (3, 7, 2)])
def test_stokes_sai_stencil_sizes_match_table(gamma, d, n, ell):
    g = _golden()["stokes_standard" if gamma == 0 else "stokes_stress"][str(d)]
    op = st.assemble_stokes(d, n, 1, gamma=gamma)
    A = op.A
    assert A.b == (d + 1) * 2 ** d                          # block dimension column of the table
    Pc = mg.pattern_power(A.pat, ell).tocsc()
    Ac = A.pat.tocsc()
    for i in (0, A.nblocks // 2, A.nblocks - 1):
        S, R = mg.sai_sets(A, ell, i, Pc, Ac)
        assert [len(R), len(S)] == g["stencil"][str(ell)]
        assert len(A.row_pattern(i)) + len(S) == g["cost"][str(ell)]


def _five_step_apply(op: st.StokesOperator, x: np.ndarray) -> np.ndarray:
    """A x by the construction of Sec. 3.1: tau = grad u + gamma grad u^T,
    sigma = L2 projection of mu tau minus p I, momentum = adjoint of the
    discrete gradient applied to sigma (plus the velocity penalty), continuity =
    minus the mass-weighted discrete divergence (minus the pressure penalty)."""
    s, d, bs, nf, N = op.scal, op.d, op.bs, op.nf, op.N
    X = x.reshape(N, nf, bs)
    u = [X[:, f, :].reshape(-1) for f in range(d)]
    p = X[:, d, :].reshape(-1)
    Minv = spla.splu(sp.csc_matrix(s.M.mat))
    out = np.zeros_like(X)
    for i in range(d):
        acc = s.E.mat @ u[i]
        for k in range(d):
            tau = s.G[k].mat @ u[i] + op.gamma * (s.G[i].mat @ u[k])
            sigma = Minv.solve(s.Mmu.mat @ tau) - (p if i == k else 0.0)
            acc = acc + s.G[k].mat.T @ (s.M.mat @ sigma)
        out[:, i, :] = acc.reshape(N, bs)
    div = sum(s.G[j].mat @ u[j] for j in range(d))
    out[:, d, :] = (-(s.M.mat @ div) - op.Ep.mat @ p).reshape(N, bs)
    return out.reshape(-1)


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("d,n,p,contrast", [(2, 6, 2, 1.0), (2, 6, 1, 1e3), (3, 4, 1, 1e-2)])
def test_components_equal_five_step_construction(gamma, d, n, p, contrast):
    """Eq. components (assembled) == the five-step construction of Sec. 3.1 on
    random vectors; a transposed G in the stress term or a flipped sign fails."""
    mesh = ldg.Mesh(d, n)
    rng = np.random.default_rng(3)
    mu = np.where(rng.random(mesh.N) < 0.3, contrast, 1.0)
    op = st.assemble_stokes(d, n, p, mu, gamma=gamma)
    for seed in range(3):
        x = np.random.default_rng(seed).standard_normal(op.A.mat.shape[0])
        ref = _five_step_apply(op, x)
        got = op.A.mat @ x
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("d,n,p", [(2, 4, 1), (2, 4, 2), (3, 3, 1)])
def test_symmetric_indefinite_with_translation_kernel(gamma, d, n, p):
    """Sec. 3.1/3.4: A is symmetric indefinite; on the periodic grid its kernel is
    exactly the constant velocities and the constant pressure (d + 1 modes)."""
    op = st.assemble_stokes(d, n, p, gamma=gamma)
    A = op.A.dense()
    s = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-15 * s
    K = st.kernel_basis(d, p, op.N)
    assert np.abs(A @ K).max() <= 1e-12 * s
    lam = np.linalg.eigvalsh(A)
    tol = 1e-10 * np.abs(lam).max()
    assert int(np.sum(np.abs(lam) < tol)) == d + 1
    assert lam[0] < -tol and lam[-1] > tol
    # velocity-velocity diagonal blocks of the standard form are the scalar LDG operator
    if gamma == 0:
        nf, bs = op.nf, op.bs
        idx = lambda f: (np.arange(op.N)[:, None] * nf * bs + f * bs + np.arange(bs)[None, :]).ravel()
        for f in range(d):
            assert np.abs(A[np.ix_(idx(f), idx(f))] - op.scal.A.dense()).max() <= 1e-13 * s
        assert np.abs(A[np.ix_(idx(d), idx(d))] + op.Ep.dense()).max() <= 1e-13 * s


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("d,n,p", [(2, 8, 2), (3, 4, 1)])
def test_stokes_coarsening_equals_rediscretisation(gamma, d, n, p):
    """Sec. 2.2 / 3.4: per-field operator coarsening (E_c = E/2 for tau ~ 1/h,
    E_p,c = 2 E_p for tau_p ~ h) reproduces the operator assembled on the coarse grid."""
    levels = st.build_stokes_levels(d, n, p, gamma=gamma)
    assert [lv.n for lv in levels] == [n >> k for k in range(len(levels))]
    for lv in levels[1:]:
        direct = st.assemble_stokes(d, lv.n, p, gamma=gamma).A
        Ac, Ad = lv.A.dense(), direct.dense()
        assert np.abs(Ac - Ad).max() <= 1e-12 * np.abs(Ad).max()
        assert (lv.A.pat != direct.pat).nnz == 0


@pytest.mark.parametrize("gamma,d,p", [(0, 2, 2), (1, 2, 2), (0, 2, 3), (1, 2, 3), (0, 3, 2), (1, 3, 2)])
def test_balancing_norms(gamma, d, p):
    """Sec. 3.3: after diag(alpha) A diag(alpha) the viscous diagonal sub-block has
    unit Frobenius norm and both coupling sub-blocks have norm zeta; the
    pressure-penalty sub-block lands between 0.2 zeta and 0.7 zeta."""
    zeta = st.ZETA[(gamma, d)][p - 1]
    mesh = ldg.Mesh(d, 4)
    for mu in (np.ones(mesh.N), np.where(np.arange(mesh.N) % 3 == 0, 1e3, 1.0)):
        op = st.assemble_stokes(d, 4, p, mu, gamma=gamma)
        bs, nf = op.bs, op.nf
        alpha = st.stokes_alpha(op.A, d, bs, zeta)
        u, q = slice(0, d * bs), slice(d * bs, nf * bs)
        for i in range(op.N):
            a = alpha[i * nf * bs:(i + 1) * nf * bs]
            D = a[:, None] * op.A.block(i, i) * a[None, :]
            assert abs(np.linalg.norm(D[u, u]) - 1.0) < 1e-12
            assert abs(np.linalg.norm(D[q, u]) - zeta) < 1e-12 * zeta
            assert abs(np.linalg.norm(D[u, q]) - zeta) < 1e-12 * zeta
            if mu.max() == mu.min():
                assert 0.2 <= np.linalg.norm(D[q, q]) / zeta <= 0.7


def _stokes_manufactured(n, p, gamma):
    """2D, mu = 1: u1 = sin kx sin ky, u2 = sin kx cos ky (not divergence free,
    so the stress term acts), p = cos kx cos ky / 2, k = 2 pi; data
    f = -lap u - gamma grad(div u) + grad p and g = div u (b_p = -M g)."""
    k = 2 * np.pi
    S, C = np.sin, np.cos
    u1 = lambda x, y: S(k * x) * S(k * y)
    u2 = lambda x, y: S(k * x) * C(k * y)
    pr = lambda x, y: 0.5 * C(k * x) * C(k * y)
    div = lambda x, y: k * C(k * x) * S(k * y) - k * S(k * x) * S(k * y)
    gdiv = (lambda x, y: -k * k * S(k * x) * S(k * y) - k * k * C(k * x) * S(k * y),
            lambda x, y: k * k * C(k * x) * C(k * y) - k * k * S(k * x) * C(k * y))
    gp = (lambda x, y: -0.5 * k * S(k * x) * C(k * y), lambda x, y: -0.5 * k * C(k * x) * S(k * y))
    f1 = lambda x, y: 2 * k * k * u1(x, y) - gamma * gdiv[0](x, y) + gp[0](x, y)
    f2 = lambda x, y: 2 * k * k * u2(x, y) - gamma * gdiv[1](x, y) + gp[1](x, y)
    d = 2
    op = st.assemble_stokes(d, n, p, gamma=gamma)
    N, bs, nf = op.N, op.bs, op.nf
    rhs = np.zeros((N, nf, bs))
    rhs[:, 0, :] = ldg.l2_project(f1, d, n, p).reshape(N, bs)
    rhs[:, 1, :] = ldg.l2_project(f2, d, n, p).reshape(N, bs)
    rhs[:, 2, :] = -ldg.l2_project(div, d, n, p).reshape(N, bs)
    b = st.project_out_kernel(rhs.reshape(-1), d, p, N)
    K = sp.csr_matrix(st.kernel_basis(d, p, N))              # disjoint supports: orthogonal columns
    bordered = sp.bmat([[op.A.mat, K], [K.T, None]], format="csc")
    x = spla.spsolve(bordered, np.concatenate([b, np.zeros(nf)]))[:-nf].reshape(N, nf, bs)
    xg, wg = npleg.leggauss(p + 3)
    W = np.multiply.outer(wg, wg).reshape(-1) * (op.h / 2) ** 2
    mesh = ldg.Mesh(d, n)
    errs = []
    for f, ex in enumerate((u1, u2, pr)):
        vals = ldg.evaluate(x[:, f, :].reshape(-1), d, n, p, xg)
        e2 = 0.0
        for e in range(N):
            c = mesh.coords(e)
            pts = [(c[a] + 0.5) * op.h + (op.h / 2) * xg for a in range(d)]
            g = np.meshgrid(*pts, indexing="ij")
            e2 += np.sum(W * (vals[e] - ex(*g).reshape(-1)) ** 2)
        errs.append(np.sqrt(e2))
    return np.hypot(errs[0], errs[1]), errs[2]


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("p,ns", [(1, (4, 8, 16)), (2, (4, 8, 16))])
def test_stokes_manufactured_convergence(gamma, p, ns):
    """Sec. 3.1: order p + 1 in velocity and at least order p in pressure."""
    res = [_stokes_manufactured(n, p, gamma) for n in ns]
    ru = np.log2(res[-2][0] / res[-1][0])
    rp = np.log2(res[-2][1] / res[-1][1])
    assert ru >= p + 1 - 0.25, res
    assert rp >= p - 0.25, res


def test_gmres_minimal_residual_and_exact_termination():
    """GMRES minimises ||V(b - A x)|| over the Krylov space K_k(VA, Vb) (checked by
    brute-force least squares) and terminates at the solution in <= n steps."""
    rng = np.random.default_rng(11)
    n = 24
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    Vm = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    V = lambda v: Vm @ v
    b = rng.standard_normal(n)
    Vb = Vm @ b
    VA = Vm @ A
    for k in range(1, 7):
        x, it, hist = st.gmres(A, V, b, tol=0.0, restart=50, max_iter=k)
        assert it == k
        Kb = np.empty((n, k))
        v = Vb.copy()
        for j in range(k):
            Kb[:, j] = v
            v = VA @ v
        Qk, _ = np.linalg.qr(Kb)
        y, *_ = np.linalg.lstsq(VA @ Qk, Vb, rcond=None)
        best = np.linalg.norm(Vb - VA @ (Qk @ y))
        got = np.linalg.norm(Vm @ (b - A @ x))
        assert abs(got - best) <= 1e-10 * np.linalg.norm(Vb)
        assert abs(hist[-1] - got) <= 1e-10 * np.linalg.norm(Vb)
        assert all(hist[i + 1] <= hist[i] * (1 + 1e-14) for i in range(len(hist) - 1))
    x, it, hist = st.gmres(A, V, b, tol=1e-12, restart=50, max_iter=200)
    assert it <= n
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(np.linalg.solve(A, b))


def test_gmres_restarted_converges_and_is_monotone():
    rng = np.random.default_rng(5)
    n = 40
    A = rng.standard_normal((n, n)) + 9 * np.eye(n)
    b = rng.standard_normal(n)
    x, it, hist = st.gmres(A, lambda v: v, b, tol=1e-10, restart=5, max_iter=400)
    assert np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


@pytest.mark.parametrize("gamma", [0, 1])
def test_stokes_vcycle_symmetric(gamma):
    """Sec. 3.4: with B1 pre- and BT post-smoothing V is symmetric (indefinite)."""
    levels = st.build_stokes_levels(2, 4, 1, gamma=gamma)
    V = st.StokesVCycle(levels, "sai", 3, 3, zeta=st.ZETA[(gamma, 2)][0])
    n = levels[0].A.mat.shape[0]
    Vd = np.column_stack([V(e) for e in np.eye(n)])
    assert np.abs(Vd - Vd.T).max() <= 1e-10 * np.abs(Vd).max()


@pytest.mark.parametrize("gamma", [0, 1])
def test_stokes_sai1_gmres_speed(gamma):
    """Sec. 3.4.1/3.4.2: SAI1 (B1 pre, BT post) with GMRES reaches eta ~ 0.6 for
    d = p = 2 in both forms; the oracle's readings land in [0.4, 0.8]."""
    levels = st.build_stokes_levels(2, 8, 2, gamma=gamma)
    V = st.StokesVCycle(levels, "sai", 3, 3, zeta=st.ZETA[(gamma, 2)][1])
    A = levels[0].A
    b = st.project_out_kernel(np.random.default_rng(0).standard_normal(A.mat.shape[0]), 2, 2, A.nblocks)
    x, it, hist = st.gmres(A.mat, V, b, tol=1e-10, max_iter=60)
    assert 0.4 <= krylov.eta(hist) <= 0.8, (it, krylov.eta(hist))
    assert np.linalg.norm(b - A.mat @ x) <= 1e-7 * np.linalg.norm(b)


def test_fgmres_minimal_true_residual_over_preconditioned_space():
    """FGMRES with a fixed linear V minimises ||b - A x|| over V K_k(A V, b)
    (brute-force least squares) and reaches the solution."""
    rng = np.random.default_rng(12)
    n = 24
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    Vm = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    AV = A @ Vm
    for k in range(1, 7):
        x, it, hist = st.fgmres(A, lambda v: Vm @ v, b, tol=0.0, restart=50, max_iter=k)
        Kb = np.empty((n, k))
        v = b.copy()
        for j in range(k):
            Kb[:, j] = v
            v = AV @ v
        Qk, _ = np.linalg.qr(Kb)
        y, *_ = np.linalg.lstsq(AV @ Qk, b, rcond=None)
        best = np.linalg.norm(b - AV @ (Qk @ y))
        got = np.linalg.norm(b - A @ x)
        assert abs(got - best) <= 1e-10 * np.linalg.norm(b)
        assert abs(hist[-1] - got) <= 1e-10 * np.linalg.norm(b)
    # restarted: converges when A V has its field of values in the right half plane
    A2 = rng.standard_normal((n, n)) + 12 * np.eye(n)
    V2 = np.eye(n) + 0.05 * rng.standard_normal((n, n))
    x, it, hist = st.fgmres(A2, lambda v: V2 @ v, b, tol=1e-12, restart=5, max_iter=400)
    assert np.linalg.norm(b - A2 @ x) <= 1e-11 * np.linalg.norm(b)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    # with V = I both variants are plain GMRES and agree
    x1, k1, h1 = st.gmres(A, lambda v: v, b, tol=1e-10, restart=50)
    x2, k2, h2 = st.fgmres(A, lambda v: v, b, tol=1e-10, restart=50)
    assert k1 == k2 and np.allclose(h1, h2, rtol=1e-10, atol=0)


def test_stokes_gauss_seidel_vs_sai1():
    """Sec. 3.4.1/3.4.2: multi-coloured GS with same-order sweeps and GMRES is an
    effective Stokes solver (paper: eta ~ 0.9 standard, ~1 stress at d = p = 2)
    and SAI1 (B1 pre, BT post) is faster than it in both forms."""
    for gamma in (0, 1):
        levels = st.build_stokes_levels(2, 8, 2, gamma=gamma)
        A = levels[0].A
        b = st.project_out_kernel(np.random.default_rng(0).standard_normal(A.mat.shape[0]), 2, 2, A.nblocks)
        col = mg.greedy_colouring(A.pat)
        Pat = A.pat.tocoo()
        assert all(col[i] != col[j] for i, j in zip(Pat.row, Pat.col) if i != j)
        assert col.max() + 1 == (2 if gamma == 0 else 4)
        _, _, h_gs = st.gmres(A.mat, st.StokesVCycle(levels, "gs", 3, 3, pre="B1", post="B1"), b, tol=1e-10,
                              max_iter=60)
        _, _, h_sai = st.gmres(A.mat, st.StokesVCycle(levels, "sai", 3, 3, zeta=st.ZETA[(gamma, 2)][1]), b,
                               tol=1e-10, max_iter=60)
        eta_gs, eta_sai = krylov.eta(h_gs), krylov.eta(h_sai)
        assert 0.5 <= eta_gs <= 1.2, eta_gs
        assert eta_sai < eta_gs, (eta_sai, eta_gs)


@pytest.mark.parametrize("gamma", [0, 1])
@pytest.mark.parametrize("mu_in,mu_out", [(1e3, 1.0), (1.0, 1e3)])
def test_stokes_coarsening_equals_rediscretisation_across_aligned_jump(gamma, mu_in, mu_out):
    """As the scalar case: with the viscosity inclusion (1/4, 3/4)^2 of Sec. 3.4.3
    aligned with every level with n >= 4, per-field coarsening (M_mu,c, E_c = E/2,
    E_p,c = 2 E_p with its min-mu weight) equals the Stokes operator assembled
    on the coarse mesh with the coarse viscosities."""
    from paper_2412_12506_gb300.inputs import square_mu
    d, n, p = 2, 16, 2
    levels = st.build_stokes_levels(d, n, p, square_mu(d, n, mu_in, mu_out), gamma=gamma)
    for lv in levels[1:]:
        if lv.n < 4:
            continue
        direct = st.assemble_stokes(d, lv.n, p, square_mu(d, lv.n, mu_in, mu_out), gamma=gamma).A
        Ac, Ad = lv.A.dense(), direct.dense()
        assert np.abs(Ac - Ad).max() <= 1e-12 * np.abs(Ad).max()
        assert (lv.A.pat != direct.pat).nnz == 0
