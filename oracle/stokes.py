"""Oracle, part 4: LDG Stokes saddle-point operator (Sec. 3) and GMRES.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): never imported by the product.

The system of Eq. components / Eq. blockform, per element the d velocity
components followed by the pressure (block size (d+1)(p+1)^d):

    A_ij (velocity i, velocity j) = delta_ij (sum_k G_k^T M_mu G_k + E) + gamma G_j^T M_mu G_i
    A_i,p                         = -G_i^T M
    A_p,j                         = -M G_j
    A_p,p                         = -E_p

with G, M_mu, M and E the scalar LDG pieces of Sec. 2.1 (oracle/ldg.py) and
gamma = 0 (standard form) or 1 (stress form).

Readings (the paper defers these to [flame]):
  * E_p = sum_faces tau_p int_f [p][q] with tau_p = taup * h / min(mu_L, mu_U)
    (Sec. 3.3 states the scaling E_p ~ h^d / mu).  The paper takes its penalty
    values from [flame]; Sec. 3.3 states that after balancing the pressure-
    penalty block has Frobenius norm between 0.2 zeta and 0.7 zeta, and
    taup = 0.05 lands there for d = 2, p = 2, 3 and d = 3, p = 2 in both forms,
    so it is the default.
  * Operator coarsening per component as in the scalar case (Sec. 2.2), with
    E_p,c = 2 I^T E_p,f I (tau_p proportional to h).
  * Balanced SAI (Sec. 3.3): alpha_u = ||A_ii^uu||_F^{-1/2} on the velocity dofs,
    alpha_p = zeta ||A_ii^uu||_F^{1/2} ||A_ii^pu||_F^{-1} on the pressure dofs,
    zeta from Table tab:zeta.
  * GMRES (Sec. 2.2 / 3.4): left preconditioned (solves V A x = V b), restarted
    every `restart` steps, modified Gram-Schmidt Arnoldi and Givens rotations;
    stops when the preconditioned residual ||V (b - A x)|| <= tol ||V b||.
    The paper does not name the orthogonalisation; MGS is the reading.
  * fgmres: the flexible right-preconditioned variant for a V-cycle applied in
    reduced precision (not an exactly linear operator); stops on ||b - A x||.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import ldg
from . import multigrid as mg
from .ldg import BOp, LDGOperator, Mesh, _from_blocks

TAUP = 0.05   # pressure penalty scale (reading above)

ZETA = {  # Table tab:zeta: (gamma, d) -> zeta by p = 1..5
    (0, 2): [0.0382, 0.131, 0.0990, 0.153, 0.142],
    (0, 3): [0.0462, 0.107, 0.113],
    (1, 2): [0.118, 0.131, 0.0814, 0.123, 0.0745],
    (1, 3): [0.0384, 0.0928, 0.0930],
}


def pressure_penalty(d: int, n: int, p: int, mu, taup: float) -> BOp:
    mesh = Mesh(d, n)
    bas = ldg.Basis1D(p)
    b = (p + 1) ** d
    h = mesh.h
    w = (h / 2.0) ** (d - 1)
    blocks = {}
    for a in range(d):
        for L, U in mesh.faces(a):
            c = taup * h / min(mu[L], mu[U]) * w
            ldg._add(blocks, (L, L), c * ldg.axis_op(np.outer(bas.hi, bas.hi), a, d))
            ldg._add(blocks, (L, U), -c * ldg.axis_op(np.outer(bas.hi, bas.lo), a, d))
            ldg._add(blocks, (U, L), -c * ldg.axis_op(np.outer(bas.lo, bas.hi), a, d))
            ldg._add(blocks, (U, U), c * ldg.axis_op(np.outer(bas.lo, bas.lo), a, d))
    return _from_blocks(blocks, mesh.N, b)


class StokesOperator:
    """Scalar pieces plus the assembled saddle-point operator A (a BOp with
    block size (d+1) * bs)."""

    def __init__(self, scal: LDGOperator, Ep: BOp, gamma: int):
        self.scal, self.Ep, self.gamma = scal, Ep, gamma
        self.d, self.bs = scal.d, scal.b
        self.nf = self.d + 1
        self.b = self.nf * self.bs
        self.h = scal.h
        self.N = Ep.nblocks
        self.A = self._assemble()

    def field_selector(self, f: int) -> sp.csr_matrix:
        """P_f: scalar dof (e, m) -> Stokes dof (e, f, m)."""
        N, bs, nf = self.N, self.bs, self.nf
        rows = (np.arange(N)[:, None] * nf * bs + f * bs + np.arange(bs)[None, :]).ravel()
        cols = np.arange(N * bs)
        return sp.csr_matrix((np.ones(N * bs), (rows, cols)), shape=(N * nf * bs, N * bs))

    def _assemble(self) -> BOp:
        d, s = self.d, self.scal
        G, Mmu, M, E = s.G, s.Mmu, s.M, s.E
        lap = E
        for k in range(d):
            lap = lap + (G[k].T @ Mmu @ G[k])
        comp = {}
        for i in range(d):
            for j in range(d):
                if self.gamma:
                    blk = G[j].T @ Mmu @ G[i]
                    comp[(i, j)] = (lap + blk) if i == j else blk
                elif i == j:
                    comp[(i, j)] = lap
            comp[(i, d)] = (G[i].T @ M).scale(-1.0)
            comp[(d, i)] = (M @ G[i]).scale(-1.0)
        comp[(d, d)] = self.Ep.scale(-1.0)
        P = [self.field_selector(f) for f in range(self.nf)]
        mat = None
        pat = None
        for (f, g), op in comp.items():
            term = P[f] @ op.mat @ P[g].T
            mat = term if mat is None else mat + term
            pat = op.pat if pat is None else pat + op.pat
        return BOp(mat, pat, self.b)


def assemble_stokes(d: int, n: int, p: int, mu=None, gamma: int = 0, tau0: float = 1.0,
                    taup: float = TAUP) -> StokesOperator:
    mesh = Mesh(d, n)
    mu = np.ones(mesh.N) if mu is None else np.asarray(mu, dtype=np.float64)
    scal = ldg.assemble(d, n, p, mu, tau0)
    return StokesOperator(scal, pressure_penalty(d, n, p, mu, taup), gamma)


def stokes_injection(I: BOp, nf: int) -> BOp:
    """Each field injected like the scalar (Sec. 3.4: transfers act on the
    individual velocity and pressure components)."""
    b = I.b
    Nf, Nc = I.pat.shape
    rows, cols, vals = [], [], []
    Ic = I.mat.tocoo()
    for f in range(nf):
        ef, mf = np.divmod(Ic.row, b)
        ec, mc = np.divmod(Ic.col, b)
        rows.append(ef * nf * b + f * b + mf)
        cols.append(ec * nf * b + f * b + mc)
        vals.append(Ic.data)
    mat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(Nf * nf * b, Nc * nf * b))
    return BOp(mat, I.pat, nf * b)


def build_stokes_levels(d: int, n: int, p: int, mu=None, gamma: int = 0, tau0: float = 1.0,
                        taup: float = TAUP):
    op = assemble_stokes(d, n, p, mu, gamma, tau0, taup)
    levels = [mg.Level(n, op)]
    levels[0].A, levels[0].b = op.A, op.b
    while levels[-1].n % 2 == 0 and levels[-1].n > 1:
        f = levels[-1]
        I = mg.injection(d, f.n, p)
        f.I = stokes_injection(I, f.op.nf)
        scal_c = mg.coarsen(f.op.scal, I)
        Ep_c = (I.T @ f.op.Ep @ I).scale(2.0)
        op_c = StokesOperator(scal_c, Ep_c, gamma)
        lv = mg.Level(f.n // 2, op_c)
        lv.A, lv.b = op_c.A, op_c.b
        levels.append(lv)
    return levels


def stokes_alpha(A: BOp, d: int, bs: int, zeta: float) -> np.ndarray:
    """Per-dof balancing of Sec. 3.3 (alpha_u on velocity dofs, alpha_p on pressure)."""
    nf = d + 1
    N = A.nblocks
    alpha = np.empty(N * nf * bs)
    for i in range(N):
        D = A.block(i, i)
        Auu = D[:d * bs, :d * bs]
        Dpu = D[d * bs:, :d * bs]
        nA = np.linalg.norm(Auu, "fro")
        au = nA ** -0.5
        ap = zeta * nA ** 0.5 / np.linalg.norm(Dpu, "fro")
        alpha[i * nf * bs:i * nf * bs + d * bs] = au
        alpha[i * nf * bs + d * bs:(i + 1) * nf * bs] = ap
    return alpha


def kernel_basis(d: int, p: int, N: int) -> np.ndarray:
    """Constant velocity components and constant pressure: (N*(d+1)*bs, d+1)."""
    bs = (p + 1) ** d
    nf = d + 1
    K = np.zeros((N * nf * bs, nf))
    for f in range(nf):
        K[np.arange(N) * nf * bs + f * bs, f] = np.sqrt(2.0) ** d
    return K


def project_out_kernel(v: np.ndarray, d: int, p: int, N: int) -> np.ndarray:
    K = kernel_basis(d, p, N)
    return v - K @ np.linalg.solve(K.T @ K, K.T @ v)


class StokesVCycle(mg.VCycle):
    """Algorithm 1 on the Stokes hierarchy; SAI balanced per Sec. 3.3."""

    def __init__(self, levels, smoother="sai", nu1=3, nu2=3, omega=0.8, ell=1, pre="B1", post="BT",
                 zeta=0.131):
        self.levels = levels
        self.nu1, self.nu2 = nu1, nu2
        self.pre, self.post = pre, post
        for lv in levels[:-1]:
            if smoother == "jacobi":
                lv.smoother = mg.Jacobi(lv.A, omega)
            elif smoother == "gs":
                lv.smoother = mg.GaussSeidel(lv.A)
            else:
                alpha = stokes_alpha(lv.A, lv.op.d, lv.op.bs, zeta)
                lv.smoother = mg.SAI(lv.A, ell, balance=True, pre=pre, post=post, alpha=alpha)
        self.bottom_pinv = mg.sym_pinv(levels[-1].A.dense())


def gmres(A, V, b: np.ndarray, tol: float = 1e-10, restart: int = 50, max_iter: int = 200):
    """Left-preconditioned restarted GMRES from x0 = 0.  Returns (x, iterations,
    history of ||V (b - A x_k)||)."""
    apply_A = A if callable(A) else (lambda v: A @ v)
    x = np.zeros_like(b)
    r = V(b - apply_A(x))
    beta0 = np.linalg.norm(r)
    hist = [beta0]
    if beta0 == 0.0:
        return x, 0, hist
    k = 0
    while k < max_iter:
        beta = np.linalg.norm(r)
        m = min(restart, max_iter - k)
        Q = np.zeros((len(b), m + 1))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[:, 0] = r / beta
        j_done = 0
        for j in range(m):
            w = V(apply_A(Q[:, j]))
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = Q[:, i] @ w
                w = w - H[i, j] * Q[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                Q[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous Givens rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * beta0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Q[:, :j_done] @ y
        if abs(g[j_done]) <= tol * beta0:
            break
        r = V(b - apply_A(x))
    return x, k, hist


def fgmres(A, V, b: np.ndarray, tol: float = 1e-10, restart: int = 50, max_iter: int = 200):
    """Flexible right-preconditioned restarted GMRES (Saad's FGMRES) from x0 = 0:
    z_j = V(q_j) is kept, the Arnoldi step orthogonalises A z_j, and
    x = x0 + Z y minimises ||b - A x|| over span(Z).  The form of GMRES used
    when V is applied in reduced precision and so is not exactly linear.
    Returns (x, iterations, history of ||b - A x_k||)."""
    apply_A = A if callable(A) else (lambda v: A @ v)
    x = np.zeros_like(b)
    r = b - apply_A(x)
    beta0 = np.linalg.norm(r)
    hist = [beta0]
    if beta0 == 0.0:
        return x, 0, hist
    k = 0
    while k < max_iter:
        beta = np.linalg.norm(r)
        m = min(restart, max_iter - k)
        Q = np.zeros((len(b), m + 1))
        Z = np.zeros((len(b), m))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[:, 0] = r / beta
        j_done = 0
        for j in range(m):
            Z[:, j] = V(Q[:, j])
            w = apply_A(Z[:, j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = Q[:, i] @ w
                w = w - H[i, j] * Q[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                Q[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * beta0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:, :j_done] @ y
        r = b - apply_A(x)
        if abs(g[j_done]) <= tol * beta0 and np.linalg.norm(r) <= tol * beta0:
            break            # the estimate is confirmed on the true residual
    return x, k, hist
