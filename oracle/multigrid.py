"""Oracle, part 2: hierarchy, smoothers and the V-cycle (Sec. 2.2-2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): never imported by the product.

Readings of passages the paper leaves open:
  * Hierarchy (Sec. 2.2, "Mesh hierarchy"): uniform h-coarsening by 2 per axis
    while n is even and n > 1; the level with odd n (or n = 1) is the bottom.
  * Injection I (Sec. 2.2, "Interpolation operator"): (I u)|_{E_f} = u|_{E_c},
    i.e. the child blocks are Kronecker products of the 1D matrices P_s.
  * Operator coarsening (Sec. 2.2, option (ii), details deferred to [dgmg]):
      G_{a,c}   = M_c^{-1} I^T M_f G_{a,f} I    (L2 projection of the fine gradient)
      M_mu,c    = I^T M_mu,f I
      E_c       = (1/2) I^T E_f I               (penalty tau/h at twice the size)
      A_c       = sum_a G_{a,c}^T M_mu,c G_{a,c} + E_c
    For mu == 1 this reproduces the operator assembled directly on the coarse
    mesh (the equivalence claimed in Sec. 2.2); a test checks that.
  * Block pattern of each operator = its structural pattern from this
    composition (BOp.pat), used for the SAI patterns of Sec. 2.3.3.
  * Block Jacobi (Eq. Jsmooth): A_ii^{-1} from a symmetric eigendecomposition,
    eigenvalues with |lambda| <= 1e-12 max|lambda| dropped (pseudo-inverse).
  * SAI (Sec. 2.3.3): S(i) = block rows of column i of the pattern of A^ell,
    R(i) = block rows touched by A[:, S(i)]; balanced with
    alpha_i = ||A_ii||_F^{-1/2}; each column is the least-squares solution of
    Atilde[R, S] X = I[R, i] by Householder QR, or the minimum-norm solution
    (SVD, relative cutoff 1e-12) when Atilde[R, S] is rank deficient.
  * Bottom solver (Sec. 2.2, "Bottom solver"): pseudo-inverse from a symmetric
    eigendecomposition, |lambda| <= 1e-12 max|lambda| treated as kernel.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .ldg import BOp, Basis1D, LDGOperator, Mesh, assemble, child_op, _from_blocks

EIG_CUTOFF = 1e-12


# ----------------------------------------------------------------------------
# Interpolation and operator coarsening (Sec. 2.2)
# ----------------------------------------------------------------------------

def injection(d: int, n_fine: int, p: int) -> BOp:
    """I_{2h}^h as a BOp of shape (N_fine*b) x (N_coarse*b); pattern is N_f x N_c."""
    assert n_fine % 2 == 0
    bas = Basis1D(p)
    b = (p + 1) ** d
    fine, coarse = Mesh(d, n_fine), Mesh(d, n_fine // 2)
    rows, cols, vals, prow, pcol = [], [], [], [], []
    ii, jj = np.meshgrid(np.arange(b), np.arange(b), indexing="ij")
    for C in range(coarse.N):
        cc = coarse.coords(C)
        for s in itertools.product((0, 1), repeat=d):
            f = fine.index(tuple(2 * cc[a] + s[a] for a in range(d)))
            blk = child_op(bas.P, s, d)
            rows.append((f * b + ii).ravel())
            cols.append((C * b + jj).ravel())
            vals.append(blk.ravel())
            prow.append(f)
            pcol.append(C)
    mat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(fine.N * b, coarse.N * b))
    pat = sp.csr_matrix((np.ones(len(prow), dtype=np.int8), (prow, pcol)),
                        shape=(fine.N, coarse.N))
    return BOp(mat, pat, b)


def coarsen(op: LDGOperator, I: BOp) -> LDGOperator:
    """Operator coarsening of Sec. 2.2 option (ii), as read in the module header."""
    It = I.T
    d, b = op.d, op.b
    h_c = 2.0 * op.h
    Nc = I.pat.shape[1]
    mass_c = (h_c / 2.0) ** d
    M_c = _from_blocks({(e, e): mass_c * np.eye(b) for e in range(Nc)}, Nc, b)
    Minv_c = _from_blocks({(e, e): np.eye(b) / mass_c for e in range(Nc)}, Nc, b)
    G_c = [Minv_c @ It @ op.M @ op.G[a] @ I for a in range(d)]
    Mmu_c = It @ op.Mmu @ I
    E_c = (It @ op.E @ I).scale(0.5)
    return LDGOperator(G_c, Mmu_c, M_c, E_c, d, b, h_c)


class Level:
    def __init__(self, n: int, op: LDGOperator):
        self.n = n
        self.op = op
        self.A = op.A
        self.N = op.A.nblocks
        self.b = op.b
        self.I = None        # injection from the next coarser level
        self.smoother = None


def build_levels(d: int, n: int, p: int, mu=None, tau0: float = 1.0):
    """Finest operator by assembly, coarser ones by operator coarsening."""
    levels = [Level(n, assemble(d, n, p, mu, tau0))]
    while levels[-1].n % 2 == 0 and levels[-1].n > 1:
        nf = levels[-1].n
        I = injection(d, nf, p)
        levels[-1].I = I
        levels.append(Level(nf // 2, coarsen(levels[-1].op, I)))
    return levels


# ----------------------------------------------------------------------------
# Symmetric pseudo-inverse (Jacobi blocks, bottom solver)
# ----------------------------------------------------------------------------

def sym_pinv(S: np.ndarray, cutoff: float = EIG_CUTOFF) -> np.ndarray:
    lam, U = np.linalg.eigh(S)
    keep = np.abs(lam) > cutoff * np.max(np.abs(lam))
    inv = np.zeros_like(lam)
    inv[keep] = 1.0 / lam[keep]
    return (U * inv) @ U.T


# ----------------------------------------------------------------------------
# Block Jacobi (Sec. 2.3.1, Eq. Jsmooth)
# ----------------------------------------------------------------------------

class Jacobi:
    def __init__(self, A: BOp, omega: float = 0.8):
        self.A = A
        self.omega = omega
        self.b = A.b
        self.N = A.nblocks
        self.Dinv = [sym_pinv(A.block(i, i)) for i in range(self.N)]

    def sweep(self, x: np.ndarray, rhs: np.ndarray, form: str = "B1") -> np.ndarray:
        """x_bar_i = (1 - w) x_i + w A_ii^{-1} (b_i - sum_{j != i} A_ij x_j)."""
        b, w = self.b, self.omega
        Ax = self.A.mat @ x
        out = np.empty_like(x)
        for i in range(self.N):
            sl = slice(i * b, (i + 1) * b)
            off = Ax[sl] - self.A.block(i, i) @ x[sl]          # sum over j != i
            out[sl] = (1.0 - w) * x[sl] + w * (self.Dinv[i] @ (rhs[sl] - off))
        return out


# ----------------------------------------------------------------------------
# Multi-coloured block Gauss-Seidel (Sec. 2.3.2)
# ----------------------------------------------------------------------------

def greedy_colouring(pat: sp.spmatrix) -> np.ndarray:
    """Colour per element for multi-coloured Gauss-Seidel (Sec. 2.3.2): elements
    visited in index order take the smallest colour no already coloured
    neighbour in the (symmetrised) block pattern of A has.  On the periodic
    Cartesian grid with one-sided fluxes and even n this is the red-black
    colouring of the 5- / 7-point block stencil."""
    P = sp.csr_matrix(pat, dtype=np.int8)
    S = (P + P.T).tocsr()
    N = S.shape[0]
    colour = -np.ones(N, dtype=int)
    for i in range(N):
        nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
        used = {int(colour[j]) for j in nb if j != i and colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


class GaussSeidel:
    """Multi-coloured block Gauss-Seidel, undamped (omega = 1, Sec. 2.3.2): the
    elements of one colour are updated together, x_i <- A_ii^{-1} (b_i -
    sum_{j != i} A_ij x_j) with the newest x_j, then the next colour.  Form "B1"
    visits the colours in increasing order (forward), "BT" in decreasing
    order (backward); forward pre- and backward post-sweeps give a symmetric
    V-cycle (Sec. 2.4, pairing (ii))."""

    def __init__(self, A: BOp, omega: float = 1.0):
        self.A = A
        self.omega = omega
        self.b = A.b
        self.N = A.nblocks
        self.colour = greedy_colouring(A.pat)
        self.ncolours = int(self.colour.max()) + 1
        self.Dinv = [sym_pinv(A.block(i, i)) for i in range(self.N)]

    def sweep(self, x: np.ndarray, rhs: np.ndarray, form: str = "B1") -> np.ndarray:
        b, w = self.b, self.omega
        order = range(self.ncolours) if form == "B1" else range(self.ncolours - 1, -1, -1)
        x = x.copy()
        for c in order:
            Ax = self.A.mat @ x
            new = {}
            for i in np.where(self.colour == c)[0]:
                sl = slice(i * b, (i + 1) * b)
                off = Ax[sl] - self.A.block(i, i) @ x[sl]
                new[i] = (1.0 - w) * x[sl] + w * (self.Dinv[i] @ (rhs[sl] - off))
            for i, v in new.items():
                x[i * b:(i + 1) * b] = v
        return x


# ----------------------------------------------------------------------------
# Balanced block SAI (Sec. 2.3.3)
# ----------------------------------------------------------------------------

def pattern_power(pat: sp.csr_matrix, ell: int) -> sp.csr_matrix:
    N = pat.shape[0]
    out = sp.identity(N, dtype=np.int64, format="csr")
    for _ in range(ell):
        out = out @ pat.astype(np.int64)
    return sp.csr_matrix((out != 0).astype(np.int8))


def sai_sets(A: BOp, ell: int, i: int, Pc=None, Ac=None):
    """S(i): block rows of column i of pattern(A^ell); R(i): rows of A[:, S(i)]."""
    if Pc is None:
        Pc = pattern_power(A.pat, ell).tocsc()
    if Ac is None:
        Ac = A.pat.tocsc()
    S = np.sort(Pc.indices[Pc.indptr[i]:Pc.indptr[i + 1]])
    R = set()
    for k in S:
        R.update(Ac.indices[Ac.indptr[k]:Ac.indptr[k + 1]].tolist())
    return S, np.array(sorted(R))


def ls_solve(M: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Least squares by Householder QR (LAPACK, as in Sec. 2.3.3); minimum-norm
    solution by SVD when M is rank deficient."""
    Q, R = np.linalg.qr(M, mode="reduced")
    dR = np.abs(np.diag(R))
    if dR.min() > 1e-12 * dR.max():
        return sla.solve_triangular(R, Q.T @ rhs)
    return np.linalg.lstsq(M, rhs, rcond=1e-12)[0]


class SAI:
    """B = diag(alpha) Btilde diag(alpha), Btilde = argmin ||Atilde B - I||_F over
    matrices with the block pattern of A^ell (Sec. 2.3.3)."""

    def __init__(self, A: BOp, ell: int = 1, balance: bool = True, pre: str = "B1",
                 post: str = "BT", alpha=None, build: bool = True):
        """alpha: optional per-dof balancing vector (Sec. 3.3, Stokes); by default
        alpha_i = ||A_ii||_F^{-1/2} on every dof of element i (Sec. 2.3.3).
        build = False prepares the least-squares data without solving every
        column (columns are then computed on demand by column(i))."""
        self.A, self.ell = A, ell
        self.pre, self.post = pre, post
        b, N = A.b, A.nblocks
        self.b, self.N = b, N
        if alpha is not None:
            self.alpha = np.asarray(alpha, dtype=np.float64)
            self.alpha_el = None
        else:
            if balance:
                alpha_el = np.array([np.linalg.norm(A.block(i, i), "fro") ** -0.5 for i in range(N)])
            else:
                alpha_el = np.ones(N)
            self.alpha_el = alpha_el
            self.alpha = np.repeat(alpha_el, b)
        self._alpha_blk = self.alpha.reshape(N, b)
        Da = sp.diags(self.alpha)
        self._At = (Da @ A.mat @ Da).tocsc()
        self._Pc = pattern_power(A.pat, ell).tocsc()
        self._Ac = A.pat.tocsc()
        if not build:
            return
        blocks = {}
        for i in range(N):
            blocks.update(self.column(i))
        self.B = _from_blocks(blocks, N, b)

    def column(self, i: int) -> dict:
        """Block column i of B: {(k, i): B_ki for k in S(i)}."""
        b = self.b
        S, R = sai_sets(self.A, self.ell, i, self._Pc, self._Ac)
        rows = np.concatenate([np.arange(r * b, (r + 1) * b) for r in R])
        cols = np.concatenate([np.arange(k * b, (k + 1) * b) for k in S])
        Mloc = self._At[:, cols].tocsr()[rows, :].toarray()
        rhs = np.zeros((len(rows), b))
        pos = int(np.where(R == i)[0][0])
        rhs[pos * b:(pos + 1) * b, :] = np.eye(b)
        X = ls_solve(Mloc, rhs)
        out = {}
        for t, k in enumerate(S):
            # B = diag(alpha) Btilde diag(alpha)
            out[(int(k), i)] = self._alpha_blk[k][:, None] * X[t * b:(t + 1) * b, :] * self._alpha_blk[i][None, :]
        return out

    def sweep(self, x: np.ndarray, rhs: np.ndarray, form: str) -> np.ndarray:
        r = self.A.mat @ x - rhs
        if form == "B1":
            return x - self.B.mat @ r           # Eq. B1
        return x - self.B.mat.T @ r             # Eq. BT


# ----------------------------------------------------------------------------
# V-cycle (Algorithm 1)
# ----------------------------------------------------------------------------

class VCycle:
    """Multigrid V-cycle of Algorithm 1 with nu1 pre- and nu2 post-sweeps.

    pairing (Sec. 2.4): for SAI the pre-sweep uses form `pre` and the
    post-sweep form `post` ("B1"/"BT"); for multi-coloured Gauss-Seidel
    ("gs") "B1" / "BT" are the forward / backward colour orders; block Jacobi
    ignores the form.
    """

    def __init__(self, levels, smoother: str = "jacobi", nu1: int = 3, nu2: int = 3,
                 omega: float = 0.8, ell: int = 1, pre: str = "B1", post: str = "BT",
                 balance: bool = True):
        self.levels = levels
        self.nu1, self.nu2 = nu1, nu2
        self.pre, self.post = pre, post
        for lv in levels[:-1]:
            if smoother == "jacobi":
                lv.smoother = Jacobi(lv.A, omega)
            elif smoother == "gs":
                lv.smoother = GaussSeidel(lv.A)
            else:
                lv.smoother = SAI(lv.A, ell, balance, pre, post)
        self.bottom_pinv = sym_pinv(levels[-1].A.dense())

    def cycle(self, lvl: int, x: np.ndarray, rhs: np.ndarray) -> np.ndarray:
        lv = self.levels[lvl]
        if lvl == len(self.levels) - 1:
            return self.bottom_pinv @ rhs                         # line 2
        for _ in range(self.nu1):                                 # line 4
            x = lv.smoother.sweep(x, rhs, self.pre)
        r2h = lv.I.mat.T @ (rhs - lv.A.mat @ x)                   # line 5
        x2h = self.cycle(lvl + 1, np.zeros(r2h.shape), r2h)       # line 6
        x = x + lv.I.mat @ x2h                                    # line 7
        for _ in range(self.nu2):                                 # line 8
            x = lv.smoother.sweep(x, rhs, self.post)
        return x

    def __call__(self, rhs: np.ndarray) -> np.ndarray:
        """The preconditioner V: the V-cycle with zero initial guess (Sec. 2.2)."""
        return self.cycle(0, np.zeros_like(rhs), rhs)
