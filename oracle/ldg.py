"""Oracle, part 1: basis and LDG operator (Sec. 2.1 of the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): never imported by the product.

Everything is FP64 and written to be read against the paper, not to be fast.

Readings of passages the paper leaves open (Sec. 2.1 defers details to its
references [dgmg, fluxx]):
  * Basis: phi_k(xi) = sqrt((2k+1)/2) P_k(xi) on [-1, 1] (orthonormal Legendre,
    "tensor-product Legendre polynomial modal basis", Sec. 2.1); mode index
    m = kx + (p+1) ky + (p+1)^2 kz.  Element E of size h maps x = x_E + (h/2) xi.
  * Discrete gradient, step (i) of Sec. 2.1, strong lifting form: for v in Q_p(E)
      int_E (G_a u) v = int_E (d_a u_E) v + sum_{faces f of E normal to a} int_f (u_hat - u_E) v n_a.
  * Viscosity-upwinded flux (Sec. 2.1, first bullet): on the face between the
    lower element L and the upper element U of axis a, u_hat is the trace of the
    element with the larger mu; on a tie (single phase) u_hat = u_L.
  * mu-weighted mass: M_mu = blockdiag(mu_E M_E), M_E = (h/2)^d I (sigma is the
    L2 projection of mu * tau with mu constant per element, step (ii)).
  * Penalty E (step (iv)): E = sum_faces tau_f int_f [u][v], [u] = u_L - u_U,
    tau_f = tau0 * min(mu_L, mu_U) / h, tau0 = 1 by default.
  * A = sum_a G_a^T M_mu G_a + E (Sec. 2.1, display after Eq. scalar3).
Periodic boundaries on the unit cube, h = 1/n.  With n <= 2 the two neighbours
along an axis coincide (or are E itself for n = 1); their contributions add.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as npleg


# ----------------------------------------------------------------------------
# 1D basis (Sec. 2.1, "tensor-product Legendre polynomial modal basis")
# ----------------------------------------------------------------------------

def phi(k: int, xi):
    """Orthonormal Legendre polynomial sqrt((2k+1)/2) P_k evaluated at xi."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    return np.sqrt((2 * k + 1) / 2.0) * npleg.legval(xi, c)


def dphi(k: int, xi):
    """Derivative of phi_k with respect to xi."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    return np.sqrt((2 * k + 1) / 2.0) * npleg.legval(xi, npleg.legder(c))


class Basis1D:
    """Reference-interval matrices for degree p, all by Gauss quadrature.

    mass[i, j]  = int phi_i phi_j               (identity for this basis)
    K[i, j]     = int phi_i phi_j'              (volume derivative term)
    hi[k], lo[k] = phi_k(+1), phi_k(-1)         (face traces)
    P[s][i, j]  = int phi_i(xi) phi_j((xi + 2s - 1)/2) dxi
                  (coefficients of the coarse mode j restricted to child s,
                   s = 0 lower half, s = 1 upper half: polynomial injection)
    """

    def __init__(self, p: int):
        self.p = p
        q = p + 2
        xg, wg = npleg.leggauss(q)
        V = np.array([phi(k, xg) for k in range(p + 1)])     # (p+1, q)
        dV = np.array([dphi(k, xg) for k in range(p + 1)])
        self.mass = (V * wg) @ V.T
        self.K = (V * wg) @ dV.T
        self.hi = np.array([phi(k, 1.0) for k in range(p + 1)])
        self.lo = np.array([phi(k, -1.0) for k in range(p + 1)])
        self.P = []
        for s in (0, 1):
            eta = (xg + 2 * s - 1) / 2.0
            Vc = np.array([phi(k, eta) for k in range(p + 1)])
            self.P.append((V * wg) @ Vc.T)


def axis_op(M1: np.ndarray, a: int, d: int) -> np.ndarray:
    """Apply the 1D matrix M1 along axis a, identity along the others.

    Mode index m = kx + (p+1) ky + (p+1)^2 kz, i.e. kx fastest, so the Kronecker
    factors run from the slowest axis (d-1) down to x (axis 0).
    """
    q = M1.shape[0]
    out = np.ones((1, 1))
    for ax in range(d - 1, -1, -1):
        out = np.kron(out, M1 if ax == a else np.eye(q))
    return out


def child_op(P, s: tuple, d: int) -> np.ndarray:
    """Injection block for the child with offsets s = (s_x, s_y[, s_z])."""
    out = np.ones((1, 1))
    for ax in range(d - 1, -1, -1):
        out = np.kron(out, P[s[ax]])
    return out


# ----------------------------------------------------------------------------
# Block-sparse operators: values as a scipy CSR over dofs, plus the block
# pattern (which blocks are structurally present) as a boolean CSR over
# elements.  The pattern is what Sec. 2.3.3 calls the block-sparse pattern.
# ----------------------------------------------------------------------------

class BOp:
    def __init__(self, mat: sp.spmatrix, pat: sp.spmatrix, b: int):
        self.mat = sp.csr_matrix(mat)
        self.pat = sp.csr_matrix((sp.csr_matrix(pat) != 0).astype(np.int8))
        self.b = b

    @property
    def nblocks(self) -> int:
        return self.pat.shape[0]

    def __matmul__(self, other: "BOp") -> "BOp":
        return BOp(self.mat @ other.mat,
                   (self.pat.astype(np.int64) @ other.pat.astype(np.int64)), self.b)

    def __add__(self, other: "BOp") -> "BOp":
        return BOp(self.mat + other.mat, (self.pat + other.pat), self.b)

    def scale(self, s: float) -> "BOp":
        return BOp(self.mat * s, self.pat, self.b)

    @property
    def T(self) -> "BOp":
        return BOp(self.mat.T, self.pat.T, self.b)

    def block(self, i: int, j: int) -> np.ndarray:
        b = self.b
        return self.mat[i * b:(i + 1) * b, j * b:(j + 1) * b].toarray()

    def dense(self) -> np.ndarray:
        return self.mat.toarray()

    def row_pattern(self, i: int) -> np.ndarray:
        return self.pat.indices[self.pat.indptr[i]:self.pat.indptr[i + 1]]


def _from_blocks(blocks: dict, N: int, b: int) -> BOp:
    """Build a BOp from {(i, j): b x b array}; duplicate keys must be pre-summed."""
    rows, cols, vals = [], [], []
    prow, pcol = [], []
    ii, jj = np.meshgrid(np.arange(b), np.arange(b), indexing="ij")
    for (i, j), blk in blocks.items():
        rows.append((i * b + ii).ravel())
        cols.append((j * b + jj).ravel())
        vals.append(blk.ravel())
        prow.append(i)
        pcol.append(j)
    mat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(N * b, N * b))
    pat = sp.csr_matrix((np.ones(len(prow), dtype=np.int8), (prow, pcol)), shape=(N, N))
    return BOp(mat, pat, b)


def _add(blocks: dict, key, val):
    if key in blocks:
        blocks[key] = blocks[key] + val
    else:
        blocks[key] = val.copy()


# ----------------------------------------------------------------------------
# Uniform periodic Cartesian mesh
# ----------------------------------------------------------------------------

class Mesh:
    def __init__(self, d: int, n: int):
        self.d, self.n = d, n
        self.N = n ** d
        self.h = 1.0 / n

    def index(self, c) -> int:
        e = 0
        for ax in range(self.d - 1, -1, -1):
            e = e * self.n + (c[ax] % self.n)
        return e

    def coords(self, e: int) -> tuple:
        c = []
        for _ in range(self.d):
            c.append(e % self.n)
            e //= self.n
        return tuple(c)

    def faces(self, a: int):
        """All faces normal to axis a as (L, U): U is L's upper neighbour."""
        for L in range(self.N):
            c = list(self.coords(L))
            c[a] += 1
            yield L, self.index(c)


# ----------------------------------------------------------------------------
# LDG operator (Sec. 2.1)
# ----------------------------------------------------------------------------

class LDGOperator:
    """G_a (a = 0..d-1), M_mu, plain mass M, penalty E and A on one mesh."""

    def __init__(self, G, Mmu, M, E, d, b, h):
        self.G, self.Mmu, self.M, self.E = G, Mmu, M, E
        self.d, self.b, self.h = d, b, h
        A = E
        for a in range(d):
            A = A + (G[a].T @ Mmu @ G[a])
        self.A = A


def assemble(d: int, n: int, p: int, mu=None, tau0: float = 1.0) -> LDGOperator:
    """Assemble the LDG Laplacian of Sec. 2.1 on the periodic n^d mesh."""
    mesh = Mesh(d, n)
    N, h = mesh.N, mesh.h
    if mu is None:
        mu = np.ones(N)
    mu = np.asarray(mu, dtype=np.float64)
    bas = Basis1D(p)
    b = (p + 1) ** d
    lo, hi = bas.lo, bas.hi
    scale_G = 1.0 / (h / 2.0)           # M_E^{-1} * (face/volume Jacobians)
    w_face = (h / 2.0) ** (d - 1)       # face integral of two tangential modes

    G = []
    for a in range(d):
        blocks = {}
        vol = scale_G * axis_op(bas.K, a, d)
        for e in range(N):
            _add(blocks, (e, e), vol)
        for L, U in mesh.faces(a):
            if mu[L] >= mu[U]:
                # u_hat = u_L: lifting acts on U through its lower face (n_a = -1):
                # -phi(-1) (phi(+1)^T u_L - phi(-1)^T u_U)
                _add(blocks, (U, U), scale_G * axis_op(np.outer(lo, lo), a, d))
                _add(blocks, (U, L), -scale_G * axis_op(np.outer(lo, hi), a, d))
            else:
                # u_hat = u_U: lifting acts on L through its upper face (n_a = +1):
                # +phi(+1) (phi(-1)^T u_U - phi(+1)^T u_L)
                _add(blocks, (L, L), -scale_G * axis_op(np.outer(hi, hi), a, d))
                _add(blocks, (L, U), scale_G * axis_op(np.outer(hi, lo), a, d))
        G.append(_from_blocks(blocks, N, b))

    mass_E = (h / 2.0) ** d
    Mmu = _from_blocks({(e, e): mu[e] * mass_E * np.eye(b) for e in range(N)}, N, b)
    M = _from_blocks({(e, e): mass_E * np.eye(b) for e in range(N)}, N, b)

    blocks = {}
    for a in range(d):
        for L, U in mesh.faces(a):
            tau = tau0 * min(mu[L], mu[U]) / h
            c = tau * w_face
            _add(blocks, (L, L), c * axis_op(np.outer(hi, hi), a, d))
            _add(blocks, (L, U), -c * axis_op(np.outer(hi, lo), a, d))
            _add(blocks, (U, L), -c * axis_op(np.outer(lo, hi), a, d))
            _add(blocks, (U, U), c * axis_op(np.outer(lo, lo), a, d))
    E = _from_blocks(blocks, N, b)
    return LDGOperator(G, Mmu, M, E, d, b, h)


# ----------------------------------------------------------------------------
# Helpers used by tests and the solver: kernel vector, L2 projection
# ----------------------------------------------------------------------------

def constant_vector(d: int, p: int, N: int) -> np.ndarray:
    """Coefficients of u == 1: mode 0 carries 1 / phi_0^d = sqrt(2)^d."""
    b = (p + 1) ** d
    c = np.zeros(N * b)
    c[0::b] = np.sqrt(2.0) ** d
    return c


def project_out_constant(v: np.ndarray, d: int, p: int, N: int) -> np.ndarray:
    """v - (c^T v / c^T c) c with c the constant-function vector (Sec. 2.2,
    bottom-solver remark on kernels): makes b consistent with the periodic kernel."""
    c = constant_vector(d, p, N)
    if v.ndim == 1:
        return v - (c @ v) / (c @ c) * c
    return v - np.outer(c, (c @ v) / (c @ c))


def l2_project(f, d: int, n: int, p: int, q: int | None = None) -> np.ndarray:
    """Moments b_{E,m} = int_E f phi_m (the 'mass basis' right-hand side of the
    footnote to Algorithm 1), by tensor Gauss quadrature with q points per axis."""
    mesh = Mesh(d, n)
    h = mesh.h
    q = q or p + 3
    xg, wg = npleg.leggauss(q)
    V = np.array([phi(k, xg) for k in range(p + 1)])       # (p+1, q)
    b = (p + 1) ** d
    out = np.zeros(mesh.N * b)
    for e in range(mesh.N):
        c = mesh.coords(e)
        pts = [(c[a] + 0.5) * h + (h / 2.0) * xg for a in range(d)]
        grids = np.meshgrid(*pts, indexing="ij")            # grids[a][i_x, i_y, ...]
        fv = f(*grids)
        W = wg
        for _ in range(d - 1):
            W = np.multiply.outer(W, wg)
        fw = fv * W * (h / 2.0) ** d
        # moment for mode (kx, ky, kz): sum fw * V[kx, ix] V[ky, iy] V[kz, iz]
        if d == 2:
            mom = np.einsum("xy,ax,by->ba", fw, V, V)
        else:
            mom = np.einsum("xyz,ax,by,cz->cba", fw, V, V, V)
        out[e * b:(e + 1) * b] = mom.reshape(-1)
    return out


def evaluate(u: np.ndarray, d: int, n: int, p: int, xi_pts: np.ndarray):
    """Values of the discrete function at the tensor grid xi_pts in every element.
    Returns array (N, len(xi_pts)^d) in the same point order as l2_project."""
    mesh = Mesh(d, n)
    b = (p + 1) ** d
    V = np.array([phi(k, xi_pts) for k in range(p + 1)])
    out = []
    for e in range(mesh.N):
        ue = u[e * b:(e + 1) * b].reshape((p + 1,) * d)       # [kz, ky, kx] / [ky, kx]
        if d == 2:
            val = np.einsum("ba,ax,by->xy", ue, V, V)
        else:
            val = np.einsum("cba,ax,by,cz->xyz", ue, V, V, V)
        out.append(val.reshape(-1))
    return np.array(out)
