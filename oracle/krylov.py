"""Oracle, part 3: multigrid-preconditioned CG and the eta metric.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): never imported by the product.

Readings:
  * Sec. 2.2 (last paragraph): the V-cycle with zero initial guess is the
    linear preconditioner V; CG needs it symmetric positive semi-definite
    (block Jacobi, or SAI with B1 pre / BT post, Sec. 2.4).
  * Stopping rule: ||b - A x_k||_2 <= tol ||b||_2 on the recurrence residual
    (the workloads ask for a 1e-10 relative residual), x_0 = 0.
  * Iteration count k = number of CG updates of x.
  * beta: Fletcher-Reeves form r_{k+1}^T z_{k+1} / r_k^T z_k for a fixed
    (FP64) V; the flexible Polak-Ribiere form r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k
    when V is applied in reduced precision (slightly nonlinear V).
  * eta (Eq. eta): eta = log 0.1 / log rho, rho = 10^slope of the least-squares
    line through (k, log10 r_k), over the recorded residual norms with
    r_k > 1e3 * eps * r_0 (the footnote to Eq. eta fits a line by simple linear
    regression; which points enter is our reading).
"""
from __future__ import annotations

import numpy as np


def pcg(A, V, b: np.ndarray, tol: float = 1e-10, max_iter: int = 200, flexible: bool = False):
    """Preconditioned CG from x0 = 0.  A: callable or matrix; V: callable.

    Returns (x, iterations, history) where history[k] = ||r_k||_2.
    """
    apply_A = A if callable(A) else (lambda v: A @ v)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r)]
    if bnorm == 0.0:
        return x, 0, hist
    z = V(r)
    p = z.copy()
    rz = r @ z
    k = 0
    while k < max_iter:
        q = apply_A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        rn = np.linalg.norm(r)
        hist.append(rn)
        if rn <= tol * bnorm:
            break
        z_new = V(r)
        if flexible:
            rz_new = r @ z_new
            beta = (rz_new - r @ z) / rz
        else:
            rz_new = r @ z_new
            beta = rz_new / rz
        z = z_new
        rz = rz_new
        p = z + beta * p
    return x, k, hist


def eta(history) -> float:
    """Iterations per factor-10 residual reduction (Eq. eta)."""
    h = np.asarray(history, dtype=np.float64)
    keep = h > 1e3 * np.finfo(np.float64).eps * h[0]
    k = np.arange(len(h))[keep]
    y = np.log10(h[keep])
    if len(k) < 2:
        return float("nan")
    slope = np.polyfit(k, y, 1)[0]
    return float(-1.0 / slope)
