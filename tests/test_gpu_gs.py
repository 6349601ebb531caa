"""GPU parity of multi-coloured block Gauss-Seidel (Sec. 2.3.2) through the C-ABI.

Tolerances as in test_gpu_parity.py: one sweep 1e-12 (1e-10 for the indefinite
Stokes blocks, whose pseudo-inverses agree to ~1e-12 times their condition);
whole V-cycles 1e-10; solves within one iteration of the oracle and 1e-9
(CG) / 1e-8 (GMRES) relative L2 after removing the kernel."""
import numpy as np
import pytest

from oracle import krylov, ldg
from oracle import multigrid as mg
from oracle import stokes as st
from paper_2412_12506_gb300.inputs import random_rhs, random_vector, square_mu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(v):
    return torch.tensor(np.asarray(v), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("d,n,p,stokes,mu_kind", [(2, 8, 2, None, None), (2, 8, 3, None, "square"),
                                                  (3, 4, 2, None, None), (2, 8, 2, 1, None)])
def test_gs_sweeps_and_vcycle_fp64(lib, d, n, p, stokes, mu_kind):
    mu = None if mu_kind is None else square_mu(d, n, mu_in=1e4)
    if stokes is None:
        levels = mg.build_levels(d, n, p, mu)
        V = mg.VCycle(levels, "gs", 3, 3, pre="B1", post="BT")
        op = lib.Operator(d, n, p, mu)
    else:
        levels = st.build_stokes_levels(d, n, p, mu, gamma=stokes)
        V = st.StokesVCycle(levels, "gs", 3, 3, pre="B1", post="BT")
        op = lib.Operator(d, n, p, mu, stokes=stokes)
    H = lib.Hierarchy(op, smoother="gs", pre="B1", post="BT")
    # 1e-10 with a coefficient jump or for the indefinite Stokes blocks: the two
    # eigendecomposition-based block inverses agree to ~1e-12 times the block
    # condition, not to rounding.
    tol = 1e-12 if stokes is None and mu_kind is None else 1e-10
    for l, lv in enumerate(levels[:-1]):
        size = lv.A.mat.shape[0]
        rhs, x = random_vector(size, 10 + l), random_vector(size, 20 + l)
        for form in ("B1", "BT"):
            got = H.level_smooth(l, form, cuda(rhs), cuda(x)).cpu().numpy()
            assert rel(got, lv.smoother.sweep(x, rhs, form)) < tol, (l, form)
            got0 = H.level_smooth(l, form, cuda(rhs)).cpu().numpy()          # x = 0
            assert rel(got0, lv.smoother.sweep(np.zeros(size), rhs, form)) < tol, (l, form)
        xt = cuda(x)                                                          # in place
        H.level_smooth(l, "BT", cuda(rhs), xt, xt)
        assert rel(xt.cpu().numpy(), lv.smoother.sweep(x, rhs, "BT")) < tol
    N0 = levels[0].A.nblocks
    r0 = random_vector(levels[0].A.mat.shape[0], 41)
    r0 = ldg.project_out_constant(r0, d, p, N0) if stokes is None else st.project_out_kernel(r0, d, p, N0)
    assert rel(H.vcycle(cuda(r0)).cpu().numpy(), V(r0)) < 1e-10


def test_gs_cg_and_gmres_solves_match_oracle(lib):
    d, n, p = 2, 32, 2
    N, b = n * n, (p + 1) ** 2
    levels = mg.build_levels(d, n, p)
    A = levels[0].A.mat
    rhs = ldg.project_out_constant(random_rhs(N, b, seed=21), d, p, N)
    op = lib.Operator(d, n, p)
    # symmetric pairing with CG
    V = mg.VCycle(levels, "gs", 3, 3, pre="B1", post="BT")
    xo, ko, _ = krylov.pcg(A, V, rhs, tol=1e-10)
    H = lib.Hierarchy(op, smoother="gs", pre="B1", post="BT")
    x, k, rr, status = H.solve(cuda(rhs), tol=1e-10)
    assert status == lib.OK and abs(k - ko) <= 1 and rr <= 1.05e-10
    xg = ldg.project_out_constant(x.cpu().numpy(), d, p, N)
    assert np.linalg.norm(xg - ldg.project_out_constant(xo, d, p, N)) <= 1e-9 * np.linalg.norm(xo)
    # same-order pairing with GMRES (asymmetric V-cycle)
    V2 = mg.VCycle(levels, "gs", 3, 3, pre="B1", post="B1")
    _, ko2, _ = st.gmres(A, V2, rhs, tol=1e-10)
    xo2, _, _ = st.gmres(A, V2, rhs, tol=1e-12)
    H2 = lib.Hierarchy(op, smoother="gs", pre="B1", post="B1", krylov="gmres")
    x2, k2, rr2, s2 = H2.solve(cuda(rhs), tol=1e-10)
    assert s2 == lib.OK and abs(k2 - ko2) <= 1
    xg2 = ldg.project_out_constant(x2.cpu().numpy(), d, p, N)
    assert np.linalg.norm(xg2 - ldg.project_out_constant(xo2, d, p, N)) <= 1e-8 * np.linalg.norm(xo2)
    # reduced precision: FP32 V-cycle, FP64 flexible CG
    H3 = lib.Hierarchy(op, smoother="gs", pre="B1", post="BT", precision="fp32")
    x3, k3, rr3, s3 = H3.solve(cuda(rhs), tol=1e-10)
    assert s3 == lib.OK and rr3 <= 1.05e-10 and k3 <= ko + 3


def test_gs_stokes_gmres_matches_oracle(lib):
    d, n, p, gamma = 2, 16, 2, 1
    levels = st.build_stokes_levels(d, n, p, gamma=gamma)
    V = st.StokesVCycle(levels, "gs", 3, 3, pre="B1", post="B1")
    N = n * n
    rhs = st.project_out_kernel(random_rhs(N, 3 * (p + 1) ** 2, seed=22), d, p, N)
    _, ko, _ = st.gmres(levels[0].A.mat, V, rhs, tol=1e-10)
    xo, _, _ = st.gmres(levels[0].A.mat, V, rhs, tol=1e-12)
    H = lib.Hierarchy(lib.Operator(d, n, p, stokes=gamma), smoother="gs", pre="B1", post="B1")
    x, k, rr, status = H.solve(cuda(rhs), tol=1e-10)
    assert status == lib.OK and abs(k - ko) <= 1
    xg = st.project_out_kernel(x.cpu().numpy(), d, p, N)
    assert np.linalg.norm(xg - st.project_out_kernel(xo, d, p, N)) <= 1e-8 * np.linalg.norm(xo)
