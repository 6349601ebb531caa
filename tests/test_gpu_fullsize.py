"""Full-size checks of the benchmarked workloads, in the launch configuration
bench.py times, against what the oracle can compute at that size.

  * 2D two-phase Stokes, 128^2, p = 2, stress form, viscosity 1 / 1e3 on the
    inclusion: the whole FP64 operator apply against the oracle's assembled
    operator; sampled block columns of the level-0 SAI (one least-squares
    problem each in the oracle); the FGMRES solve with an FP32 V-cycle checked
    by the oracle's own residual ||b - A x|| / ||b||.
  * 2D interface problem, 256^2, p = 3, contrast 1e4, 64 right-hand sides on
    the tensor-core hierarchy: the batched FP32 operator apply on sampled
    right-hand sides against the oracle, and the batched solve checked by the
    oracle's residual on sampled right-hand sides.
Tolerances: FP64 apply 1e-12 (as in test_gpu_parity.py); SAI columns 1e-9
(two independent least-squares solves); FP32-split tensor-core apply within
2^-14 * sum_j |a_ij x_j| per entry (x and A each split into two BF16 parts,
|a - hi - lo| <= 2^-17 |a|: the dropped lo*lo product costs at most 2^-16, the
two split remainders 2^-17 each, FP32 accumulation of <= 240 products
< 2^-16; rows cancel across the 1e4 jump, so the bound is on sum |a x|); solves
at the requested residual (1e-9 for Stokes FGMRES, the FP64 attainable level
on this operator; 1e-10 for the interface CG) plus 5% for the independent
residual evaluation.
"""
import numpy as np
import pytest

from oracle import ldg
from oracle import multigrid as mg
from oracle import stokes as st
from paper_2412_12506_gb300.inputs import fourier_force_rhs, random_rhs, random_vector, square_mu

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


def test_stokes_128_full_size(lib):
    d, n, p, gamma = 2, 128, 2, 1
    mu = square_mu(d, n, mu_in=1e3)
    ref = st.assemble_stokes(d, n, p, mu, gamma=gamma)
    A = ref.A.mat.tocsr()
    op = lib.Operator(d, n, p, mu, stokes=gamma)
    x = random_vector(op.size, 90)
    y = op.apply(torch.tensor(x, device="cuda")).cpu().numpy()
    assert rel(y, A @ x) < 1e-12
    # sampled SAI block columns of level 0 (interior, interface, corner elements)
    H = lib.Hierarchy(op, smoother="sai", precision="fp64")
    alpha = st.stokes_alpha(ref.A, d, ref.bs, st.ZETA[(gamma, d)][p - 1])
    sai = mg.SAI(ref.A, 1, alpha=alpha, build=False)   # columns on demand
    b = ref.b
    for i in (0, n * n // 2 + n // 4, n * (n // 4) + n // 4, n * n - 1):
        col = sai.column(i)
        for c in range(b):
            e = np.zeros(op.size)
            e[i * b + c] = 1.0
            got = H.level_apply(0, lib.MAT_B, torch.tensor(e, device="cuda")).cpu().numpy()
            for (k, _), blk in col.items():
                assert rel(got[k * b:(k + 1) * b], blk[:, c]) < 1e-9, (i, c, k)
    # the benchmarked solve: FGMRES, FP32 V-cycle, true residual 1e-9
    rhs = fourier_force_rhs(d, n, p, seed=0, nmodes=8)
    rt = torch.tensor(rhs, device="cuda")
    op.project_kernel(rt)
    Hm = lib.Hierarchy(op, smoother="sai", precision="fp32", krylov="fgmres")
    xs, k, rr, status = Hm.solve(rt, tol=1e-9)
    assert status == lib.OK and rr <= 1e-9
    bh, xh = rt.cpu().numpy(), xs.cpu().numpy()
    assert np.linalg.norm(bh - A @ xh) <= 1.05e-9 * np.linalg.norm(bh)


def test_interface_256_batched_full_size(lib):
    d, n, p, R = 2, 256, 3, 64
    mu = square_mu(d, n, mu_in=1e4)
    ref = ldg.assemble(d, n, p, mu)
    A = ref.A.mat.tocsr()
    N, b = n * n, (p + 1) ** 2
    op = lib.Operator(d, n, p, mu)
    H = lib.Hierarchy(op, smoother="sai", precision="fp32", max_rhs=R)
    X = np.stack([random_vector(op.size, 200 + r) for r in range(R)])        # [rhs][element][mode]
    Xb = np.ascontiguousarray(X.reshape(R, N, b).transpose(1, 0, 2)).reshape(-1)   # [element][rhs][mode]
    Y = H.level_apply_batched(0, lib.MAT_A, torch.tensor(Xb, dtype=torch.float32, device="cuda"), R)
    Y = Y.cpu().numpy().reshape(N, R, b).transpose(1, 0, 2).reshape(R, -1)
    absA = abs(A)
    for r in (0, 17, R - 1):
        # x and A are each split into two BF16 parts (|x - hi - lo| <= 2^-17 |x|);
        # worst case per product 2^-16 + 2 * 2^-17 plus FP32 accumulation, under
        # 2^-14; bounded against sum |a x| because the 1e4 jump makes rows cancel
        bound = 2.0 ** -14 * (absA @ np.abs(X[r]))
        assert np.all(np.abs(Y[r] - A @ X[r]) <= bound), r
    B = np.stack([ldg.project_out_constant(random_rhs(N, b, seed=300 + r), d, p, N) for r in range(R)])
    Xs, its, res, status = H.solve(torch.tensor(B, device="cuda"), tol=1e-10)
    assert status == lib.OK and max(res) <= 1.05e-10
    Xs = Xs.cpu().numpy()
    for r in (0, 31, R - 1):
        assert np.linalg.norm(B[r] - A @ Xs[r]) <= 1.1e-10 * np.linalg.norm(B[r]), r
