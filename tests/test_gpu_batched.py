"""Batched right-hand sides: tensor-core block apply and batched CG (GPU).

  * The tcgen05 apply (blocks stored as BF16 operand images -- hi and lo for
    FP32 storage --, FP32 vectors split into hi/lo BF16 parts, FP32
    accumulation in tensor memory) matches the FP64 product of the stored
    blocks to 1e-5 relative for R = 1 ... 128.
  * A batched solve gives every right-hand side the same iterate, bit for bit,
    as solving it alone (per-RHS scalars, converged RHS frozen), reaches the
    1e-10 residual, and agrees with the FP64 oracle solution.
  * Stacked multi-RHS applies and V-cycles equal the single-RHS ones.
"""
import numpy as np
import pytest
from bsr_dense import bsr_to_dense

from oracle import krylov, ldg
from oracle import multigrid as mg
from paper_2412_12506_gb300.inputs import random_rhs, square_mu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


def _batch_layout(stacked, N, b):
    """[rhs][element][mode] -> [element][rhs][mode]"""
    R = stacked.shape[0]
    return np.ascontiguousarray(stacked.reshape(R, N, b).transpose(1, 0, 2))


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("d,n,p", [(2, 10, 3), (3, 6, 3)])
@pytest.mark.parametrize("R", [1, 5, 64, 128])
def test_tensor_core_apply_matches_stored_blocks(lib, d, n, p, R, prec):
    """BF16 blocks: 2 MMAs (x hi/lo); FP32 blocks: 3 MMAs (A and x hi/lo)."""
    op = lib.Operator(d, n, p)
    H = lib.Hierarchy(op, smoother="sai", precision=prec, max_rhs=2, nu1=1, nu2=1)
    N, b = op.N, op.b
    rng = np.random.default_rng(R)
    for which in (lib.MAT_A, lib.MAT_B, lib.MAT_BT):
        rp, col, vals = H.export_level(0, which)
        M = bsr_to_dense(rp, col, vals)
        xs = rng.standard_normal((R, N * b)).astype(np.float32)
        xb = torch.tensor(_batch_layout(xs, N, b), device="cuda")
        y = H.level_apply_batched(0, which, xb, R).cpu().numpy()
        ref = _batch_layout((M @ xs.astype(np.float64).T).T, N, b)
        err = np.abs(y - ref).max() / np.abs(ref).max()
        assert err < 1e-5, (which, err)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_cached_tensor_core_apply_against_stored_blocks_and_per_use_kernel(lib, prec):
    """The cached kernel (max_rhs <= 64, 2D b = 16: one MMA per block on the
    packed [x_hi; x_lo] operand) against the FP64 product of the exported
    stored blocks (FP32 accumulation: 1e-5 of the largest entry) and against
    the per-use kernel (taken for max_rhs > 64), on every level of an
    interface hierarchy whose coarse rows have extra blocks.  Whole V-cycles
    (all epilogues: plain, residual, update) are no less accurate against the
    FP64 V-cycle than the per-use kernel's (the 1e4 contrast amplifies the
    FP32 rounding of the applies to ~1e-3 in both).  A right-hand side applied
    alone gives bit for bit its result in the 64-wide batch."""
    from paper_2412_12506_gb300.inputs import square_mu
    d, n, p = 2, 24, 3
    op = lib.Operator(d, n, p, square_mu(d, n, 1e4))
    Hc = lib.Hierarchy(op, smoother="sai", precision=prec, max_rhs=64, nu1=2, nu2=2)
    Hu = lib.Hierarchy(op, smoother="sai", precision=prec, max_rhs=65, nu1=2, nu2=2)
    H64 = lib.Hierarchy(op, smoother="sai", precision="fp64", max_rhs=64, nu1=2, nu2=2)
    assert Hc.tc_schedule[0] > 0 and Hu.tc_schedule[0] == 0
    rng = np.random.default_rng(9)
    for R in (1, 7, 64):
        for level in range(Hc.nlevels - 1):
            inf = Hc.info(level)
            N, b = inf["N"], inf["b"]
            xs = rng.standard_normal((R, N * b)).astype(np.float32)
            xb = torch.tensor(_batch_layout(xs, N, b).reshape(-1), device="cuda")
            for which in (lib.MAT_A, lib.MAT_B, lib.MAT_BT):
                yc = Hc.level_apply_batched(level, which, xb, R)
                yu = Hu.level_apply_batched(level, which, xb, R)
                rp, col, vals = Hc.export_level(level, which)
                ref = _batch_layout((bsr_to_dense(rp, col, vals) @ xs.astype(np.float64).T).T, N, b).reshape(-1)
                scale = np.abs(ref).max()
                assert np.abs(yc.cpu().numpy() - ref).max() <= 1e-5 * scale, (R, level, which)
                assert float((yc - yu).abs().max()) <= 2e-5 * scale, (R, level, which)
                if R == 64:
                    y1 = Hc.level_apply_batched(level, which, xb.view(N, R, b)[:, :1, :].contiguous().view(-1), 1)
                    assert torch.equal(y1.view(N, b), yc.view(N, R, b)[:, 0, :]), (level, which)
        X = torch.tensor(rng.standard_normal((R, op.size)), device="cuda")
        op.project_kernel(X)
        V64 = H64.vcycle(X)
        ec = float((Hc.vcycle(X) - V64).abs().max() / V64.abs().max())
        eu = float((Hu.vcycle(X) - V64).abs().max() / V64.abs().max())
        print(f"\nR = {R}: V-cycle error vs FP64, cached {ec:.2e}, per-use {eu:.2e}")
        assert ec <= 2.0 * eu + 1e-6
    torch.cuda.synchronize()


def test_stacked_apply_and_vcycle_equal_single(lib):
    d, n, p = 2, 8, 3
    op = lib.Operator(d, n, p)
    H = lib.Hierarchy(op, smoother="sai", precision="bf16", max_rhs=4)
    gen = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn(4, op.size, dtype=torch.float64, device="cuda", generator=gen)
    op.project_kernel(X)
    Y = op.apply(X)
    V = H.vcycle(X)
    for r in range(4):
        assert torch.equal(Y[r], op.apply(X[r].clone()))
        assert torch.equal(V[r], H.vcycle(X[r].clone()))


@pytest.mark.parametrize("prec,d,n,p,mu_kind,outer", [
    ("bf16", 2, 16, 3, None, "auto"), ("bf16", 3, 6, 3, None, "auto"), ("bf16", 2, 16, 3, "square100", "auto"),
    ("fp32", 2, 16, 3, None, "auto"), ("fp32", 3, 6, 3, None, "fp64"), ("fp32", 2, 32, 3, "square", "auto"),
    ("fp32", 2, 16, 3, None, "df")])
def test_batched_solve_equals_alone_and_oracle(lib, prec, d, n, p, mu_kind, outer):
    """outer = auto picks the double-FP32 outer apply for mu == 1 and FP64 for
    the contrast cases; fp64 / df force one of them."""
    mu = None if mu_kind is None else square_mu(d, n, mu_in=1e2 if mu_kind == "square100" else 1e4)
    N, b = n ** d, (p + 1) ** d
    R = 20 if d == 2 else 6         # 20 x 16 outputs per block row: several per thread in the FP64-level apply
    rhs = np.stack([ldg.project_out_constant(random_rhs(N, b, seed=100 + r), d, p, N) for r in range(R)])
    op = lib.Operator(d, n, p, mu)
    H = lib.Hierarchy(op, smoother="sai", precision=prec, max_rhs=R, outer=outer)
    X, its, res, st = H.solve(torch.tensor(rhs, device="cuda"))
    assert st == lib.OK
    assert max(res) <= 1.05e-10
    levels = mg.build_levels(d, n, p, mu)
    V = mg.VCycle(levels, "sai", 3, 3)
    for r in (range(R) if R <= 6 else (0, 7, R - 1)):
        xa, ka, ra, sa = H.solve(torch.tensor(rhs[r], device="cuda"))
        assert sa == lib.OK and ka == its[r]
        assert torch.equal(xa, X[r]), r           # alone == in the batch, bit for bit
        xo, ko, _ = krylov.pcg(levels[0].A.mat, V, rhs[r], tol=1e-12)
        xg = ldg.project_out_constant(X[r].cpu().numpy(), d, p, N)
        xo = ldg.project_out_constant(xo, d, p, N)
        assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)
    print(f"\nbatched {prec} d={d} n={n} p={p} mu={mu_kind}: iterations {its}")


def test_multi_rhs_without_tensor_cores_and_limits(lib):
    """max_rhs > 1 off the tensor-core path (b = 9; FP16 storage; Gauss-Seidel)
    runs the CUDA-core kernels with one grid row per right-hand side: each
    right-hand side is bitwise the same alone and in the batch.  nrhs above
    max_rhs and Stokes operators with max_rhs > 1 are rejected."""
    for d, n, p, kw in ((2, 8, 2, dict(smoother="sai", precision="bf16")),
                        (2, 8, 3, dict(smoother="sai", precision="fp16")),
                        (2, 8, 2, dict(smoother="gs", precision="fp32"))):
        op = lib.Operator(d, n, p)
        H = lib.Hierarchy(op, max_rhs=4, **kw)
        N, b = n ** d, (p + 1) ** d
        B = np.stack([ldg.project_out_constant(random_rhs(N, b, seed=60 + r), d, p, N) for r in range(3)])
        Xb, kb, rb, st = H.solve(torch.tensor(B, device="cuda"), tol=1e-10)
        assert st == lib.OK and max(rb) <= 1.05e-10
        x1, k1, r1, s1 = H.solve(torch.tensor(B[1], device="cuda"), tol=1e-10)
        assert s1 == lib.OK and k1 == kb[1]
        assert np.array_equal(x1.cpu().numpy(), Xb[1].cpu().numpy())
    op3 = lib.Operator(2, 8, 3)
    H = lib.Hierarchy(op3, smoother="sai", precision="bf16", max_rhs=2)
    with pytest.raises(lib.LdgmgError):
        H.solve(torch.zeros(3, op3.size, dtype=torch.float64, device="cuda"))
    with pytest.raises(lib.LdgmgError) as e:
        lib.Hierarchy(lib.Operator(2, 8, 2, stokes=0), precision="fp32", max_rhs=2)
    assert e.value.status == lib.EUNSUPPORTED

def test_autotuned_launch_shape_does_not_change_results(lib):
    """The setup-time autotuner picks the tensor-core apply's shape by timing
    (the cached kernel's strip width for 2D b = 16, CTAs per SM of the per-use
    kernel otherwise); the apply's result does not depend on it, so two
    hierarchies that may have tuned differently give bitwise equal solves."""
    d, n, p, R = 2, 32, 3, 16
    N, b = n * n, (p + 1) ** 2
    op = lib.Operator(d, n, p)
    H1 = lib.Hierarchy(op, smoother="sai", precision="fp32", max_rhs=R)
    H2 = lib.Hierarchy(op, smoother="sai", precision="fp32", max_rhs=R)
    c1, t1 = H1.tuning
    strip, slots, lpr = H1.tc_schedule
    assert strip in (4, 8, 16) and slots >= 8 and 1.0 <= lpr < 5.0 and t1 > 0.0
    rhs = np.stack([ldg.project_out_constant(random_rhs(N, b, seed=80 + r), d, p, N) for r in range(R)])
    X1, k1, _, s1 = H1.solve(torch.tensor(rhs, device="cuda"))
    X2, k2, _, s2 = H2.solve(torch.tensor(rhs, device="cuda"))
    assert s1 == s2 == lib.OK and k1 == k2 and torch.equal(X1, X2)
    print(f"\ntuned CTAs per SM: {H1.tuning} / {H2.tuning}")


def test_bounded_wait_gives_up_and_context_stays_usable(lib):
    """A device wait on an mbarrier that nothing arrives on gives up after the
    tensor-core kernel's spin limit (each try capped at ~1 us) and reports
    ETIMEOUT; the CUDA context stays usable afterwards."""
    import time
    t0 = time.time()
    assert lib.selftest_bounded_wait() == lib.ETIMEOUT
    assert time.time() - t0 < 30.0
    op = lib.Operator(2, 4, 1)
    x = torch.randn(op.size, dtype=torch.float64, device="cuda")
    y = op.apply(x)
    ref = op.apply(x.clone())
    assert torch.equal(y, ref) and torch.isfinite(y).all()
