"""Grouped solves (ldgmg_solve_group): many small problems of different
classes (mesh, degree, coefficient field, smoother, V-cycle precision) in one
launch per cluster size, each a whole CG solve with the V-cycle of Algorithm 1
(Sec. 2.2) run by one thread-block cluster.

  * First CG iterate x_1 = alpha V b (max_iter = 1; FP64) element-wise against
    the oracle's V-cycle and CG step: this pins every step of the in-kernel
    V-cycle (smoother, restriction, prolongation, bottom solve) for SAI,
    Jacobi and Gauss-Seidel, 2D and 3D, every cluster size.
  * Whole solves of a mixed group against ldgmg_solve of each problem alone:
    iteration counts within one, the true residual (recomputed by ldgmg_apply)
    at tol, A (x - x_alone) within the two residuals; one kernel launch per
    cluster size.
  * Host buffers, repeated hierarchies, a zero right-hand side, a non-finite
    right-hand side (EINVAL for that problem only), max_iter (ENOTCONV), and
    refusal of hierarchies the grouped kernel does not take.
"""
import numpy as np
import pytest

from oracle import ldg
from oracle import multigrid as mg
from paper_2412_12506_gb300.inputs import random_rhs, square_mu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg   # raises if libldgmg.so is missing
    return ldgmg


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def mu_of(d, n, contrast):
    return None if contrast is None else square_mu(d, n, mu_in=contrast)


def consistent_rhs(d, n, p, seed):
    N, b = n ** d, (p + 1) ** d
    return ldg.project_out_constant(random_rhs(N, b, seed=seed), d, p, N)


# (d, n, p, contrast, smoother, precision); the unknowns N b set the cluster
# size (about 1024 per CTA): 1, 2, 4, 4, 8, 8, 8, 8
CLASSES = [
    (2, 16, 1, None, "sai", "fp64"),       # 1024 unknowns
    (2, 8, 4, 1e2, "sai", "fp32"),         # 1600
    (3, 8, 1, None, "jacobi", "fp64"),     # 4096
    (2, 16, 3, None, "gs", "fp32"),        # 4096
    (2, 32, 2, 1e4, "sai", "fp32"),        # 9216
    (2, 16, 4, None, "sai", "bf16"),       # 6400
    (2, 32, 4, 1e4, "sai", "fp32"),        # 25600
    (3, 8, 2, None, "sai", "fp64"),        # 13824
]
CLUSTERS = [1, 2, 4, 4, 8, 8, 8, 8]

_H = {}


def hier(lib, d, n, p, contrast, smoother, prec, **kw):
    key = (d, n, p, contrast, smoother, prec, tuple(sorted(kw.items())))
    if key not in _H:
        op = lib.Operator(d, n, p, mu_of(d, n, contrast))
        _H[key] = lib.Hierarchy(op, smoother=smoother, precision=prec, nu1=3, nu2=3, **kw)
    return _H[key]


def test_cluster_sizes(lib):
    for cls, c in zip(CLASSES, CLUSTERS):
        assert lib.Group.cluster(hier(lib, *cls)) == c, cls


@pytest.mark.parametrize("d,n,p,contrast,smoother", [
    (2, 16, 1, None, "sai"), (2, 8, 3, 1e4, "sai"), (3, 4, 3, None, "sai"), (2, 16, 2, None, "jacobi"),
    (3, 8, 1, None, "jacobi"), (2, 16, 3, None, "gs"), (3, 4, 2, 1e2, "gs"), (2, 16, 4, None, "sai")])
def test_first_iterate_matches_oracle(lib, d, n, p, contrast, smoother):
    """max_iter = 1: x_1 = alpha z, z = V b, alpha = (b . z) / (z . A z) (Sec. 2.2)."""
    mu = mu_of(d, n, contrast)
    levels = mg.build_levels(d, n, p, mu)
    V = mg.VCycle(levels, smoother, 3, 3)
    b = consistent_rhs(d, n, p, seed=3)
    z = V(b)
    A = levels[0].A.mat
    x1 = (b @ z) / (z @ (A @ z)) * z
    H = hier(lib, d, n, p, contrast, smoother, "fp64", max_iter=1)
    g = lib.Group()
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    it, rr, st = g.solve([(H, torch.tensor(b, device="cuda"), x, 1e-10)], check=False)
    assert st == [lib.ENOTCONV] and it == [1]
    # SAI blocks from the device least squares agree with LAPACK's to ~1e-12
    # (1e-10 with a coefficient jump); the V-cycle inherits that
    tol = 1e-10 if (smoother == "sai" and contrast) else 1e-11
    assert rel(x.cpu().numpy(), x1) < tol
    res = np.linalg.norm(b - A @ x1) / np.linalg.norm(b)
    assert abs(rr[0] - res) <= 1e-9 * res


def test_mixed_group_matches_individual_solves(lib):
    probs, ref = [], []
    for k, cls in enumerate(CLASSES):
        d, n, p = cls[:3]
        H = hier(lib, *cls)
        for j in range(2):
            b = torch.tensor(consistent_rhs(d, n, p, seed=100 + 2 * k + j), device="cuda")
            xs, ks, rrs, sts = H.solve(b.clone(), 1e-10)
            assert sts == lib.OK
            ref.append((xs.clone(), ks, rrs))
            probs.append((H, b, torch.zeros_like(b), 1e-10))
    g = lib.Group()
    l0 = lib.kernel_launches()
    it, rr, st = g.solve(probs)
    assert lib.kernel_launches() - l0 == len(set(CLUSTERS))
    for (H, b, x, _), (xs, ks, rrs), k, r, s in zip(probs, ref, it, rr, st):
        assert s == lib.OK
        assert abs(k - ks) <= 1, (k, ks)
        y = H.op.apply(x)
        true = float(torch.linalg.norm(b - y) / torch.linalg.norm(b))
        assert r <= 1.05e-10 and true <= 1.05e-10
        # the two FP64 residuals differ by their rounding, ~eps |A| |x| / |b|
        # (up to ~1e-13 at contrast 1e4), not by a relative amount
        assert abs(true - r) <= 1e-3 * r + 1e-12
        # both iterates meet tol, so A (x - xs) is at most the sum of their
        # residuals; x - xs itself is that times the conditioning (up to ~1e7
        # at contrast 1e4), checked only for gross disagreement
        dA = float(torch.linalg.norm(H.op.apply(x - xs)) / torch.linalg.norm(b))
        assert dA <= r + rrs + 1e-14
        assert float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs)) < 1e-4


def test_host_buffers_repeats_and_special_cases(lib):
    cls = (2, 16, 2, 1e2, "sai", "fp32")
    d, n, p = cls[:3]
    H = hier(lib, *cls)
    H2 = hier(lib, *CLASSES[4])
    b1 = torch.tensor(consistent_rhs(d, n, p, seed=5))              # host
    b2 = torch.tensor(consistent_rhs(d, n, p, seed=6), device="cuda")
    bz = torch.zeros(b1.numel(), dtype=torch.float64)             # zero rhs
    bn = b1.clone()
    bn[7] = float("nan")                                          # non-finite rhs
    d2, n2, p2 = CLASSES[4][:3]
    b3 = torch.tensor(consistent_rhs(d2, n2, p2, seed=7))
    xs = [torch.full_like(b1, 5.0), torch.zeros_like(b2), torch.full_like(bz, 3.0), torch.zeros_like(bn),
          torch.zeros_like(b3)]
    probs = [(H, b1, xs[0], 1e-10), (H, b2, xs[1], 1e-10), (H, bz, xs[2], 1e-10), (H, bn, xs[3], 1e-10),
             (H2, b3, xs[4], 1e-9)]
    g = lib.Group()
    it, rr, st = g.solve(probs, check=False)
    assert st == [lib.OK, lib.OK, lib.OK, lib.EINVAL, lib.OK]
    assert it[2] == 0 and rr[2] == 0.0 and float(xs[2].abs().max()) == 0.0
    assert rr[4] <= 1.05e-9
    xa, ka, _, _ = H.solve(b1.cuda(), 1e-10)
    assert abs(it[0] - ka) <= 1
    assert float(torch.linalg.norm(xs[0].cuda() - xa) / torch.linalg.norm(xa)) < 1e-4
    # the same problem twice in one group gives the same result
    x5, x6 = torch.zeros_like(b2), torch.zeros_like(b2)
    it2, _, _ = g.solve([(H, b2, x5, 1e-10), (H, b2, x6, 1e-10)])
    assert torch.equal(x5, x6) and torch.equal(x5, xs[1]) and it2 == [it[1], it[1]]


def test_max_iter_and_refusals(lib):
    H = hier(lib, 2, 16, 2, None, "sai", "fp32", max_iter=3)
    b = torch.tensor(consistent_rhs(2, 16, 2, seed=9), device="cuda")
    x = torch.zeros_like(b)
    it, rr, st = lib.Group().solve([(H, b, x, 1e-10)], check=False)
    assert st == [lib.ENOTCONV] and it == [3] and 0 < rr[0] < 1
    with pytest.raises(lib.LdgmgError):
        lib.Group().solve([(H, b, x, 0.0)])
    # a tensor-core (batched) hierarchy and a Stokes hierarchy are refused
    op = lib.Operator(2, 16, 3)
    Hb = lib.Hierarchy(op, smoother="sai", precision="fp32", max_rhs=8)
    assert lib.Group.cluster(Hb) == 0
    b16 = torch.tensor(consistent_rhs(2, 16, 3, seed=2), device="cuda")
    with pytest.raises(lib.LdgmgError) as e:
        lib.Group().solve([(Hb, b16, torch.zeros_like(b16), 1e-10)])
    assert e.value.status == lib.EUNSUPPORTED
    Hs = lib.Hierarchy(lib.Operator(2, 8, 2, stokes=1), smoother="sai")
    assert lib.Group.cluster(Hs) == 0
