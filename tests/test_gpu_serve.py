"""The serving engine on the GPU: real solves through ldgmg_server_*.

  * A request's result is bitwise the same served alone and served in a mix
    with other classes and with copies of itself batched together.
  * Every result reaches the requested relative residual; one class is
    compared with the FP64 oracle solution (error below 1e-7, as for the
    mixed-precision solves of test_gpu_parity.py).
  * Admission under a budget that holds about one class: classes are evicted
    and rebuilt, results stay correct and bitwise repeatable.
"""
import numpy as np
import pytest

from oracle import krylov, ldg
from oracle import multigrid as mg
from oracle import stokes as st
from paper_2412_12506_gb300.inputs import random_rhs, square_mu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


CLASSES = [
    # (dim, n, p, stokes, mu)
    (2, 32, 3, None, "square"),    # b = 16: batched tensor-core class
    (2, 16, 2, None, None),        # b = 9
    (3, 8, 3, None, None),         # b = 64: batched
    (2, 8, 2, 1, None),            # Stokes stress form, GMRES
]


def _mu(dim, n, kind):
    return None if kind is None else square_mu(dim, n, mu_in=1e4)


def _rhs(dim, n, p, stokes, seed):
    N = n ** dim
    if stokes is None:
        return ldg.project_out_constant(random_rhs(N, (p + 1) ** dim, seed=seed), dim, p, N)
    return st.project_out_kernel(random_rhs(N, (dim + 1) * (p + 1) ** dim, seed=seed), dim, p, N)


def test_alone_equals_mix_and_accuracy(lib):
    s = lib.Server(workers=3, max_batch=16, precision="fp32")
    alone = {}
    for ci, (d, n, p, sk, mk) in enumerate(CLASSES):
        t = s.submit(d, n, p, _rhs(d, n, p, sk, 100 + ci), mu=_mu(d, n, mk), stokes=sk)
        x, r = s.wait(t)
        assert r["status"] == lib.OK and r["relres"] <= 1.05e-10 and r["batch"] == 1, r
        alone[ci] = x.copy()
    # the mix: every class several times, own right-hand side repeated among others
    order = []
    rng = np.random.default_rng(0)
    for k in range(40):
        ci = int(rng.integers(len(CLASSES)))
        d, n, p, sk, mk = CLASSES[ci]
        same = k % 3 == 0
        seed = 100 + ci if same else 1000 + k
        order.append((ci, same, s.submit(d, n, p, _rhs(d, n, p, sk, seed), mu=_mu(d, n, mk), stokes=sk)))
    batches = []
    for ci, same, t in order:
        x, r = s.wait(t)
        assert r["status"] == lib.OK and r["relres"] <= 1.05e-10, r
        batches.append(r["batch"])
        if same:
            assert np.array_equal(x, alone[ci]), ci
    assert max(batches) > 1
    stats = s.stats()
    assert stats["completed"] == stats["submitted"] == 44 and stats["builds"] == len(CLASSES)
    s.close()
    # accuracy of one class against the FP64 oracle
    d, n, p, sk, mk = CLASSES[1]
    rhs = _rhs(d, n, p, sk, 101)
    levels = mg.build_levels(d, n, p)
    xo, _, _ = krylov.pcg(levels[0].A.mat, mg.VCycle(levels, "sai", 3, 3), rhs, tol=1e-12)
    N = n ** d
    err = np.linalg.norm(ldg.project_out_constant(alone[1], d, p, N) - ldg.project_out_constant(xo, d, p, N))
    assert err <= 1e-7 * np.linalg.norm(xo)


def test_admission_under_a_small_budget(lib):
    d, n, p = 2, 32, 2
    probe = lib.Server(workers=1, max_batch=1, precision="fp32")
    t = probe.submit(d, n, p, _rhs(d, n, p, None, 1))
    x_ref, _ = probe.wait(t)
    one = probe.stats()["bytes_resident"]
    probe.close()
    assert one > 0
    s = lib.Server(workers=2, max_batch=1, hbm_budget=int(one * 1.5), precision="fp32")
    mus = [None, np.full(n * n, 2.0), np.full(n * n, 3.0)]     # three classes of one size
    tickets = [(k, s.submit(d, n, p, _rhs(d, n, p, None, 1), mu=mus[k])) for rep in range(3) for k in range(3)]
    outs = {}
    for k, t in tickets:
        x, r = s.wait(t)
        assert r["status"] == lib.OK and r["relres"] <= 1.05e-10
        if k in outs:
            assert np.array_equal(x, outs[k])       # rebuilt classes give the same result
        outs[k] = x
    assert np.array_equal(outs[0], x_ref)
    stats = s.stats()
    assert stats["evictions"] >= 1 and stats["bytes_peak"] <= int(one * 1.5)
    s.close()


def test_reduced_precision_class_falls_back_to_fp64(lib):
    """A 3D p = 3 interface class with contrast 1e4 does not converge with an
    FP32 V-cycle (its SAI blocks span the contrast); the engine rebuilds that
    class once with an FP64 V-cycle and solves its requests again, so every
    request still reaches the tolerance.  A class that converges in FP32 keeps
    its FP32 hierarchy."""
    d, n, p = 3, 16, 3
    N, b = n ** d, (p + 1) ** d
    mu = square_mu(d, n, mu_in=1e4)
    s = lib.Server(workers=2, max_batch=4, precision="fp32", max_iter=200)
    rhs = [ldg.project_out_constant(random_rhs(N, b, seed=300 + k), d, p, N) for k in range(3)]
    tickets = [s.submit(d, n, p, r, mu=mu, tol=1e-10) for r in rhs]
    t_ok = s.submit(2, 16, 2, ldg.project_out_constant(random_rhs(256, 9, seed=9), 2, 2, 256), tol=1e-10)
    for t in tickets:
        _, r = s.wait(t)
        assert r["status"] == lib.OK and r["relres"] <= 1.05e-10, r
    assert s.wait(t_ok)[1]["status"] == lib.OK
    assert s.stats()["precision_fallbacks"] == 1
    s.close()


def test_grouped_small_classes(lib):
    """Small scalar classes (group_dofs) are served by grouped calls; each
    result meets tol and is bitwise the same alone and in a mixed group (a
    problem's arithmetic depends only on its own class and data)."""
    small = [(2, 16, 1, None), (2, 16, 2, "square"), (3, 8, 1, None), (2, 32, 4, "square"), (2, 16, 3, None)]
    s = lib.Server(workers=2, max_batch=16, precision="fp32", group_dofs=32768, group_max=64)
    alone = {}
    for ci, (d, n, p, mk) in enumerate(small):
        x, r = s.wait(s.submit(d, n, p, _rhs(d, n, p, None, 200 + ci), mu=_mu(d, n, mk)))
        assert r["status"] == lib.OK and r["relres"] <= 1.05e-10 and r["batch"] == 1, r
        alone[ci] = x.copy()
    order = []
    rng = np.random.default_rng(1)
    for k in range(60):
        ci = int(rng.integers(len(small) + 1))
        if ci == len(small):       # a larger class with its own calls
            order.append((ci, False, s.submit(2, 64, 3, _rhs(2, 64, 3, None, 3000 + k))))
            continue
        d, n, p, mk = small[ci]
        same = k % 4 == 0
        seed = 200 + ci if same else 2000 + k
        order.append((ci, same, s.submit(d, n, p, _rhs(d, n, p, None, seed), mu=_mu(d, n, mk))))
    nsmall = len(small) + sum(1 for ci, _, _ in order if ci < len(small))
    batches = []
    for ci, same, t in order:
        x, r = s.wait(t)
        assert r["status"] == lib.OK and r["relres"] <= 1.05e-10, r
        if ci < len(small):
            batches.append(r["batch"])
        if same:
            assert np.array_equal(x, alone[ci]), ci
    st_ = s.stats()
    assert st_["group_requests"] == nsmall
    assert st_["group_calls"] < nsmall and max(batches) > 1
    s.close()
