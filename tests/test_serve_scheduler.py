"""The serving engine's scheduler (include/ldgmg_serve.h) on the CPU.

The server runs with simulate = 1: the real scheduler, builder and worker
threads, class cache, admission, eviction and batching, with timed stand-ins
for builds and solves (no device work, no results).  The GPU behaviour --
real solves, alone-vs-mix equality -- is tested in test_gpu_serve.py.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


def _rhs(dim, n, p, stokes=None):
    b = (p + 1) ** dim * (1 if stokes is None else dim + 1)
    return np.zeros(n ** dim * b)


def test_all_requests_complete_and_batch_per_class(lib):
    # simulated solves slower than the submissions (which copy up to 13 MB of
    # right-hand side each), so that requests queue up behind running solves
    s = lib.Server(workers=2, max_batch=8, hbm_budget=1 << 40, simulate=True, simulate_solve_s=0.05,
                   precision="fp32")
    tickets = []
    # scalar classes take batches (capped at 2^22 dofs per call: the 256^2 p = 4
    # class takes at most 2); Stokes (GMRES) takes one right-hand side per call
    for i in range(48):
        if i % 4 == 0:
            tickets.append(("b16", s.submit(2, 16, 3, _rhs(2, 16, 3))))
        elif i % 4 == 1:
            tickets.append(("b9", s.submit(2, 16, 2, _rhs(2, 16, 2))))
        elif i % 4 == 2:
            tickets.append(("stokes", s.submit(2, 8, 2, _rhs(2, 8, 2, 1), stokes=1)))
        else:
            tickets.append(("big", s.submit(2, 256, 4, _rhs(2, 256, 4))))
    res = {kind: [] for kind in ("b16", "b9", "stokes", "big")}
    for kind, t in tickets:
        _, r = s.wait(t)
        assert r["status"] == lib.OK and r["iters"] == 0 and np.isnan(r["relres"])
        assert r["t_submit"] <= r["t_start"] <= r["t_end"]
        res[kind].append(r)
    st = s.stats()
    assert st["submitted"] == st["completed"] == 48
    assert st["builds"] == 4 and st["evictions"] == 0 and st["classes_resident"] == 4
    assert all(r["batch"] == 1 for r in res["stokes"])
    assert all(1 <= r["batch"] <= 2 for r in res["big"])
    assert all(1 <= r["batch"] <= 8 for r in res["b16"] + res["b9"])
    assert max(r["batch"] for r in res["b16"]) > 1 and max(r["batch"] for r in res["b9"]) > 1
    assert st["solve_calls"] < 48
    s.close()


def test_admission_by_footprint_evicts_lru(lib):
    # a budget that holds about one 2D 32^2 p = 2 class at a time
    probe = lib.Server(workers=1, max_batch=1, hbm_budget=1 << 40, simulate=True, simulate_solve_s=0.0)
    t = probe.submit(2, 32, 2, _rhs(2, 32, 2))
    probe.wait(t)
    one = probe.stats()["bytes_resident"]
    probe.close()
    budget = int(one * 1.5)
    s = lib.Server(workers=1, max_batch=1, hbm_budget=budget, simulate=True, simulate_solve_s=0.002)
    mus = [np.full(32 * 32, 1.0 + k) for k in range(4)]          # four classes of equal size
    order = []
    for rep in range(3):
        for k in range(4):
            order.append(s.submit(2, 32, 2, _rhs(2, 32, 2), mu=mus[k]))
    for t in order:
        _, r = s.wait(t)
        assert r["status"] == lib.OK
    st = s.stats()
    assert st["completed"] == 12
    assert st["bytes_peak"] <= budget
    assert st["evictions"] >= 3 and st["builds"] == st["evictions"] + st["classes_resident"]
    s.close()


def test_fifo_across_classes_with_one_worker(lib):
    s = lib.Server(workers=1, max_batch=1, hbm_budget=1 << 40, simulate=True, simulate_solve_s=0.003)
    tickets = [s.submit(2, 8, 1 + (i % 3), _rhs(2, 8, 1 + (i % 3))) for i in range(15)]
    starts = [s.wait(t)[1]["t_start"] for t in tickets]
    assert starts == sorted(starts)
    s.close()


def test_class_larger_than_the_budget_is_refused(lib):
    """Admission by footprint holds for every class: one whose estimate alone
    exceeds the budget is never built, its requests (queued and later ones)
    complete with ENOMEM, and classes that fit are still served."""
    probe = lib.Server(workers=1, max_batch=1, hbm_budget=1 << 40, simulate=True, simulate_solve_s=0.0)
    probe.wait(probe.submit(2, 16, 1, _rhs(2, 16, 1)))
    small = probe.stats()["bytes_resident"]
    probe.close()
    s = lib.Server(workers=1, max_batch=1, hbm_budget=small + small // 2, simulate=True, simulate_solve_s=0.0)
    big = [s.submit(2, 64, 3, _rhs(2, 64, 3)) for _ in range(2)]
    ok = s.submit(2, 16, 1, _rhs(2, 16, 1))
    for t in big:
        _, r = s.wait(t)
        assert r["status"] == lib.ENOMEM and np.isnan(r["relres"])
    assert s.wait(ok)[1]["status"] == lib.OK
    _, r = s.wait(s.submit(2, 64, 3, _rhs(2, 64, 3)))
    assert r["status"] == lib.ENOMEM
    st = s.stats()
    assert st["builds"] == 1 and st["build_failures"] == 1 and st["bytes_peak"] <= st["hbm_budget"]
    s.close()


def test_bad_requests(lib):
    s = lib.Server(workers=1, max_batch=1, hbm_budget=1 << 30, simulate=True)
    with pytest.raises(lib.LdgmgError):
        s.submit(4, 8, 1, np.zeros(10))
    with pytest.raises(lib.LdgmgError):
        s.submit(2, 8, 1, _rhs(2, 8, 1), stokes=3)
    with pytest.raises(lib.LdgmgError):
        s.submit(2, 8, 1, _rhs(2, 8, 1), tol=0.0)
    with pytest.raises(lib.LdgmgError):
        s.wait(12345)
    s.close()
    with pytest.raises(lib.LdgmgError):
        lib.Server(workers=0, simulate=True)
    with pytest.raises(lib.LdgmgError):
        lib.Server(max_batch=65, simulate=True)


def test_small_classes_share_grouped_calls(lib):
    # classes with at most group_dofs unknowns are served together: one grouped
    # call takes the oldest queued requests of every ready small class (up to
    # group_max); larger classes keep their own calls; one more worker (the
    # small lane, index `workers`) takes grouped calls only
    s = lib.Server(workers=1, max_batch=8, hbm_budget=1 << 40, simulate=True, simulate_solve_s=0.05,
                   group_dofs=4096, group_max=6, precision="fp32")
    small = [(2, 16, 1), (2, 16, 2), (3, 8, 1), (2, 32, 1)]      # 1024, 2304, 4096, 4096 unknowns
    tickets = []
    for i in range(24):
        d, n, p = small[i % 4]
        tickets.append(("small", (d, n, p), s.submit(d, n, p, _rhs(d, n, p))))
    tickets.append(("big", None, s.submit(2, 32, 2, _rhs(2, 32, 2))))    # 9216 unknowns
    got = []
    for kind, cls, t in tickets:
        _, r = s.wait(t)
        assert r["status"] == lib.OK
        got.append((kind, cls, r))
    st = s.stats()
    assert st["completed"] == 25 and st["builds"] == 5
    assert st["group_requests"] == 24
    assert st["group_calls"] >= 4 and st["group_calls"] < 24
    assert all(r["batch"] <= 6 for kind, _, r in got if kind == "small")
    # the small lane (worker 1) serves grouped calls only
    assert any(r["worker"] == 1 for kind, _, r in got if kind == "small")
    assert all(r["worker"] == 0 for kind, _, r in got if kind == "big")
    # some grouped call served requests of different classes
    calls = {}
    for kind, cls, r in got:
        if kind == "small":
            calls.setdefault((r["t_start"], r["t_end"]), set()).add(cls)
    assert max(len(v) for v in calls.values()) > 1
    # oldest first across classes: grouped calls start in submission order (two
    # workers -- the regular one and the small lane -- may wake up in either
    # order, so a few milliseconds of jitter; serving a later request a whole
    # call before an earlier one would show as an inversion of ~50 ms)
    starts = [r["t_start"] for kind, _, r in got if kind == "small"]
    assert all(b >= a - 0.005 for a, b in zip(starts, starts[1:]))
    s.close()


def test_group_options_are_checked(lib):
    with pytest.raises(lib.LdgmgError):
        lib.Server(workers=1, simulate=True, group_max=70000)


def test_precision_fallback_grouped_and_per_class(lib):
    # simulate_notconv_n = 16: classes with n = 16 "do not converge" while their
    # V-cycle is FP32.  The grouped class (2D 16^2 p = 1, 1,024 unknowns) and the
    # per-class one (2D 16^2 p = 4, 6,400 unknowns) must each be rebuilt once
    # with an FP64 V-cycle and their requests served again, in order; the n = 8
    # class is untouched.
    s = lib.Server(workers=1, max_batch=4, hbm_budget=1 << 40, simulate=True, simulate_solve_s=0.01,
                   group_dofs=4096, precision="fp32", simulate_notconv_n=16)
    order = []
    for i in range(12):
        d, n, p = [(2, 16, 1), (2, 16, 4), (2, 8, 1)][i % 3]
        order.append(((d, n, p), s.submit(d, n, p, _rhs(d, n, p))))
    got = {}
    for cls, t in order:
        _, r = s.wait(t)
        assert r["status"] == lib.OK, (cls, r)
        got.setdefault(cls, []).append(r)
    st = s.stats()
    assert st["completed"] == 12
    assert st["precision_fallbacks"] == 2
    assert st["builds"] == 5                      # 3 classes + 2 FP64 rebuilds
    assert st["group_requests"] == 8              # the 2D 16^2 p = 1 and 8^2 p = 1 requests
    # each class's requests start in submission order
    for rs in got.values():
        starts = [r["t_start"] for r in rs]
        assert all(b >= a - 0.005 for a, b in zip(starts, starts[1:]))
    s.close()
