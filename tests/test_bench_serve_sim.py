"""bench.py's serving section end to end on the CPU: the real scheduler in
simulate mode (timed stand-ins for builds and solves, no device work) driven
by the section's own stream, comparison arms and summaries, so the JSON it
reports keeps its shape without a GPU."""
import json
import sys

import numpy as np
import pytest


def test_serve_section_shape(monkeypatch):
    from paper_2412_12506_gb300 import ldgmg
    monkeypatch.setattr(sys, "argv", ["bench.py", "--serve-requests", "120", "--serve-fp64-prefix", "40"])
    import bench

    class SimServer(ldgmg.Server):
        def __init__(self, *a, **kw):
            kw.update(simulate=True, simulate_solve_s=0.001, hbm_budget=1 << 40)
            super().__init__(*a, **kw)

    class Lib:
        pass

    lib = Lib()
    for k in dir(ldgmg):
        if not k.startswith("__"):
            setattr(lib, k, getattr(ldgmg, k))
    lib.Server = SimServer
    out = bench.run_serve(bench.parse(), lib, None, np, None, None, lambda: None)
    json.dumps(out)
    assert out["requests"] == 120 and out["classes"] > 0
    for arm in ("same_prefix", "ungrouped_same_prefix", "fp64_one_at_a_time"):
        assert out[arm]["requests"] == 40
        assert set(out[arm]["latency_ms"]) == {"p50", "p99"}
    sizes = out["by_size"]
    assert sum(v["requests"] for v in sizes.values()) == 120
    assert out["small_requests"] == sizes.get("small_le_16k", {"requests": 0})["requests"]
    # simulated solves carry no residual: nothing counts as reaching tol
    assert out["reached_tol"] == 0
