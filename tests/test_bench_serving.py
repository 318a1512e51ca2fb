"""Host flow of bench.py's serving pass on the CPU: the device calls are
replaced by host fakes (a runner that sleeps in proportion to a request's
unknowns), so the saturated pass, the rate rule and the fields of the JSON
line are checked without a GPU."""

import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_serving_pass_fields_and_rate_rule(monkeypatch):
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    from paper_2311_17500_gb300 import serve

    def fake_runner(desc_of, keep_solution=False, device=None):
        def run(req):
            n = W.n_dofs(desc_of(req))
            time.sleep(1e-9 * n)
            return dict(stats=dict(total_gmres=7), n_dof=n)
        return run

    monkeypatch.setattr(serve, "gpu_runner", fake_runner)
    monkeypatch.setattr(serve, "gpu_footprint", lambda desc_of: (lambda r: 1 << 20))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a, **k: (64 << 20, 128 << 20))
    f = bench.serving_pass(12, 0.0, 4, 0, clocks=False)
    cfg = f["config"]
    assert f["done"] == 12 and f["failed"] == 0 and f["rejected"] == 0
    sat = cfg["saturated"]
    assert sat["done"] == 12
    assert cfg["arrival_rate_per_s"] == pytest.approx(0.8 * sat["requests_per_s"])
    assert cfg["rate_rule"].startswith("0.8")
    assert f["latency_ms"]["p99"] >= f["latency_ms"]["p50"] > 0.0
    assert f["queue_ms"]["p99"] >= f["queue_ms"]["p50"] >= 0.0
    assert f["value"] > 0.0 and cfg["gmres_iters_mean"] == 7
    assert cfg["peak_admitted_gb"] * 1e9 <= cfg["budget_gb"] * 1e9 + 1
    given = bench.serving_pass(6, 50.0, 2, 0, clocks=False)
    assert given["config"]["rate_rule"] == "given" and given["config"]["saturated"] is None
