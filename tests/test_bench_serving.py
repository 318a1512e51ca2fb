"""Host flows of bench.py on the CPU: the serving pass and the linear-solve
timing.  The device calls are replaced by host fakes (a runner that sleeps in
proportion to a request's unknowns, host events), so the saturated pass, the
rate rule and the fields of the JSON line are checked without a GPU."""

import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_serving_pass_fields_and_rate_rule(monkeypatch, tmp_path):
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
    log = tmp_path / "requests.jsonl"
    f = bench.serving_pass(12, 0.0, 4, 0, clocks=False, log_path=str(log))
    import json
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [x["id"] for x in lines] == list(range(12))
    assert all(x["status"] == "done" and x["done_s"] >= x["admitted_s"] >= 0.0 for x in lines)
    assert all(x["n_dof"] == W.n_dofs(dict(x, d=2)) for x in lines)
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


def test_linear_solve_timing_flow(monkeypatch):
    """bench.time_linear_solve on the CPU: device tensors and events replaced
    by host fakes; the frozen linearization is taken once, every solve starts
    from the saved iterate, and the untimed first solve is left out."""
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench

    zeros = torch.zeros
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: zeros(*a, **{x: v for x, v in k.items() if x != "device"}))

    class Event:
        clock = [0.0]

        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            Event.clock[0] += 1.0
            self.t = Event.clock[0]

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(torch.cuda, "Event", Event)

    class Solver:
        def __init__(self):
            self.calls = []

        def rhs(self, f):
            self.calls.append("rhs")

        def linearize(self, u, w, kind):
            self.calls.append(("linearize", kind))

        def linsolve(self, b, x, allow_unconverged=False):
            self.calls.append("linsolve")
            return dict(gmres_iters=11, outer_iters=2, rel_res=3e-9)

    u2 = torch.arange(5, dtype=torch.float64)
    s = Solver()
    out = bench.time_linear_solve(s, u2, u2 * 0, None, 3)
    assert s.calls == ["rhs", ("linearize", "picard")] + ["linsolve"] * 4
    assert out["ms"] == pytest.approx(1.0) and out["dof_per_s"] == pytest.approx(5 / 1e-3)
    assert out["gmres_iters"] == 11 and out["outer_iters"] == 2 and out["rel_res"] == 3e-9
