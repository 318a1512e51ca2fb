"""Host logic of the serving loop (paper_2311_17500_gb300.serve), on the CPU.

The engine is driven with host-only runners that sleep for a request's
"work" and record what was in flight, so that admission by memory, the slot
limit, first-come first-served order, rejection, failure handling and the
latency summary are checked without a GPU.
"""

import threading
import time

import numpy as np
import pytest

import workloads as W
from paper_2311_17500_gb300 import serve


class Probe:
    """A runner that sleeps `work` seconds and records concurrency and bytes in flight."""

    def __init__(self, footprint, fail_ids=()):
        self.footprint = footprint
        self.fail_ids = set(fail_ids)
        self.lock = threading.Lock()
        self.active = 0
        self.bytes = 0
        self.max_active = 0
        self.max_bytes = 0
        self.started = []

    def __call__(self, req):
        fp = self.footprint(req)
        with self.lock:
            self.active += 1
            self.bytes += fp
            self.max_active = max(self.max_active, self.active)
            self.max_bytes = max(self.max_bytes, self.bytes)
            self.started.append(req["id"])
        try:
            time.sleep(req["work"])
            if req["id"] in self.fail_ids:
                raise RuntimeError("injected failure")
            return dict(ok=req["id"])
        finally:
            with self.lock:
                self.active -= 1
                self.bytes -= fp


def stream(n, gap, work, sizes):
    return [dict(id=i, arrival=i * gap, work=work, size=sizes[i % len(sizes)], desc=None) for i in range(n)]


def fp_of(req):
    return req["size"]


def test_all_requests_complete_in_order_of_arrival():
    reqs = stream(8, 0.005, 0.01, [10])
    probe = Probe(fp_of)
    eng = serve.Engine(probe, fp_of, budget_bytes=1000, max_slots=3)
    recs = eng.run(reqs)
    assert [r["status"] for r in recs] == ["done"] * 8
    assert sorted(probe.started) == list(range(8))
    for r in recs:
        assert r["admitted"] >= r["arrival"] - 1e-3
        assert r["done"] >= r["admitted"] + 0.009
        assert r["result"] == dict(ok=r["id"])
    adm = [r["admitted"] for r in recs]
    assert adm == sorted(adm)                          # first come, first served


def test_memory_budget_and_slot_limit_hold():
    # every request arrives at once; sizes 40/70/30: at most 100 bytes may run together
    reqs = stream(12, 0.0, 0.01, [40, 70, 30])
    probe = Probe(fp_of)
    eng = serve.Engine(probe, fp_of, budget_bytes=100, max_slots=3)
    recs = eng.run(reqs)
    assert all(r["status"] == "done" for r in recs)
    assert probe.max_bytes <= 100
    assert probe.max_active <= 3
    assert eng.peak_bytes <= 100
    adm = [r["admitted"] for r in recs]
    assert adm == sorted(adm)                          # admitted in arrival order


def test_oversized_request_is_rejected_without_blocking():
    reqs = stream(5, 0.002, 0.005, [10])
    reqs[2]["size"] = 500
    probe = Probe(fp_of)
    recs = serve.Engine(probe, fp_of, budget_bytes=100, max_slots=2).run(reqs)
    assert recs[2]["status"] == "rejected" and "exceeds the budget" in recs[2]["error"]
    assert [r["status"] for i, r in enumerate(recs) if i != 2] == ["done"] * 4
    assert 2 not in probe.started


def test_failed_request_releases_its_memory():
    # a budget for one request at a time: a failure must not stall the rest
    reqs = stream(4, 0.0, 0.005, [60])
    probe = Probe(fp_of, fail_ids={1})
    recs = serve.Engine(probe, fp_of, budget_bytes=100, max_slots=4).run(reqs)
    assert [r["status"] for r in recs] == ["done", "failed", "done", "done"]
    assert "injected failure" in recs[1]["error"]
    assert probe.max_active == 1


def test_summary_percentiles_and_throughput():
    recs = [dict(id=i, arrival=0.0, admitted=0.1 * i, done=0.1 * i + 1.0, status="done") for i in range(10)]
    recs.append(dict(id=10, arrival=0.0, admitted=None, done=0.0, status="rejected"))
    out = serve.summary(recs, n_dofs=lambda r: 100)
    lat = np.array([0.1 * i + 1.0 for i in range(10)])
    assert out["done"] == 10 and out["rejected"] == 1 and out["failed"] == 0
    assert out["p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert out["p99_s"] == pytest.approx(np.percentile(lat, 99))
    assert out["makespan_s"] == pytest.approx(1.9)
    wait = np.array([0.1 * i for i in range(10)])
    assert out["queue_p50_s"] == pytest.approx(np.percentile(wait, 50))
    assert out["queue_p99_s"] == pytest.approx(np.percentile(wait, 99))
    assert out["dof_per_s"] == pytest.approx(1000 / 1.9)


def test_n_unknowns_matches_the_workload_count():
    for req in W.serving_requests(n_req=6, seed=11):
        assert serve.n_unknowns(req["desc"]) == W.n_dofs(req["desc"])


def test_serving_stream_is_seeded_and_in_range():
    a = W.serving_requests(n_req=64, seed=4, rate=2.0)
    b = W.serving_requests(n_req=64, seed=4, rate=2.0)
    assert [r["desc"] for r in a] == [r["desc"] for r in b]
    arr = [r["arrival"] for r in a]
    assert arr == sorted(arr) and arr[0] > 0.0
    for r in a:
        d = r["desc"]
        assert d["d"] == 2 and d["p"] in (2, 3)
        assert all(32 <= n <= 256 for n in d["n_el"]) and 64 <= d["n_el_t"] <= 512
        assert 2e-4 <= d["D"][0] <= 2e-3 and d["D"][0] == d["D"][1]
        box = d["source"]["boxes"][0]
        assert 0.0 <= box["lo"][0] <= 0.9 and box["hi"][0] == pytest.approx(box["lo"][0] + 0.1)


def test_arrival_rate_scales_the_same_requests():
    """Exponential gaps scale with 1/rate and the shapes do not depend on the
    rate, so a stream can be replayed at a rate measured from its own
    saturated pass."""
    one = W.serving_requests(n_req=32, seed=4, rate=1.0)
    for rate in (0.5, 3.0, 17.0):
        r = W.serving_requests(n_req=32, seed=4, rate=rate)
        assert [a["desc"] for a in r] == [a["desc"] for a in one]
        assert np.allclose([a["arrival"] * rate for a in r], [a["arrival"] for a in one], rtol=1e-12)


class Transient(RuntimeError):
    pass


def test_retryable_failure_runs_again_after_a_completion():
    # request 1 fails once (as if device memory were held elsewhere) while 0
    # runs; the others run long enough for that failure to be seen first
    reqs = stream(3, 0.0, 0.3, [10])
    calls = {}
    lock = threading.Lock()

    def run(req):
        with lock:
            calls[req["id"]] = calls.get(req["id"], 0) + 1
            first = calls[req["id"]] == 1
        if req["id"] == 1 and first:
            raise Transient("out of memory")
        time.sleep(req["work"])
        return dict(ok=req["id"])

    eng = serve.Engine(run, fp_of, budget_bytes=100, max_slots=3, retryable=lambda e: isinstance(e, Transient))
    recs = eng.run(reqs)
    assert [r["status"] for r in recs] == ["done"] * 3
    assert recs[1]["retries"] == 1 and calls[1] == 2
    assert recs[0]["retries"] == 0 and recs[2]["retries"] == 0


def test_retryable_failure_alone_is_a_failure():
    reqs = stream(1, 0.0, 0.0, [10])

    def run(req):
        raise Transient("out of memory")

    recs = serve.Engine(run, fp_of, budget_bytes=100, max_slots=2,
                        retryable=lambda e: isinstance(e, Transient)).run(reqs)
    assert recs[0]["status"] == "failed" and recs[0]["retries"] == 0


def test_retries_are_bounded():
    reqs = stream(2, 0.0, 0.01, [10])
    calls = {1: 0}

    def run(req):
        if req["id"] == 1:
            calls[1] += 1
            raise Transient("out of memory")
        time.sleep(0.3)
        return dict(ok=0)

    recs = serve.Engine(run, fp_of, budget_bytes=100, max_slots=2, max_retries=2,
                        retryable=lambda e: isinstance(e, Transient)).run(reqs)
    assert recs[0]["status"] == "done"
    assert recs[1]["status"] == "failed" and recs[1]["retries"] <= 2 and calls[1] == recs[1]["retries"] + 1


def test_out_of_memory_is_retryable():
    from paper_2311_17500_gb300 import _lib as L
    assert serve.device_memory_exhausted(L.StError(L.ST_ERR_OOM, "st_setup failed"))
    assert not serve.device_memory_exhausted(L.StError(L.ST_ERR_CUDA, "st_solve failed"))
    assert not serve.device_memory_exhausted(ValueError("x"))
