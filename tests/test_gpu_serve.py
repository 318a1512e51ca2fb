"""The serving loop on the GPU: requests of the seeded serving stream, shrunk
to small shapes, run concurrently (one stream and one handle per request);
every served solution must equal, bit for bit, a solve of the same request
run alone.  All reductions on the path are in a fixed order, so running
requests side by side must not change their results.
"""

import numpy as np
import pytest
import torch

import workloads as W
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def small_requests(n=5):
    reqs = W.serving_requests(n_req=n, seed=21, rate=50.0)
    rng = np.random.Generator(np.random.PCG64(21))
    for r in reqs:
        d = r["desc"]
        d["n_el"] = [int(rng.integers(6, 13)), int(rng.integers(6, 13))]
        d["n_el_t"] = int(rng.integers(8, 17))
        d["max_fp"] = 2
        d["gmres_m"] = 60
    return reqs


def test_served_solutions_equal_standalone_solves():
    torch_cuda()
    library()
    from paper_2311_17500_gb300 import serve

    reqs = small_requests()
    desc_of = lambda r: r["desc"]
    fp = serve.gpu_footprint(desc_of)
    budget = 3 * max(fp(r) for r in reqs)
    eng = serve.Engine(serve.gpu_runner(desc_of, keep_solution=True), fp, budget_bytes=budget, max_slots=3)
    recs = eng.run(reqs)
    assert [r["status"] for r in recs] == ["done"] * len(reqs), [r["error"] for r in recs]
    assert eng.peak_bytes <= budget
    alone = serve.gpu_runner(desc_of, keep_solution=True)
    for req, rec in zip(reqs, recs):
        ref = alone(req)
        got = rec["result"]
        assert got["stats"]["fp_iters"] == ref["stats"]["fp_iters"] == 2
        assert np.array_equal(got["u"], ref["u"]) and np.array_equal(got["w"], ref["w"])
        assert np.all(np.isfinite(got["u"])) and np.abs(got["u"]).max() > 0.0
    out = serve.summary(recs, n_dofs=lambda r: r["result"]["n_dof"])
    assert out["done"] == len(reqs) and out["p99_s"] >= out["p50_s"] > 0.0
    torch.cuda.synchronize()
