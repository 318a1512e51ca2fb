"""Serving loop over the C ABI: admission by device memory, one worker stream
per admitted request, arrival-to-completion latency.

Requests arrive at their `arrival` offsets (seconds from the start of the
run).  The engine admits them first come, first served: the request at the
head of the queue starts when its device footprint (st_footprint plus its
solution vectors) fits into the memory budget left by the requests in flight
and a worker slot is free.  A request that could never fit is rejected
instead of blocking the queue.  Each admitted request runs in a worker
thread on its own CUDA stream (the library's entry points release the GIL,
so the kernels of the requests in flight overlap on the device); its memory
is returned to the budget when it completes.  A request whose run raises is
recorded as failed and its memory is returned as well; one that ran out of
device memory held outside the budget may go back to the head of the queue
instead (see Engine).  A record's "error" keeps the last failure, also for a
request that completed after a retry.

The engine itself is plain Python and device-agnostic: `run_request` does the
work of one request and `footprint` sizes it.  `gpu_runner` and
`gpu_footprint` are the GB300 versions (st_setup + st_solve on a private
stream); the tests also drive the engine with host-only runners.
"""

import concurrent.futures as cf
import time

import numpy as np


class Engine:
    """First-come first-served admission under a byte budget and a slot limit.

    A request whose run raises an exception that `retryable` accepts (device
    memory exhausted by something outside the budget, for instance) goes back
    to the head of the queue, at most `max_retries` times.  It is admitted
    again only after another request has completed, and only while other
    requests are in flight; otherwise it is recorded as failed."""

    def __init__(self, run_request, footprint, budget_bytes, max_slots, clock=time.perf_counter,
                 retryable=None, max_retries=2):
        if max_slots < 1:
            raise ValueError("max_slots must be at least 1")
        self.run_request = run_request
        self.footprint = footprint
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.clock = clock
        self.retryable = retryable or (lambda exc: False)
        self.max_retries = int(max_retries)

    def run(self, requests):
        """Serve `requests` (dicts with "id", "arrival" and "desc"); returns one
        record per request, in id order."""
        pending = sorted(requests, key=lambda r: (r["arrival"], r["id"]))
        records = {}
        for r in pending:
            records[r["id"]] = dict(id=r["id"], arrival=float(r["arrival"]), footprint=int(self.footprint(r)),
                                    status="pending", admitted=None, done=None, result=None, error=None,
                                    retries=0)
        by_id = {r["id"]: r for r in pending}
        retry_after = {}      # request id -> completions count at its failure
        queue = []            # arrived, not yet admitted (FIFO)
        active = {}           # future -> request id
        used = 0
        peak = 0
        nxt = 0
        completions = 0
        t0 = self.clock()
        with cf.ThreadPoolExecutor(max_workers=self.max_slots) as pool:
            while nxt < len(pending) or queue or active:
                now = self.clock() - t0
                while nxt < len(pending) and pending[nxt]["arrival"] <= now:
                    queue.append(pending[nxt])
                    records[pending[nxt]["id"]]["status"] = "queued"
                    nxt += 1
                # admission, strictly in arrival order
                while queue and len(active) < self.max_slots:
                    head = queue[0]
                    rec = records[head["id"]]
                    if rec["footprint"] > self.budget:
                        rec["status"] = "rejected"
                        rec["error"] = "footprint %d bytes exceeds the budget of %d bytes" % (rec["footprint"],
                                                                                            self.budget)
                        rec["done"] = self.clock() - t0
                        queue.pop(0)
                        continue
                    if used + rec["footprint"] > self.budget:
                        break
                    if head["id"] in retry_after and completions <= retry_after[head["id"]]:
                        break         # a retry waits for memory to be released
                    retry_after.pop(head["id"], None)
                    queue.pop(0)
                    used += rec["footprint"]
                    peak = max(peak, used)
                    rec["status"] = "running"
                    rec["admitted"] = self.clock() - t0
                    active[pool.submit(self.run_request, head)] = head["id"]
                # wait for a completion or the next arrival
                timeout = None
                if nxt < len(pending):
                    timeout = max(0.0, pending[nxt]["arrival"] - (self.clock() - t0))
                if not active:
                    if timeout is not None and timeout > 0.0:
                        time.sleep(timeout)
                    continue
                done, _ = cf.wait(list(active), timeout=timeout, return_when=cf.FIRST_COMPLETED)
                for fut in done:
                    rid = active.pop(fut)
                    rec = records[rid]
                    used -= rec["footprint"]
                    rec["done"] = self.clock() - t0
                    exc = fut.exception()
                    if exc is None:
                        completions += 1
                        rec["status"] = "done"
                        rec["result"] = fut.result()
                    elif self.retryable(exc) and rec["retries"] < self.max_retries and active:
                        rec["retries"] += 1
                        rec["status"] = "queued"
                        rec["done"] = None
                        rec["error"] = "%s: %s" % (type(exc).__name__, exc)
                        retry_after[rid] = completions
                        queue.insert(0, by_id[rid])
                    else:
                        completions += 1
                        rec["status"] = "failed"
                        rec["error"] = "%s: %s" % (type(exc).__name__, exc)
        self.peak_bytes = peak
        return [records[k] for k in sorted(records)]


def summary(records, n_dofs=None):
    """Latency percentiles (arrival to completion), time waiting for admission
    (arrival to admission) and throughput of a run."""
    ok = [r for r in records if r["status"] == "done"]
    lat = np.array([r["done"] - r["arrival"] for r in ok], dtype=float)
    svc = np.array([r["done"] - r["admitted"] for r in ok], dtype=float)
    wait = np.array([r["admitted"] - r["arrival"] for r in ok], dtype=float)
    out = dict(requests=len(records), done=len(ok),
               failed=sum(r["status"] == "failed" for r in records),
               rejected=sum(r["status"] == "rejected" for r in records))
    if len(ok):
        makespan = max(r["done"] for r in ok) - min(r["arrival"] for r in records)
        out.update(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                   mean_s=float(lat.mean()), service_mean_s=float(svc.mean()), makespan_s=float(makespan),
                   queue_p50_s=float(np.percentile(wait, 50)), queue_p99_s=float(np.percentile(wait, 99)))
        if n_dofs is not None:
            units = sum(n_dofs(r) for r in ok)
            out["dof_per_s"] = float(units / makespan) if makespan > 0 else None
    return out


def n_unknowns(desc):
    """N_s N_t of a description: n_l = n_el + p per direction, N_t = n_el_t + p - 1."""
    n = int(desc["n_el_t"]) + int(desc["p"]) - 1
    for ne in desc["n_el"]:
        n *= int(ne) + int(desc["p"])
    return n


def gpu_footprint(desc_of):
    """Footprint of a request on the device: the library's workspaces plus the
    two FP64 solution vectors the runner allocates."""
    from . import _lib as L

    def fp(req):
        desc = desc_of(req)
        return int(L.footprint(desc)) + 2 * 8 * n_unknowns(desc)
    return fp


def device_memory_exhausted(exc):
    """True for the library's ST_ERR_OOM and for torch's out-of-memory error:
    the request can run once memory held elsewhere is released."""
    from . import _lib as L
    if isinstance(exc, L.StError):
        return exc.code == L.ST_ERR_OOM
    return type(exc).__name__ == "OutOfMemoryError"


def gpu_runner(desc_of, keep_solution=False, device=None):
    """Runs one request: st_setup and st_solve (u = w = 0 initially) on a
    private stream of `device` (default: the current device when the runner
    is made; worker threads do not inherit it); returns the solver
    statistics, the operator form set-up chose and whether the FP32
    preconditioner's transforms ran on the tensor cores (and u, w on the host
    when `keep_solution`)."""
    import torch
    from . import _lib as L
    dev = torch.cuda.current_device() if device is None else int(device)

    def run(req):
        torch.cuda.set_device(dev)
        desc = desc_of(req)
        n = n_unknowns(desc)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            u = torch.zeros(n, dtype=torch.float64, device="cuda")
            w = torch.zeros(n, dtype=torch.float64, device="cuda")
            s = L.Solver(desc, stream.cuda_stream)
            try:
                st = s.solve(u.data_ptr(), w.data_ptr(), allow_unconverged=True)
                stream.synchronize()
                form = {1: "bands", 2: "lean"}.get(s.dims["operator_form"], "?")
                tc = bool(s.dims["precond_tc"])
            finally:
                s.close()
            out = dict(stats=st, n_dof=n, operator_form=form, precond_tc=tc)
            if keep_solution:
                out["u"] = u.cpu().numpy()
                out["w"] = w.cpu().numpy()
        return out
    return run
