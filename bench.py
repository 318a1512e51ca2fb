#!/usr/bin/env python
"""Benchmark of the space-time IgA monodomain solver on GB300.

One step = one pass of the whole hot path: one fixed-point iteration of
Sec. 3.1 (ionic quadrature, Theta-hat, low rank, reaction + SU bands, the
preconditioned GMRES solve of A u = f to true relative residual 1e-8, the
w-update, relaxation and the stopping norm), starting every step from the
same saved iterate k = 2.  The default workload is the largest configuration
(3D cube, p = 3, 96^3 spatial x 192 time elements, 188,238,006 unknowns,
mixed precision, the lean operator form that fits it in one GB300);
--workload c3_cube_3d selects the 3D p = 2, 64^3 x 128 one and c2_aniso_2d
the 2D anisotropic one (p = 3, 128 x 128 x 256 elements).  The set-up (1D
data, eigendecompositions, LU factors) runs once per problem and is reported
apart.

Output: one JSON line (rank 0).  `value` is unknowns per second of the mixed
FP32/FP64 path with inputs resident on the device; `fp64` gives the FP64 path
on the same step; `e2e` measures the same step through the C ABI from pinned
host buffers, copies included; `roofline` reports the dominant kernel: in
the lean form the reaction + SU kernel, bound by FP32 arithmetic (the
reaction integrated at every space-time Gauss point), against the FP32 peak
derived from the SM count and clock; in the band form the fused band kernel
against the measured HBM bandwidth.  The whole FP32 apply against 16 bytes
per unknown (x in, y out, u^k and w^k in) is given beside it.  `linear_solve`
times one solve at the frozen linearization in both precisions;
`cpu_baseline` times the CPU oracle on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload c5_cube_3d|c3_cube_3d|c2_aniso_2d]
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c5_cube_3d"
# DRAM bytes (read + write) of the dominant kernel per unit of its work (one
# coefficient of one Gauss row at one time row) from an ncu capture of the
# same kernel on a smaller case of the same form and degree, scaled to a
# full launch by the units it processes; absent until captured, and removed
# whenever that kernel changes.
TRAFFIC_PER_UNIT = {"c5_cube_3d": 23.67}   # xlean_kernel<float,3>, 32^3 x 64 lean case: 895.8 MB / 37.85 M units
# bounded CPU samples of each workload (same physics, fewer elements): the
# cpu_baseline of our line (one step, about 10 s of oracle work) and each step
# of the reference arm (a few seconds, so that its whole run stays short)
CPU_SAMPLES = {"c5_cube_3d": dict(n_el=[4, 4, 4], n_el_t=6),
               "c3_cube_3d": dict(n_el=[6, 6, 6], n_el_t=12),
               "c2_aniso_2d": dict(n_el=[12, 12], n_el_t=24)}
REF_SAMPLES = {"c5_cube_3d": dict(n_el=[3, 3, 3], n_el_t=6),
               "c3_cube_3d": dict(n_el=[5, 5, 5], n_el_t=10),
               "c2_aniso_2d": dict(n_el=[12, 12], n_el_t=24)}
# algorithmic bytes of one FP32 operator apply per unknown (the method's
# compulsory traffic): x read and y written, u^k and w^k read for the exact
# reaction coefficient at the Gauss points, 4 bytes each
APPLY_BYTES_PER_DOF = 16.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(CPU_SAMPLES))
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64 comparison (it is skipped by default under torchrun with more than one "
                         "rank on the 96^3 x 192 workload, where it holds every GPU for minutes; --fp64 forces it)")
    ap.add_argument("--fp64", action="store_true", help="run the FP64 comparison whatever the rank count")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="FP64 fixed-point steps beside the mixed ones (default 1; 0 on the 96^3 x 192 workload, "
                         "whose FP64 linear solve alone takes minutes)")
    ap.add_argument("--profiled-steps", type=int, default=1, help="steps repeated with per-stage events")
    ap.add_argument("--scale", default=None,
                    help="element counts n_el..., n_el_t (a smaller case of the same physics, e.g. for profiling)")
    ap.add_argument("--form", default=None, choices=["auto", "bands", "lean"],
                    help="operator form (default: the workload's, auto)")
    ap.add_argument("--serve", action="store_true",
                    help="the serving stream instead of the single workload (latency p50/p99, DoF/s)")
    ap.add_argument("--requests", type=int, default=256, help="--serve: requests in the stream")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="--serve: Poisson arrival rate (requests/s); 0 = 0.8 x the measured saturated rate")
    ap.add_argument("--slots", type=int, default=8, help="--serve: requests in flight at most")
    ap.add_argument("--serve-log", default=None, help="--serve: write one JSON line per request to this file")
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="requests of the short serving pass in the default run (0: none; default 64, "
                         "0 on the 96^3 x 192 workload)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, 1900.0, "fallback", 2070.0


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.path is None or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_step(desc_sample):
    """One fixed-point step of the oracle from u = w = 0 (runs in a child process
    pinned to one thread so that `cores` is exact)."""
    code = (
        "import json, sys, time; sys.path.insert(0, %r)\n"
        "import workloads as W\n"
        "from oracle import Oracle\n"
        "desc = json.loads(%r)\n"
        "t = time.perf_counter(); o = Oracle(desc); u, w, h = o.solve(max_fp=1); dt = time.perf_counter() - t\n"
        "print(json.dumps(dict(seconds=dt, n_dof=o.st.N_dof)))\n" % (ROOT, json.dumps(desc_sample)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def cpu_sample_desc(samples=None):
    import workloads as W
    d = W.config(WORKLOAD, scale=(samples or CPU_SAMPLES)[WORKLOAD])
    d["max_fp"] = 1
    return d


def sample_shape(samples=None):
    c = (samples or CPU_SAMPLES)[WORKLOAD]
    return "x".join(str(v) for v in c["n_el"]) + f"x{c['n_el_t']}"


def cpu_baseline():
    out = cpu_oracle_step(cpu_sample_desc())
    return {"value": out["n_dof"] / out["seconds"], "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"one fixed-point step from u=w=0 of the same physics on {sample_shape()} "
                      f"elements ({out['n_dof']} DoF): "
                      f"sparse space-time assembly + SuperLU direct solve, {out['seconds']:.1f} s"}


def whole_job(ms_local, units_local, dist, device):
    """Whole-job step time and rate over the ranks: every rank solves its own
    replica of the workload (the problems are independent, so no data moves
    between ranks); the step time is the maximum over ranks and the rate is
    the units of all ranks over that time.  Returns (ms, units per second)."""
    import torch
    t = torch.tensor([ms_local, float(units_local)], dtype=torch.float64, device=device)
    if dist is not None:
        mx = t[:1].clone()
        tot = t[1:].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        t = torch.cat([mx, tot])
    ms, units = float(t[0].item()), float(t[1].item())
    return ms, units / (ms / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_name(desc):
    d = desc["d"]
    dom = "unit square" if d == 2 else "unit cube" if d == 3 else "unit interval"
    D = desc["D"]
    dstr = f"D={D[0]:g} I" if len(set(D)) == 1 else "D=diag(" + ",".join(f"{v:g}" for v in D) + ")"
    stim = {"c2_aniso_2d": "seeded corner stimulus", "c3_cube_3d": "planar stimulus x<0.05",
            "c5_cube_3d": "two staggered corner stimuli"}.get(WORKLOAD, "stimulus")
    return (f"{WORKLOAD}: {d}D {dom}, p={desc['p']}, " + "x".join(str(v) for v in desc["n_el"]) +
            f" x {desc['n_el_t']} elements, {dstr}, {stim}, "
            f"{desc['stabilization'].upper() if desc['stabilization'] == 'su' else 'Galerkin'}, "
            f"Picard step from saved iterate k=2")


# the metric of both arms (ours and the reference arm's oracle)
METRIC = "space-time solve throughput (one fixed-point step incl. linear solve at rel.res 1e-8), mixed vs FP64"


def run_reference(args):
    import workloads as W
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    desc = cpu_sample_desc(REF_SAMPLES)
    times = []
    n_dof = None
    for k in range(args.warmup + args.steps):
        out = cpu_oracle_step(desc)
        n_dof = out["n_dof"]
        if k >= args.warmup:
            times.append(out["seconds"])
    ms = 1000.0 * sum(times) / len(times)
    value = n_dof / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "DoF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(W.config(WORKLOAD)),
                       "sample": f"each step: the same physics on {sample_shape(REF_SAMPLES)} "
                                 f"elements ({n_dof} DoF), one fixed-point step from u = w = 0"},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                             "sample": "CPU FP64 oracle: sparse assembly + SuperLU, one fixed-point step"},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_linear_solve(solver, u2, w2, stream, reps, warm=1):
    """Time of one linear solve to relative residual 1e-8 (st_linsolve) with
    the linearization frozen at the saved iterate (u2, w2) and x0 = u2; the
    right-hand side is f.  Mean of `reps` solves after `warm` untimed ones."""
    import torch
    n = u2.numel()
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.empty_like(f)
    solver.rhs(f.data_ptr())
    solver.linearize(u2.data_ptr(), w2.data_ptr(), "picard")
    out = None
    times = []
    for k in range(reps + warm):
        x.copy_(u2)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        out = solver.linsolve(f.data_ptr(), x.data_ptr(), allow_unconverged=True)
        ev1.record(stream)
        ev1.synchronize()
        if k >= warm:
            times.append(ev0.elapsed_time(ev1))
    ms = sum(times) / len(times)
    return {"ms": ms, "dof_per_s": n / (ms / 1000.0), "gmres_iters": out["gmres_iters"],
            "outer_iters": out["outer_iters"], "rel_res": out["rel_res"]}


def run_ours(args):
    import torch
    import workloads as W
    from paper_2311_17500_gb300 import build as B
    B.build()
    import paper_2311_17500_gb300 as P
    P.load()

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    desc = W.config(WORKLOAD)
    if args.scale:
        vals = [int(v) for v in args.scale.split(",")]
        desc["n_el"] = vals[:-1]
        desc["n_el_t"] = vals[-1]
    if args.form:
        desc["operator_form"] = args.form
    desc["max_fp"] = 1
    desc["rtol"] = 1e-8
    desc["gmres_m"] = 150
    desc["max_it"] = 3000

    def fit_m(d):
        """Largest Krylov size <= 150 whose handle fits in 90 % of the free
        device memory, with room for the bench's own vectors."""
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        room = 0.9 * free - 10 * 8 * W.n_dofs(d)
        m = 150
        while m > 10 and P.footprint(dict(d, gmres_m=m)) > room:
            m -= 10
        return m

    def make(precision):
        d = dict(desc, precision=precision)
        d["gmres_m"] = fit_m(d)
        t0 = time.perf_counter()
        s = P.Solver(d, sptr)
        torch.cuda.synchronize()
        s.desc_m = d["gmres_m"]
        return s, time.perf_counter() - t0

    big = WORKLOAD == "c5_cube_3d"
    fp64_steps = args.fp64_steps if args.fp64_steps is not None else (0 if big else 1)
    serve_requests = args.serve_requests if args.serve_requests is not None else (0 if big else 64)
    s, setup_s = make("mixed")
    s_m = s.desc_m
    s_form = {1: "bands", 2: "lean"}.get(s.dims["operator_form"], "?")
    s_tc = bool(s.dims["precond_tc"])
    N = s.dims["N_dof"]
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(u)
    for _ in range(2):                       # iterate k = 2 of the nonlinear loop
        s.solve(u.data_ptr(), w.data_ptr(), allow_unconverged=True)
    u2, w2 = u.clone(), w.clone()

    def step(solver):
        u.copy_(u2)
        w.copy_(w2)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = solver.solve(u.data_ptr(), w.data_ptr(), allow_unconverged=True)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1), st

    for _ in range(args.warmup):
        step(s)
    lib = P.load()
    peaks = measured_peaks()
    # the timed steps
    n0 = lib.st_launch_count()
    barrier()
    times, stats = [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            ms, st = step(s)
            times.append(ms)
            stats.append(st)
    barrier()
    launches = lib.st_launch_count() - n0
    clocks = clk.summary()
    # the same steps again with per-stage CUDA events on the solver's stream
    # (their recording costs a few percent, so they stay out of the headline)
    s.profile(True)
    ptimes = []
    for _ in range(max(1, args.profiled_steps)):
        ms, _ = step(s)
        ptimes.append(ms)
    barrier()
    prof = s.profile_read()
    s.profile(False)
    ms_local = sum(times) / len(times)
    ms_step, value = whole_job(ms_local, N, dist, "cuda")
    st_last = stats[-1]

    # roofline of the dominant kernel (stage qband: one launch per FP32
    # apply), from the profiled steps' per-stage CUDA events on the solver's
    # stream.  Lean form: the reaction at every space-time Gauss point and the
    # SU rank terms, counted as the flops of its sum-factorized quadrature,
    # against the FP32 peak (SMs x 128 lanes x 2 flop per FMA x the maximum SM
    # clock).  Band form: the fused band kernel against the measured HBM
    # bandwidth, its bytes being the stored time bands and the x rows.
    hbm, bf16, src, sm_max = peaks
    q = prof["qband"]
    nl = max(q["launches"], 1)
    t_launch = q["ms"] / nl
    units = q["bytes"] / nl / 24.0   # lean: x, y FP32 and u^k, w^k pairs per unit
    tpu = TRAFFIC_PER_UNIT.get(WORKLOAD) if args.scale is None else None
    if s_form == "lean":
        flops = q["flops"] / nl
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        achieved = flops / (t_launch / 1000.0) / 1e12 if t_launch > 0 else 0.0
        roof = {"bound": "alu", "kernel": "xlean_kernel<float,%d> (stage qband)" % desc["p"],
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tpu * units if tpu else None,
                "algorithmic_flops_per_launch": flops,
                "flops_rule": "per (Gauss row, x element, time row): x, u^k, w^k at the p+1 x Gauss points; "
                              "at the (p+1)^2 space-time points of the next time element C(u,w) x and its test "
                              "against p+1 time functions; the R rank bands; the x projection",
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop per FMA x {sm_max:g} MHz",
                "algorithmic_bytes_per_launch": q["bytes"] / nl,
                "hbm_gbs": q["bytes"] / nl / (t_launch / 1000.0) / 1e9 if t_launch > 0 else None}
    else:
        achieved = q["bytes"] / nl / (t_launch / 1000.0) / 1e9 if t_launch > 0 else 0.0
        roof = {"bound": "hbm", "kernel": "xband_fused_kernel<float,%d> (stage qband)" % desc["p"],
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "algorithmic_bytes_per_launch": q["bytes"] / nl,
                "bytes_rule": "stored time bands (p+1 per spatial Gauss point and time row) + x rows in and out",
                "peak_source": src}
    t_apply = sum(prof[k]["ms"] for k in ("kron", "interp", "qband")) / nl
    alg = APPLY_BYTES_PER_DOF * N
    roof.update({"launch_ms": t_launch, "launches": nl, "share_of_step": q["ms"] / sum(ptimes),
                 "apply_hbm_view": {"ms": t_apply, "algorithmic_bytes": alg,
                                    "gbs": alg / (t_apply / 1000.0) / 1e9 if t_apply > 0 else None,
                                    "frac_of_hbm": alg / (t_apply / 1000.0) / 1e9 / hbm if t_apply > 0 else None,
                                    "rule": f"whole FP32 apply, {APPLY_BYTES_PER_DOF:g} B per unknown: x in, "
                                            "y out, u^k and w^k in"},
                 "profiled_ms_per_step": sum(ptimes) / len(ptimes),
                 "stages_ms_per_step": {k: v["ms"] / len(ptimes) for k, v in prof.items()},
                 "stages_gbs": {k: (v["bytes"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] > 0 and v["bytes"] > 0 else None)
                                for k, v in prof.items()}})

    # e2e: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hu = u2.cpu().pin_memory()
        hw = w2.cpu().pin_memory()
        ou = torch.empty_like(hu).pin_memory()
        ow = torch.empty_like(hw).pin_memory()
        e_ms = []
        for k in range(1 if big else 2):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            u.copy_(hu, non_blocking=True)
            w.copy_(hw, non_blocking=True)
            s.solve(u.data_ptr(), w.data_ptr(), allow_unconverged=True)
            ou.copy_(u, non_blocking=True)
            ow.copy_(w, non_blocking=True)
            ev1.record(stream)
            ev1.synchronize()
            e_ms.append(ev0.elapsed_time(ev1))
        em = sum(e_ms) / len(e_ms)
        e2e = {"value": ws * N / (em / 1000.0), "unit": "DoF/s", "h2d_bytes_per_step": 2 * 8 * N,
               "d2h_bytes_per_step": 2 * 8 * N}
    # the linear solve alone, mixed and FP64, at the same frozen linearization
    linear = {}
    try:
        linear["mixed"] = time_linear_solve(s, u2, w2, stream, 1 if big else 2, warm=0 if big else 1)
    except Exception as e:  # noqa: BLE001 (reported in the line, never fatal)
        linear["mixed"] = {"error": f"{type(e).__name__}: {e}"}
    s.close()

    fp64 = None
    # replicas repeat the same FP64 solve; on the largest workload it takes
    # minutes, so a multi-rank run leaves it out unless asked for
    if not args.no_fp64 and (args.fp64 or ws == 1 or not big):
        s64, setup64 = make("fp64")
        fp64 = {"setup_s": setup64, "gmres_m": s64.desc_m}
        if fp64_steps > 0:
            u.copy_(u2); w.copy_(w2)
            step(s64)                                   # warm-up
            f_ms = []
            f_st = None
            for _ in range(fp64_steps):
                ms, f_st = step(s64)
                f_ms.append(ms)
            fm = sum(f_ms) / len(f_ms)
            fp64.update({"value": N / (fm / 1000.0), "ms_per_step": fm, "gmres_iters": f_st["gmres_iters"],
                         "rel_res": f_st["rel_res"], "speedup_mixed_vs_fp64": fm / ms_step})
        try:
            # with no FP64 step before it the solve is timed cold: its own first
            # FP64 residual is the warm-up of the FP64 kernels
            linear["fp64"] = time_linear_solve(s64, u2, w2, stream, 1, warm=0 if fp64_steps == 0 else 1)
            if "ms" in linear.get("mixed", {}):
                linear["speedup_mixed_vs_fp64"] = linear["fp64"]["ms"] / linear["mixed"]["ms"]
        except Exception as e:  # noqa: BLE001
            linear["fp64"] = {"error": f"{type(e).__name__}: {e}"}
        s64.close()

    serving = None
    if ws == 1 and serve_requests > 0:
        # the serving stream, shortened: latency percentiles beside the step
        # throughput; a failure here is reported in the line, never fatal
        try:
            f = serving_pass(serve_requests, 0.0, args.slots, local, clocks=False)
            serving = {k: f[k] for k in ("value", "unit", "latency_ms", "queue_ms", "service_ms_mean", "requests",
                                         "done", "failed", "rejected", "errors", "config")}
        except Exception as e:  # noqa: BLE001
            serving = {"error": f"{type(e).__name__}: {e}"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline()

    srt = sorted(times)
    line = {
        "metric": METRIC,
        "value": value, "unit": "DoF/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+df64+f64", "data": "synthetic",
        "config": {"workload": workload_name(desc),
                   "N_dof": N, "precision": f"mixed: FP32 inner GMRES({s_m}) + FP64 refinement",
                   "operator_form": s_form, "gmres_m": s_m,
                   "preconditioner": ("TF32 tensor-core (tcgen05) FD transforms" if s_tc
                                      else "FP32 CUDA-core FD transforms"),
                   "l2": "inputs larger than L2 (vectors of %.0f MB FP32; %s)" % (
                       4 * N / 1e6, "the Gauss-row arrays of x, u^k, w^k" if s_form == "lean" else "the stored time bands"),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "setup_s": setup_s},
        "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
        "solve": {"gmres_iters": st_last["gmres_iters"], "outer_iters": st_last["outer_iters"],
                  "rel_res": st_last["rel_res"], "rank": st_last["rank"]},
        "gpu_launches": launches,
        "roofline": roof,
        "fp64": fp64,
        "linear_solve": linear,
        "e2e": e2e,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "serving": serving,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def serving_pass(n_requests, rate, slots, local, clocks=True, log_path=None):
    """The serving stream: seeded 2D requests (p in {2,3}, 32..256 elements per
    direction, 64..512 time elements, D log-uniform, a stimulus at a uniform
    position) arriving as a Poisson stream.  A request is st_setup and one
    fixed-point step (GMRES-IR to relative residual 1e-8) from u = w = 0, on its
    own stream; admission is first come, first served under 85 % of the free
    device memory and a slot limit.  Returns the fields of the JSON line:
    unknowns per second over the makespan, arrival-to-completion latency
    percentiles, admission waits and the workload.

    With rate 0 the arrival rate is set from the stream itself: a first pass
    serves every request at once (all arrive at t = 0), which gives the
    saturated throughput in requests/s; the timed pass then runs the same
    requests as a Poisson stream at 0.8 of that rate."""
    import torch
    import workloads as W
    from paper_2311_17500_gb300 import serve
    # arrivals drawn at rate 1 and scaled: every rate gives the same requests
    unit = W.serving_requests(n_req=n_requests, seed=4, rate=1.0)

    def at_rate(r):
        return [dict(q, arrival=(q["arrival"] / r if r else 0.0)) for q in unit]

    def desc_of(r):
        d = dict(r["desc"])
        d.update(max_fp=1, rtol=1e-8, gmres_m=150, max_it=3000)
        return d

    runner, footprint = serve.gpu_runner(desc_of), serve.gpu_footprint(desc_of)
    # library, tensor-core self-test and caches warmed outside the timed stream
    runner(dict(unit[0], desc=dict(unit[0]["desc"], n_el=[16, 16], n_el_t=16)))
    torch.cuda.synchronize()
    free, _total = torch.cuda.mem_get_info()
    budget = int(0.85 * free)
    saturated = None
    given = rate > 0
    if not given:
        recs0 = serve.Engine(runner, footprint, budget, slots,
                             retryable=serve.device_memory_exhausted).run(at_rate(0.0))
        torch.cuda.synchronize()
        out0 = serve.summary(recs0, n_dofs=lambda r: r["result"]["n_dof"])
        if not out0["done"]:
            raise RuntimeError("no request of the saturated pass completed: %s" % recs0[0]["error"])
        rate = 0.8 * out0["done"] / out0["makespan_s"]
        saturated = {"requests_per_s": out0["done"] / out0["makespan_s"], "dof_per_s": out0.get("dof_per_s"),
                     "makespan_s": out0["makespan_s"], "done": out0["done"], "failed": out0["failed"],
                     "rejected": out0["rejected"]}
    reqs = at_rate(rate)
    eng = serve.Engine(runner, footprint, budget, slots, retryable=serve.device_memory_exhausted)
    if clocks:
        with Clocks(local) as ck:
            recs = eng.run(reqs)
    else:
        ck = None
        recs = eng.run(reqs)
    torch.cuda.synchronize()
    out = serve.summary(recs, n_dofs=lambda r: r["result"]["n_dof"])
    n_dof = [W.n_dofs(desc_of(r)) for r in reqs]
    errors = {}
    for r in recs:
        if r["status"] in ("failed", "rejected"):
            errors[r["error"]] = errors.get(r["error"], 0) + 1
            if len(errors) == 1 and errors[r["error"]] == 1:
                d = desc_of(reqs[r["id"]])
                print(f"request {r['id']} ({d['p']}, {d['n_el']}, {d['n_el_t']}): {r['error']}", file=sys.stderr)
    iters = [r["result"]["stats"]["total_gmres"] for r in recs if r["status"] == "done"]
    # requests whose FP32 preconditioner ran on CUDA cores (an axis wider than
    # the tensor-core transform takes, n_l > 256)
    no_tc = sum(1 for r in recs if r["status"] == "done" and r["result"].get("precond_tc") is False)
    if log_path:
        # one JSON line per request: its shape, its times and how it ended
        with open(log_path, "w") as f:
            for r in recs:
                d = desc_of(reqs[r["id"]])
                f.write(json.dumps({"id": r["id"], "p": d["p"], "n_el": d["n_el"], "n_el_t": d["n_el_t"],
                                    "n_dof": W.n_dofs(d), "arrival_s": r["arrival"], "admitted_s": r["admitted"],
                                    "done_s": r["done"], "status": r["status"], "retries": r["retries"],
                                    "gmres": (r["result"] or {}).get("stats", {}).get("total_gmres"),
                                    "operator_form": (r["result"] or {}).get("operator_form"),
                                    "precond_tc": (r["result"] or {}).get("precond_tc"),
                                    "error": r["error"]}) + "\n")
    fields = {
        "value": out.get("dof_per_s"), "unit": "DoF/s",
        "latency_ms": {"p50": 1e3 * out["p50_s"], "p99": 1e3 * out["p99_s"], "mean": 1e3 * out["mean_s"]}
        if out["done"] else None,
        "service_ms_mean": 1e3 * out["service_mean_s"] if out["done"] else None,
        "queue_ms": {"p50": 1e3 * out["queue_p50_s"], "p99": 1e3 * out["queue_p99_s"]} if out["done"] else None,
        "makespan_s": out.get("makespan_s"),
        "requests": out["requests"], "done": out["done"], "failed": out["failed"], "rejected": out["rejected"],
        "retries": sum(r["retries"] for r in recs),
        "cuda_core_preconditioner": no_tc,
        "errors": dict(sorted(errors.items(), key=lambda kv: -kv[1])[:5]),
        "failed_shapes": [[desc_of(reqs[r["id"]])["p"]] + desc_of(reqs[r["id"]])["n_el"] +
                          [desc_of(reqs[r["id"]])["n_el_t"]] for r in recs if r["status"] == "failed"][:12],
        "config": {"workload": f"serving stream: {n_requests} seeded 2D requests, p in {{2,3}}, 32..256 "
                               f"elements per direction, 64..512 time elements, D log-uniform in [2e-4,2e-3], "
                               f"Poisson arrivals at {rate:.3g}/s; a request = set-up + one fixed-point step "
                               f"to rel.res 1e-8 from u = w = 0",
                   "unknowns_per_request": {"min": min(n_dof), "median": int(sorted(n_dof)[len(n_dof) // 2]),
                                            "max": max(n_dof)},
                   "arrival_rate_per_s": rate,
                   "rate_rule": "given" if given else "0.8 x saturated throughput of the same requests",
                   "saturated": saturated,
                   "slots": slots, "budget_gb": budget / 1e9, "peak_admitted_gb": eng.peak_bytes / 1e9,
                   "gmres_iters_mean": (sum(iters) / len(iters)) if iters else None},
    }
    if ck is not None:
        fields["clocks"] = ck.summary()
    return fields


def run_serve(args):
    """The serving stream alone (see serving_pass): one JSON line."""
    import torch
    from paper_2311_17500_gb300 import build as B
    B.build()
    import paper_2311_17500_gb300 as P
    P.load()
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    fields = serving_pass(args.requests, args.rate, args.slots, local, log_path=args.serve_log)
    line = {"metric": "serving stream: unknowns/s over the makespan and arrival-to-completion latency p50/p99",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32+df64+f64", "data": "synthetic", **fields}
    if rank == 0:
        print(json.dumps(line))


def main():
    global WORKLOAD
    args = parse()
    WORKLOAD = args.workload
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
