"""Runs st_setup and st_solve for a sequence of problem shapes in one process,
against a library linked to the launch-auditing stand-in runtime (see
fake_cudart.cpp); prints one JSON line per shape.

usage: run_shapes.py [--concurrent K] LIBRARY SHAPE...
       with SHAPE = p,n_el_x[,n_el_y[,n_el_z]],n_el_t
With --concurrent K the shapes go through the serving engine instead, with
K requests in flight on K threads, each with its own handle.  With --api every
entry point of the C ABI runs once per shape.  With --other-device D the
calling thread has device D current during st_solve (the handle was set up
on device 0).
"""

import ctypes
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_2311_17500_gb300 import _lib as L  # noqa: E402


def describe(base, shape):
    """SHAPE[:option...], options fp64 (FP64 GMRES), newton, galerkin, symmetric
    (support extension), wzero (w fixed at zero), bands / lean (operator form;
    default: the library's choice), lrreact (low-rank reaction coefficient)."""
    sizes, *opts = shape.split(":")
    v = [int(a) for a in sizes.split(",")]
    p, n_el, n_el_t = v[0], v[1:-1], v[-1]
    d = len(n_el)
    box = base["source"]["boxes"][0]
    desc = dict(base, d=d, p=p, n_el=n_el, n_el_t=n_el_t, D=[base["D"][0]] * d, max_fp=1, gmres_m=8,
                max_it=16, rtol=1e-8)
    desc["source"] = dict(base["source"], boxes=[dict(box, lo=[0.05] * d, hi=[0.15] * d)])
    for o in opts:
        if o == "fp64":
            desc["precision"] = "fp64"
        elif o == "newton":
            desc["nonlinear"] = "newton"
        elif o == "galerkin":
            desc["stabilization"] = "galerkin"
        elif o == "symmetric":
            desc["suppext"] = "symmetric"
        elif o == "wzero":
            desc["fix_w_zero"] = True
        elif o in ("bands", "lean"):
            desc["operator_form"] = o
        elif o == "lrreact":
            desc["eps_reaction"] = 1e-3
        else:
            raise ValueError("unknown option " + o)
    return desc


def solve_once(rt, desc, stream=0x1000, other_device=None):
    """st_setup + st_solve on `stream` (any non-zero value names a stream of
    its own: the stand-in runtime never dereferences it); with other_device,
    the calling thread has that device current during st_solve.  The error
    text, or None."""
    n = W.n_dofs(desc)
    try:
        s = L.Solver(desc, stream)
        u, w = rt.audit_alloc(8 * n), rt.audit_alloc(8 * n)
        ctypes.memset(u, 0, 8 * n)
        ctypes.memset(w, 0, 8 * n)
        if other_device is not None:
            rt.cudaSetDevice(other_device)
        try:
            s.solve(u, w, allow_unconverged=True)
        finally:
            s.close()
            if other_device is not None:
                cur = ctypes.c_int(-1)
                rt.cudaGetDevice(ctypes.byref(cur))
                rt.cudaSetDevice(0)
                if cur.value != other_device:
                    return "the calling thread's device was not restored"
    except Exception as e:  # values read back are not results: a NaN exit is expected
        return str(e)
    return None


def exercise_api(rt, desc, stream=0x1000, other_device=None):
    """Every entry point of the C ABI once on one handle (garbage values: only
    the launches, copies and allocations are of interest); the error texts."""
    n = W.n_dofs(desc)
    errors = []

    def call(name, fn):
        try:
            return fn()
        except Exception as e:  # values read back are not results
            errors.append(f"{name}: {e}")
            return None

    dev = {k: rt.audit_alloc(8 * n) for k in ("u", "w", "w2", "f", "x", "y", "sol")}
    for k in dev:
        ctypes.memset(dev[k], 0, 8 * n)
    s = call("setup", lambda: L.Solver(desc, stream))
    if s is None:
        return errors
    if other_device is not None:
        rt.cudaSetDevice(other_device)
    call("rhs", lambda: s.rhs(dev["f"]))
    info = call("ionic", lambda: s.ionic(dev["u"], dev["w"])) or {}
    call("linearize", lambda: s.linearize(dev["u"], dev["w"], "newton", keep_theta=True))
    for prec in (L.ST_FP64, L.ST_MIXED):
        call("apply", lambda: s.apply(dev["x"], dev["y"], prec))
        call("precond", lambda: s.precond(dev["x"], dev["y"], prec))
    call("linsolve", lambda: s.linsolve(dev["f"], dev["sol"], allow_unconverged=True))
    call("wupdate", lambda: s.wupdate(dev["u"], dev["w2"]))
    call("profile", lambda: s.profile(True))
    call("apply (profiled)", lambda: s.apply(dev["x"], dev["y"], L.ST_MIXED))
    call("profile_read", lambda: s.profile_read())
    call("profile off", lambda: s.profile(False))
    rank = int(info.get("rank", 0))
    d = s.dims
    for what, count in (("theta_hat", n), ("fd_eig", sum(d["n"][:desc["d"]])), ("lowrank_s", rank),
                        ("lowrank_u", d["N_t"] * rank), ("lowrank_v", d["N_s"] * rank),
                        ("tau_q", desc["p"] * desc["n_el_t"] * (desc["p"] + 1))):
        call("get " + what, lambda: s.get(what, count))
    call("close", s.close)
    if other_device is not None:
        cur = ctypes.c_int(-1)
        rt.cudaGetDevice(ctypes.byref(cur))
        if cur.value != other_device:
            errors.append("the calling thread's device was not restored")
        rt.cudaSetDevice(0)   # the handle-free call runs on the caller's device, where its buffers are
    a0 = rt.audit_alloc_calls()
    call("wupdate_static", lambda: L.wupdate_static(desc, dev["u"], dev["w2"], stream))
    if rt.audit_alloc_calls() != a0:
        errors.append("wupdate_static allocated or freed memory")
    return errors


def main():
    args = sys.argv[1:]
    concurrent, api, other = 0, False, None
    while args[0].startswith("--"):
        if args[0] == "--concurrent":
            concurrent, args = int(args[1]), args[2:]
        elif args[0] == "--api":
            api, args = True, args[1:]
        elif args[0] == "--other-device":
            other, args = int(args[1]), args[2:]
        else:
            raise SystemExit("unknown option " + args[0])
    L.load(args[0])
    rt = ctypes.CDLL("libcudart.so.13")
    rt.audit_alloc.restype = ctypes.c_void_p
    rt.audit_alloc.argtypes = [ctypes.c_size_t]
    rt.audit_violations.restype = ctypes.c_longlong
    rt.audit_launches.restype = ctypes.c_longlong
    rt.audit_device_bytes.restype = ctypes.c_longlong
    rt.audit_device_peak_reset.restype = ctypes.c_longlong
    rt.audit_pointer_checks.restype = ctypes.c_longlong
    rt.audit_alloc_calls.restype = ctypes.c_longlong
    base = W.serving_requests(n_req=1, seed=21)[0]["desc"]
    if concurrent:
        from paper_2311_17500_gb300 import serve
        reqs = [dict(id=i, arrival=0.0, desc=describe(base, sh)) for i, sh in enumerate(args[1:])]
        eng = serve.Engine(lambda r: solve_once(rt, r["desc"], stream=0x1000 + 16 * r["id"]), lambda r: 1,
                           budget_bytes=concurrent,
                           max_slots=concurrent)
        recs = eng.run(reqs)
        for sh, rec in zip(args[1:], recs):
            print(json.dumps(dict(shape=sh, status=rec["status"], error=rec["result"])), flush=True)
        print(json.dumps(dict(violations=rt.audit_violations(), launches=rt.audit_launches())), flush=True)
        return
    if api:
        for shape in args[1:]:
            v0, l0 = rt.audit_violations(), rt.audit_launches()
            errs = exercise_api(rt, describe(base, shape), other_device=other)
            print(json.dumps(dict(shape=shape, violations=rt.audit_violations() - v0,
                                  launches=rt.audit_launches() - l0, errors=errs)), flush=True)
        return
    for shape in args[1:]:
        v0, l0 = rt.audit_violations(), rt.audit_launches()
        desc = describe(base, shape)
        b0 = rt.audit_device_bytes()
        rt.audit_device_peak_reset()
        err = solve_once(rt, desc, other_device=other)
        # device bytes the handle held at its peak (set-up and solve; the two
        # solution vectors are allocated through the same runtime)
        peak = rt.audit_device_peak_reset() - b0
        print(json.dumps(dict(shape=shape, violations=rt.audit_violations() - v0,
                              launches=rt.audit_launches() - l0, error=err, peak_bytes=peak,
                              footprint=L.footprint(desc) + 2 * 8 * W.n_dofs(desc),
                              pointer_checks=rt.audit_pointer_checks())), flush=True)


if __name__ == "__main__":
    main()
