"""Host-side launch logic of the library, audited on the CPU.

The library's objects are linked against a stand-in CUDA runtime that runs no
kernel (tests/launch_audit/fake_cudart.cpp).  st_setup and st_solve are then
driven over a sequence of problem shapes in one process, and every kernel
launch is checked against GB300 limits: block and grid extents, dynamic
shared memory against the kernel's own limit (48 KB unless it opted in),
shared memory per block, registers per block (from the ptxas report of the
build), cluster size.  Every copy and memset is checked against its
allocation, and every tensor map against the encoder's rules.  Each handle
gets a stream of its own, so no launch or asynchronous copy may use the legacy
stream, and the stream-ordered allocations are checked against the streams of
their copies, memsets and frees.

One process runs every shape because shared-memory opt-ins are per process:
the sequence starts with p = 3 and then moves to p = 2 wide-x shapes. That
order once left p = 2 instances of the fused x pass without their opt-in.
"""

import json
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
AUDIT = os.path.join(ROOT, "tests", "launch_audit")

# p, n_el per spatial direction, n_el_t: p = 1..4, d = 1..3, tiny and ragged
# meshes, x axes wide enough for every fused-pass width, long time axes, and
# the serving order of the shapes (p = 3 first, then p = 2 wide x); then FP64 GMRES, Newton,
# Galerkin, the symmetric support extension and w fixed at zero
SHAPES = ["3,16,16,16", "3,120,33,64", "2,194,33,64", "2,216,33,64", "2,150,33,64", "3,254,40,16",
          "2,255,32,16", "1,300,20,16", "4,200,20,16", "2,5,4,6", "3,4,5,5", "1,6,5,7", "4,6,5,7", "2,1,2,3",
          "2,8,8,512", "2,7,9", "3,40,20", "2,3,4,3,4", "3,8,8,8,16", "4,10,10,10,8", "1,20,20,20,8",
          "2,200,8,8,8", "3,16,16,16:fp64", "2,194,33,64:fp64:newton", "3,120,33,64:newton",
          "2,8,8,8,16:fp64", "2,9,7,12:galerkin", "3,9,7,12:symmetric:wzero", "1,40,12:fp64",
          # the band form where the lean one is the default, and the lean form at its widest x
          "3,16,16,16:bands", "3,120,33,64:bands", "2,200,8,8,8:bands:fp64", "3,8,8,8,16:bands:newton",
          "1,255,8,16:lean", "4,252,6,8:lean:fp64", "2,20,6,5,8:lean:newton",
          # the low-rank reaction coefficient in both forms
          "2,9,7,12:lrreact", "3,8,8,8,16:bands:lrreact", "2,20,6,5,8:lean:lrreact:newton", "1,40,12:lrreact"]


def _have_tools():
    nvcc = shutil.which("nvcc") or (os.path.exists("/usr/local/cuda/bin/nvcc") and "/usr/local/cuda/bin/nvcc")
    return bool(nvcc) and shutil.which("g++") is not None and os.path.exists("/usr/local/cuda/include/cuda.h")


@pytest.fixture(scope="module")
def audit_env():
    if not _have_tools():
        pytest.skip("nvcc, g++ or the CUDA headers are missing")
    from paper_2311_17500_gb300 import build as B
    B.build()
    cu = [s for s in B.SOURCES if s.endswith(".cu")]
    if not all(os.path.exists(B.resources_path(s)) for s in cu):
        B.build(force=True)
    out = os.path.join(B.OBJDIR, "audit")
    os.makedirs(out, exist_ok=True)
    lib = os.path.join(out, "libst_audit.so")
    subprocess.run([B.nvcc(), *B.ARCH, "-shared", "-o", lib, *B.objects(), "-cudart", "shared"], check=True,
                   capture_output=True)
    rt = os.path.join(out, "libcudart.so.13")
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I/usr/local/cuda/include",
                    "-Wl,-soname,libcudart.so.13", "-Wl,--version-script=" + os.path.join(AUDIT, "cudart.map"),
                    os.path.join(AUDIT, "fake_cudart.cpp"), "-o", rt], check=True, capture_output=True)
    table = os.path.join(out, "resources.txt")
    with open(table, "w") as f:
        for s in cu:
            kernel = None
            for line in open(B.resources_path(s)):
                m = re.search(r"Compiling entry function '(\S+)'", line)
                if m:
                    kernel = m.group(1)
                    continue
                m = re.search(r"Used (\d+) registers", line)
                if m and kernel:
                    sm = re.search(r"(\d+) bytes smem", line)
                    f.write(f"{kernel} {m.group(1)} {sm.group(1) if sm else 0}\n")
                    kernel = None
    sigs = os.path.join(out, "signatures.txt")
    write_signatures(table, sigs)
    return dict(lib=lib, dir=out, table=table, sigs=sigs)


def parameter_kinds(demangled):
    """'P' (pointer) or 'S' (anything else) per parameter of a demangled
    function signature such as 'void f<float, 2>(float*, float const*, int)'."""
    if not demangled.endswith(")"):
        return None
    depth, start = 0, None
    for i in range(len(demangled) - 1, -1, -1):
        c = demangled[i]
        if c == ")":
            depth += 1
        elif c == "(":
            depth -= 1
            if depth == 0:
                start = i
                break
    if start is None:
        return None
    params, depth, cur = [], 0, ""
    for c in demangled[start + 1:-1]:
        if c in "<(":
            depth += 1
        elif c in ">)":
            depth -= 1
        if c == "," and depth == 0:
            params.append(cur.strip())
            cur = ""
        else:
            cur += c
    if cur.strip():
        params.append(cur.strip())
    return "".join("P" if p.endswith("*") else "S" for p in params)


def write_signatures(table, path):
    """Pointer parameters of every kernel, from its demangled name (c++filt)."""
    names = [line.split()[0] for line in open(table) if line.strip()]
    res = subprocess.run(["c++filt"], input="\n".join(names), capture_output=True, text=True, check=True)
    with open(path, "w") as f:
        for name, dem in zip(names, res.stdout.splitlines()):
            kinds = parameter_kinds(dem.strip())
            if kinds:
                f.write(f"{name} {kinds}\n")


def run(audit_env, shapes, **extra):
    env = dict(os.environ, LD_LIBRARY_PATH=audit_env["dir"], AUDIT_RESOURCES=audit_env["table"],
               AUDIT_SIGNATURES=audit_env["sigs"],
               AUDIT_LOG=os.path.join(audit_env["dir"], "launches.log"), **extra)
    res = subprocess.run([sys.executable, os.path.join(AUDIT, "run_shapes.py"), audit_env["lib"], *shapes],
                         env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    rows = [json.loads(line) for line in res.stdout.splitlines() if line.startswith("{")]
    assert [r["shape"] for r in rows] == list(shapes)
    log = open(env["AUDIT_LOG"]).read()
    return rows, log


def test_every_launch_within_limits(audit_env):
    # every handle gets a stream of its own: nothing may run on the legacy stream
    rows, log = run(audit_env, SHAPES, AUDIT_FORBID_NULL_STREAM="1")
    bad = [line for line in log.splitlines() if line.startswith("VIOLATION")]
    assert not bad, "\n".join(bad[:10])
    for r in rows:
        assert r["violations"] == 0, r
        # set-up, linearization, both operators, the preconditioner and Arnoldi ran
        assert r["launches"] >= 60, r
        assert r["error"] is None or "CUDA error" not in r["error"], r
    # the tensor-core transforms and their tensor maps were audited too, and the
    # pointer arguments of the launches
    assert "tc_xform" in log and "tensor map" in log
    assert rows[-1]["pointer_checks"] >= sum(r["launches"] for r in rows) > 0   # every kernel takes a pointer


def test_footprint_bounds_what_a_handle_allocates(audit_env):
    """The serving loop admits a request by st_footprint (plus its two
    solution vectors): that figure must not be below what set-up and solve
    allocate on the device, or admission over-commits device memory.  A
    first small problem takes the once-per-process tensor-core self-test, whose
    buffers belong to no handle."""
    rows, _ = run(audit_env, ["2,2,2,3"] + SHAPES + ["1,1,1,1", "4,1,1,1", "1,1,1,1,1", "4,1,1,1,1"])
    for r in rows[1:]:
        assert r["peak_bytes"] > 0, r
        assert r["peak_bytes"] <= r["footprint"], r
        # and not so far above it that admission turns requests away for nothing
        assert r["footprint"] <= 1.25 * r["peak_bytes"] + (1 << 20), r


def test_audit_sees_a_missing_opt_in(audit_env):
    """With opt-ins ignored, the kernels that need more than 48 KB of dynamic
    shared memory are refused: the audit can see the failure it guards against."""
    rows, log = run(audit_env, ["3,120,33,64:bands", "2,194,33,64:bands"], AUDIT_IGNORE_OPTIN="1")
    assert sum(r["violations"] for r in rows) > 0
    assert "no opt-in" in log
    assert any(r["error"] and "pending since the launch at" in r["error"] for r in rows)


def test_requests_in_flight_together(audit_env):
    """The serving engine with four requests in flight on four threads, each
    with its own handle (shared state of the library: the tensor-core
    self-test, the opt-in masks, the per-thread error detail)."""
    shapes = ["3,16,16,16", "2,194,33,64", "3,120,33,64", "2,216,33,64", "2,5,4,6", "3,4,5,5,5", "1,30,30,16",
              "4,20,20,8"]
    env = dict(os.environ, LD_LIBRARY_PATH=audit_env["dir"], AUDIT_RESOURCES=audit_env["table"],
               AUDIT_SIGNATURES=audit_env["sigs"],
               AUDIT_LOG=os.path.join(audit_env["dir"], "launches_concurrent.log"), AUDIT_FORBID_NULL_STREAM="1")
    res = subprocess.run([sys.executable, os.path.join(AUDIT, "run_shapes.py"), "--concurrent", "4",
                          audit_env["lib"], *shapes], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    rows = [json.loads(line) for line in res.stdout.splitlines() if line.startswith("{")]
    per_request, total = rows[:-1], rows[-1]
    assert [r["shape"] for r in per_request] == shapes
    for r in per_request:
        assert r["status"] == "done", r
        assert r["error"] is None or "CUDA error" not in r["error"], r
    assert total["violations"] == 0
    assert total["launches"] >= 60 * len(shapes)


STREAM_PROBE = r'''
import ctypes, sys
rt = ctypes.CDLL(sys.argv[1])
rt.audit_violations.restype = ctypes.c_longlong
rt.cudaMallocAsync.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_void_p]
rt.cudaMemsetAsync.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]
rt.cudaFreeAsync.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
p = ctypes.c_void_p()
assert rt.cudaMallocAsync(ctypes.byref(p), 4096, ctypes.c_void_p(0x1000)) == 0
v0 = rt.audit_violations()
rt.cudaMemsetAsync(p, 0, 4096, ctypes.c_void_p(0x1000))
v1 = rt.audit_violations()
rt.cudaMemsetAsync(p, 0, 4096, ctypes.c_void_p(0x2000))
print(v1 - v0, rt.audit_violations() - v1)
rt.cudaFreeAsync(p, ctypes.c_void_p(0x1000))
'''


def test_audit_sees_a_stream_ordered_allocation_used_elsewhere(audit_env, tmp_path):
    """The stand-in runtime flags a memset of stream-ordered memory on another
    stream than the one it was allocated on.  (A process of its own: one that
    has loaded the real runtime would resolve the same library name to it.)"""
    script = tmp_path / "stream_probe.py"
    script.write_text(STREAM_PROBE)
    env = dict(os.environ, AUDIT_LOG=str(tmp_path / "log.txt"))
    res = subprocess.run([sys.executable, str(script), os.path.join(audit_env["dir"], "libcudart.so.13")],
                         env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    assert res.stdout.split() == ["0", "1"]


CHECKER = r'''
import ctypes, sys
rt = ctypes.CDLL(sys.argv[1])
rt.audit_violations.restype = ctypes.c_longlong
class Dim3(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint), ("y", ctypes.c_uint), ("z", ctypes.c_uint)]
class Config(ctypes.Structure):
    _fields_ = [("grid", Dim3), ("block", Dim3), ("smem", ctypes.c_size_t), ("stream", ctypes.c_void_p),
                ("attrs", ctypes.c_void_p), ("nattrs", ctypes.c_uint)]
host_fn = ctypes.create_string_buffer(8)
rt.__cudaRegisterFunction(None, host_fn, None, b"probe_kernel", -1, None, None, None, None, None)
dev = ctypes.c_void_p()
rt.cudaMalloc(ctypes.byref(dev), ctypes.c_size_t(256))
def launch(ptr, stream=None):
    p = ctypes.c_void_p(ptr)
    n = ctypes.c_int(3)
    args = (ctypes.c_void_p * 2)(ctypes.cast(ctypes.byref(p), ctypes.c_void_p), ctypes.cast(ctypes.byref(n), ctypes.c_void_p))
    cfg = Config(Dim3(1, 1, 1), Dim3(32, 1, 1), 0, stream, None, 0)
    rt.cudaLaunchKernelExC(ctypes.byref(cfg), host_fn, args)
v0 = rt.audit_violations()
launch(dev.value + 64)
launch(0)
v1 = rt.audit_violations()
launch(ctypes.addressof(host_fn))
v2 = rt.audit_violations()
rt.cudaMallocAsync.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_void_p]
pooled = ctypes.c_void_p()
rt.cudaMallocAsync(ctypes.byref(pooled), 256, ctypes.c_void_p(0x1000))
launch(pooled.value, 0x1000)
v3 = rt.audit_violations()
launch(pooled.value, 0x2000)
print(v1 - v0, v2 - v1, v3 - v2, rt.audit_violations() - v3)
'''


def test_audit_sees_a_pointer_outside_the_device_allocations(audit_env, tmp_path):
    """A launch whose pointer parameter points into no device allocation is
    flagged, and so is one on another stream than its stream-ordered memory; a
    pointer into an allocation, or null, is not."""
    sigs = tmp_path / "sigs.txt"
    sigs.write_text("probe_kernel PS\n")
    script = tmp_path / "probe.py"
    script.write_text(CHECKER)
    env = dict(os.environ, AUDIT_SIGNATURES=str(sigs), AUDIT_LOG=str(tmp_path / "log.txt"))
    res = subprocess.run([sys.executable, str(script), os.path.join(audit_env["dir"], "libcudart.so.13")],
                         env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    assert res.stdout.split() == ["0", "1", "0", "1"]


def test_every_entry_point(audit_env):
    """Every entry point of the C ABI once per shape (right-hand side,
    linearizations, both operators and preconditioners, the linear solve, the
    w-updates with and without a handle, the per-stage timing, the internal
    arrays): every launch, copy and pointer within the limits, no CUDA error,
    and no allocation or free of any kind inside the handle-free w-update."""
    shapes = ["3,16,16,16", "2,194,33,64", "2,5,4,6", "1,6,7", "2,3,4,3,4", "4,6,5,7", "3,120,33,64:fp64"]
    env = dict(os.environ, LD_LIBRARY_PATH=audit_env["dir"], AUDIT_RESOURCES=audit_env["table"],
               AUDIT_SIGNATURES=audit_env["sigs"], AUDIT_FORBID_NULL_STREAM="1",
               AUDIT_LOG=os.path.join(audit_env["dir"], "launches_api.log"))
    res = subprocess.run([sys.executable, os.path.join(AUDIT, "run_shapes.py"), "--api", audit_env["lib"], *shapes],
                         env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    rows = [json.loads(line) for line in res.stdout.splitlines() if line.startswith("{")]
    assert [r["shape"] for r in rows] == shapes
    for r in rows:
        assert r["violations"] == 0, r
        assert r["launches"] >= 100, r
        assert not [e for e in r["errors"] if "CUDA error" in e or "out of memory" in e], r
        assert "wupdate_static allocated or freed memory" not in r["errors"], r


def test_serving_stream_in_arrival_order(audit_env):
    """The 256 requests of the serving stream, in arrival order, in one
    process (the order in which the fused pass's instances first ran when a
    shared-memory opt-in was missing): no launch refused, no CUDA error, and
    st_footprint above every handle's allocations.  Device memory is filled
    only in its first MiB so that the large requests fit in host memory."""
    import workloads as W
    reqs = W.serving_requests(n_req=256, seed=4, rate=1.0)
    shapes = [f'{r["desc"]["p"]},{r["desc"]["n_el"][0]},{r["desc"]["n_el"][1]},{r["desc"]["n_el_t"]}' for r in reqs]
    rows, _ = run(audit_env, shapes, AUDIT_FORBID_NULL_STREAM="1", AUDIT_FILL_BYTES=str(1 << 20))
    assert sum(r["violations"] for r in rows) == 0
    for r in rows:
        assert r["error"] is None or "CUDA error" not in r["error"], r
        assert r["peak_bytes"] <= r["footprint"], r


def test_entry_points_run_on_the_handles_device(audit_env):
    """A handle set up on device 0 and driven from a thread with device 1
    current: every launch still finds its memory on its own device, and the
    thread's device is restored on return."""
    env = dict(os.environ, LD_LIBRARY_PATH=audit_env["dir"], AUDIT_RESOURCES=audit_env["table"],
               AUDIT_SIGNATURES=audit_env["sigs"], AUDIT_LOG=os.path.join(audit_env["dir"], "launches_dev.log"))
    shapes = ["3,16,16,16", "2,194,33,64", "2,3,4,3,4"]
    res = subprocess.run([sys.executable, os.path.join(AUDIT, "run_shapes.py"), "--other-device", "1",
                          audit_env["lib"], *shapes], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    rows = [json.loads(line) for line in res.stdout.splitlines() if line.startswith("{")]
    assert [r["shape"] for r in rows] == shapes
    for r in rows:
        assert r["violations"] == 0, r
        assert r["error"] is None or ("CUDA error" not in r["error"] and "restored" not in r["error"]), r
    # and every other entry point the same way
    res = subprocess.run([sys.executable, os.path.join(AUDIT, "run_shapes.py"), "--api", "--other-device", "1",
                          audit_env["lib"], *shapes], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    rows = [json.loads(line) for line in res.stdout.splitlines() if line.startswith("{")]
    assert [r["shape"] for r in rows] == shapes
    for r in rows:
        assert r["violations"] == 0, r
        assert not [e for e in r["errors"] if "CUDA error" in e or "restored" in e], r
