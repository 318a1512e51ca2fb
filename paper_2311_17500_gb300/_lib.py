"""ctypes binding of libst.so (include/st.h).

Argument marshalling only: problem dictionaries become the C struct, device
pointers are passed as integers, status codes become exceptions.  Every
computation happens inside the library's CUDA kernels.  There is no CPU
fallback: loading fails loudly when the library is missing.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libst.so")

ST_OK, ST_ERR_ARG, ST_ERR_OOM, ST_ERR_CUDA, ST_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
ST_ERR_BREAKDOWN, ST_ERR_NAN, ST_ERR_TIMEOUT, ST_ERR_STATE, ST_ERR_CAPACITY = 5, 6, 7, 8, 9
ST_WUPDATE_STATIC_CAPACITY = 73728
ST_SRC = {"zero": 0, "stim": 1, "heat_mms": 2, "e1_mms": 3}
ST_GALERKIN, ST_SU = 0, 1
ST_PICARD, ST_NEWTON = 0, 1
ST_FP64, ST_MIXED = 0, 1
ST_SUPPEXT = {"literal": 0, "symmetric": 1}
ST_FORM = {"auto": 0, "bands": 1, "lean": 2}
ST_INNER = {"auto": 0, "fp32": 1, "df": 2}
ST_PRECOND = {"auto": 0, "tf32": 1, "fp32": 2, "fp64": 3}
ST_MAX_STIM = 8
GET = dict(theta_hat=0, lowrank_s=1, lowrank_u=2, lowrank_v=3, tau_q=4, fd_eig=5, bands_1d=6, reaction_s=7,
           reaction_u=8, reaction_v=9, reaction_tb=10)

EXPORTS = ["st_footprint", "st_setup", "st_destroy", "st_error_string", "st_get_dims", "st_ionic",
           "st_linearize", "st_apply", "st_precond", "st_linsolve", "st_wupdate", "st_rhs", "st_solve",
           "st_get", "st_profile", "st_profile_read", "st_launch_count",
           "st_tc_selftest", "st_wupdate_static", "st_last_cuda_error"]
STAGES = ["kron", "interp", "qband", "fd_gemm", "fd_lu", "arnoldi", "ionic", "lowrank", "apply64"]


class StStim(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("amp", ctypes.c_double)]


class StProblemDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("p", ctypes.c_int), ("n_el", ctypes.c_int * 3), ("n_el_t", ctypes.c_int),
                ("T", ctypes.c_double), ("C_m", ctypes.c_double), ("D", ctypes.c_double * 3),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c1", ctypes.c_double),
                ("c2", ctypes.c_double), ("d_e", ctypes.c_double),
                ("source_kind", ctypes.c_int), ("n_stim", ctypes.c_int), ("stim", StStim * ST_MAX_STIM),
                ("stabilization", ctypes.c_int), ("suppext", ctypes.c_int), ("eps_theta", ctypes.c_double),
                ("nonlinear", ctypes.c_int), ("alpha", ctypes.c_double), ("delta", ctypes.c_double),
                ("max_fp", ctypes.c_int), ("fix_w_zero", ctypes.c_int), ("precision", ctypes.c_int),
                ("gmres_m", ctypes.c_int), ("rtol", ctypes.c_double), ("max_it", ctypes.c_int),
                ("operator_form", ctypes.c_int), ("inner_op", ctypes.c_int),
                ("eps_reaction", ctypes.c_double),
                ("breaks", ctypes.POINTER(ctypes.c_double) * 3), ("breaks_t", ctypes.POINTER(ctypes.c_double)),
                ("precond_arith", ctypes.c_int)]


class StDims(ctypes.Structure):
    _fields_ = [("N_s", ctypes.c_longlong), ("N_t", ctypes.c_longlong), ("N_dof", ctypes.c_longlong),
                ("Q_s", ctypes.c_longlong), ("n", ctypes.c_int * 3), ("operator_form", ctypes.c_int),
                ("precond_tc", ctypes.c_int)]


class StIonicInfo(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("u_max", ctypes.c_double), ("ut_max", ctypes.c_double),
                ("den", ctypes.c_double), ("r_max", ctypes.c_double), ("theta_fro", ctypes.c_double),
                ("rank_reaction", ctypes.c_int)]


class StStats(ctypes.Structure):
    _fields_ = [("fp_iters", ctypes.c_int), ("gmres_iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("total_gmres", ctypes.c_int), ("rank", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("last_diff", ctypes.c_double)]


def _struct_dict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


class StError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg}: status {code}")
        self.code = code


_lib = None


def load(path=None):
    """Load libst.so (raises OSError when it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or LIB_PATH)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    P = ctypes.POINTER
    lib.st_footprint.argtypes = [P(StProblemDesc), P(sz)]
    lib.st_setup.argtypes = [P(StProblemDesc), vp, P(vp)]
    lib.st_destroy.argtypes = [vp]
    lib.st_error_string.argtypes = [i]
    lib.st_error_string.restype = ctypes.c_char_p
    lib.st_get_dims.argtypes = [vp, P(StDims)]
    lib.st_ionic.argtypes = [vp, vp, vp, P(StIonicInfo)]
    lib.st_linearize.argtypes = [vp, vp, vp, i, i, P(StIonicInfo)]
    lib.st_apply.argtypes = [vp, i, vp, vp]
    lib.st_precond.argtypes = [vp, i, vp, vp]
    lib.st_linsolve.argtypes = [vp, vp, vp, P(StStats)]
    lib.st_wupdate.argtypes = [vp, vp, vp]
    lib.st_wupdate_static.argtypes = [P(StProblemDesc), vp, vp, vp]
    lib.st_rhs.argtypes = [vp, vp]
    lib.st_solve.argtypes = [vp, vp, vp, P(StStats)]
    lib.st_get.argtypes = [vp, i, vp, sz]
    lib.st_profile.argtypes = [vp, i]
    d = ctypes.c_double
    lib.st_profile_read.argtypes = [vp, i, P(d), P(d), P(d), P(ctypes.c_longlong)]
    lib.st_tc_selftest.argtypes = [P(i), P(ctypes.c_double)]
    lib.st_launch_count.argtypes = []
    lib.st_launch_count.restype = ctypes.c_longlong
    lib.st_last_cuda_error.argtypes = []
    lib.st_last_cuda_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("st_error_string", "st_launch_count", "st_last_cuda_error"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def make_desc(desc):
    """C description from a problem dictionary (see workloads)."""
    c = StProblemDesc()
    c.d = int(desc["d"])
    c.p = int(desc["p"])
    for l in range(3):
        c.n_el[l] = int(desc["n_el"][l]) if l < c.d else 1
        c.D[l] = float(desc["D"][l]) if l < c.d else 1.0
    c.n_el_t = int(desc["n_el_t"])
    c.T, c.C_m = float(desc["T"]), float(desc["C_m"])
    c.a, c.b, c.c1, c.c2, c.d_e = (float(desc[k]) for k in ("a", "b", "c1", "c2", "d_e"))
    src = desc["source"]
    c.source_kind = ST_SRC[src["kind"]]
    boxes = src.get("boxes", []) if src["kind"] == "stim" else []
    if len(boxes) > ST_MAX_STIM:
        raise ValueError("too many stimulus boxes")
    c.n_stim = len(boxes)
    for k, bx in enumerate(boxes):
        for l in range(min(c.d, 3)):   # d > 3 is left to the library to reject
            c.stim[k].lo[l] = bx["lo"][l]
            c.stim[k].hi[l] = bx["hi"][l]
        c.stim[k].t0, c.stim[k].t1, c.stim[k].amp = bx["t0"], bx["t1"], bx["amp"]
    c.stabilization = ST_SU if desc["stabilization"] == "su" else ST_GALERKIN
    c.suppext = ST_SUPPEXT[desc.get("suppext", "literal")]
    c.eps_theta = float(desc["eps_theta"])
    c.nonlinear = ST_NEWTON if desc["nonlinear"] == "newton" else ST_PICARD
    c.alpha, c.delta = float(desc["alpha"]), float(desc["delta"])
    c.max_fp = int(desc["max_fp"])
    c.fix_w_zero = 1 if desc.get("fix_w_zero") else 0
    c.precision = ST_MIXED if desc["precision"] == "mixed" else ST_FP64
    c.gmres_m = int(desc["gmres_m"])
    c.rtol = float(desc["rtol"])
    c.max_it = int(desc["max_it"])
    c.operator_form = ST_FORM[desc.get("operator_form", "auto")]
    c.inner_op = ST_INNER[desc.get("inner_op", "auto")]
    c.eps_reaction = float(desc.get("eps_reaction", -1.0))
    # breakpoint arrays (None = uniform): the struct keeps the ctypes arrays alive
    keep = []

    def darr(vals):
        a = (ctypes.c_double * len(vals))(*[float(v) for v in vals])
        keep.append(a)
        return ctypes.cast(a, ctypes.POINTER(ctypes.c_double))

    breaks = desc.get("breaks") or [None] * c.d
    for l in range(min(c.d, 3)):
        if breaks[l] is not None:
            c.breaks[l] = darr(breaks[l])
    if desc.get("breaks_t") is not None:
        c.breaks_t = darr(desc["breaks_t"])
    c._keep = keep
    c.precond_arith = ST_PRECOND[desc.get("precond_arith", "auto")]
    return c


def _check(code, what):
    if code != ST_OK:
        lib = load()
        msg = lib.st_error_string(code).decode()
        if code in (ST_ERR_CUDA, ST_ERR_OOM):
            detail = lib.st_last_cuda_error().decode()
            if detail:
                msg += ": " + detail
        raise StError(code, f"{what} failed ({msg})")


def tc_selftest():
    """(usable, max_rel_err) of the tensor-core transform self-test."""
    lib = load()
    u, e = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib.st_tc_selftest(ctypes.byref(u), ctypes.byref(e)), "st_tc_selftest")
    return bool(u.value), e.value


def wupdate_static(desc, u_ptr, w_ptr, stream=0):
    """Handle-free w-update into the library's fixed device scratch
    (st_wupdate_static); raises StError(ST_ERR_CAPACITY) when
    2 N_t (2p+1) exceeds ST_WUPDATE_STATIC_CAPACITY doubles."""
    lib = load()
    c = make_desc(desc)
    _check(lib.st_wupdate_static(ctypes.byref(c), ctypes.c_void_p(u_ptr), ctypes.c_void_p(w_ptr),
                                 ctypes.c_void_p(stream)), "st_wupdate_static")


def footprint(desc):
    lib = load()
    c = make_desc(desc)
    out = ctypes.c_size_t(0)
    _check(lib.st_footprint(ctypes.byref(c), ctypes.byref(out)), "st_footprint")
    return out.value


class Solver:
    """One st_handle.  Vector arguments are raw device pointers (ints)."""

    def __init__(self, desc, stream=0):
        self.lib = load()
        self._c = make_desc(desc)
        h = ctypes.c_void_p()
        _check(self.lib.st_setup(ctypes.byref(self._c), ctypes.c_void_p(stream), ctypes.byref(h)), "st_setup")
        self.h = h
        dims = StDims()
        _check(self.lib.st_get_dims(self.h, ctypes.byref(dims)), "st_get_dims")
        self.dims = _struct_dict(dims)
        self.dims["n"] = list(dims.n)

    def close(self):
        if self.h:
            self.lib.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ionic(self, u_ptr, w_ptr):
        info = StIonicInfo()
        _check(self.lib.st_ionic(self.h, ctypes.c_void_p(u_ptr), ctypes.c_void_p(w_ptr), ctypes.byref(info)),
               "st_ionic")
        return _struct_dict(info)

    def linearize(self, u_ptr, w_ptr, kind, keep_theta=False):
        info = StIonicInfo()
        k = ST_NEWTON if kind == "newton" else ST_PICARD
        _check(self.lib.st_linearize(self.h, ctypes.c_void_p(u_ptr), ctypes.c_void_p(w_ptr), k,
                                     1 if keep_theta else 0, ctypes.byref(info)), "st_linearize")
        return _struct_dict(info)

    def apply(self, x_ptr, y_ptr, prec=ST_FP64):
        _check(self.lib.st_apply(self.h, prec, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr)), "st_apply")

    def precond(self, r_ptr, z_ptr, prec=ST_FP64):
        _check(self.lib.st_precond(self.h, prec, ctypes.c_void_p(r_ptr), ctypes.c_void_p(z_ptr)), "st_precond")

    def linsolve(self, b_ptr, x_ptr, allow_unconverged=False):
        st = StStats()
        code = self.lib.st_linsolve(self.h, ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr), ctypes.byref(st))
        if not (allow_unconverged and code == ST_ERR_NOT_CONVERGED):
            _check(code, "st_linsolve")
        out = _struct_dict(st)
        out["status"] = code
        return out

    def wupdate(self, u_ptr, w_ptr):
        _check(self.lib.st_wupdate(self.h, ctypes.c_void_p(u_ptr), ctypes.c_void_p(w_ptr)), "st_wupdate")

    def rhs(self, f_ptr):
        _check(self.lib.st_rhs(self.h, ctypes.c_void_p(f_ptr)), "st_rhs")

    def solve(self, u_ptr, w_ptr, allow_unconverged=False):
        st = StStats()
        code = self.lib.st_solve(self.h, ctypes.c_void_p(u_ptr), ctypes.c_void_p(w_ptr), ctypes.byref(st))
        if not (allow_unconverged and code == ST_ERR_NOT_CONVERGED):
            _check(code, "st_solve")
        out = _struct_dict(st)
        out["status"] = code
        return out

    def profile(self, enable):
        _check(self.lib.st_profile(self.h, 1 if enable else 0), "st_profile")

    def profile_read(self):
        """{stage: dict(ms, bytes, flops, launches)} of the recorded launches."""
        out = {}
        for k, name in enumerate(STAGES):
            ms, b, f, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
            _check(self.lib.st_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(b), ctypes.byref(f),
                                            ctypes.byref(n)), "st_profile_read")
            out[name] = dict(ms=ms.value, bytes=b.value, flops=f.value, launches=n.value)
        return out

    def get(self, what, count):
        """Copy an internal FP64 array of `count` values to a host bytes buffer."""
        buf = (ctypes.c_double * max(count, 1))()
        _check(self.lib.st_get(self.h, GET[what], ctypes.cast(buf, ctypes.c_void_p), 8 * count), "st_get")
        return list(buf)[:count]
