"""Checks of full-size results on rows the oracle computes one by one
(oracle/rows.py), shared by the GPU test at the workload's full size and its
CPU self-check on a small mesh.  Each check takes host arrays."""

import numpy as np

import workloads as W
from oracle import rows as OR


def sample_rows(st, desc, seed, n_random=48):
    """Rows at the corners of space-time, at t = 0 inside the stimulus box, and
    random rows."""
    n, N_s = st.N_dof, st.N_s
    fixed = [0, N_s - 1, n - N_s, n - 1, n // 2]
    box = desc["source"]["boxes"][0]
    idx = 0
    stride = 1
    for l in range(st.d):
        c = 0.5 * (box["lo"][l] + box["hi"][l])
        k = min(st.n[l] - 1, int(c * desc["n_el"][l]) + 1)
        idx += k * stride
        stride *= st.n[l]
    fixed += [idx + it * N_s for it in range(min(3, st.N_t))]
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.unique(np.concatenate([fixed, rng.integers(0, n, size=n_random)])).astype(np.int64)


def linearization_inputs(n):
    """Seeded fields for the linearization and seeded vectors for the operators."""
    return dict(u=0.1 * W.random_vector(n, seed=11), w=0.1 * W.random_vector(n, seed=12),
                x=W.random_vector(n, seed=13), r=W.random_vector(n, seed=14))


# Residual rows A-hat z - r of a preconditioner output z with forward error e
# (max norm, relative to max |z|) come out at about 500 e of max |r|: measured
# on the oracle's assembled A-hat of this workload at 648 and 12,274 unknowns,
# with z the direct solve plus absolute noise (the rounding pattern of a
# transform method).  The small meshes bound e by 1e-10, hence:
PRECOND_RESIDUAL_TOL = 5e-8


def check_rhs(st, desc, rows, f):
    ref = OR.load_rows(st, OR.source_fn(st, desc), rows)
    err = np.abs(f[rows] - ref).max()
    assert err <= 1e-12 * np.abs(f).max(), err
    return ref


def check_apply(st, desc, rows, inp, y, tol):
    ref = OR.apply_rows(st, OR.picard_galerkin_terms(st, desc, inp["u"], inp["w"]), rows, inp["x"])
    err = np.abs(y[rows] - ref).max()
    assert err <= tol * np.abs(y).max(), (err, np.abs(y).max())


def check_precond(st, desc, rows, inp, z, tol):
    res = OR.apply_rows(st, OR.precond_terms(st, desc), rows, z) - inp["r"][rows]
    err = np.abs(res).max()
    assert err <= tol * np.abs(inp["r"]).max(), err


def check_solution(st, desc, rows, inp, f_rows, f_norm, x, rtol):
    """A row of f - A x is at most the residual norm, which the solve bounds by
    rtol ||f||."""
    res = f_rows - OR.apply_rows(st, OR.picard_galerkin_terms(st, desc, inp["u"], inp["w"]), rows, x)
    err = np.abs(res).max()
    assert err <= rtol * f_norm, (err, rtol * f_norm)
