"""The allocation-free w-update (st_wupdate_static) against st_wupdate.

The file name keeps it late in collection, after the parity, serving and
tensor-core tests have used the device.  Two calls in a row on different problems (the
second overwrites the fixed device scratch with other bands), then a problem
that fills the scratch exactly; each result is compared with st_wupdate on a
handle set up from the same description, at the tolerance of the FP64
w-update parity test.  A problem one time function larger is rejected before
any device work.
"""

import os
import shutil

import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import library, dev, empty, host, ptr, stream, rel


def problem(d, p, n_el, n_el_t):
    desc = W.base_desc(d=d, p=p, n_el=n_el, n_el_t=n_el_t, T=8.0, C_m=1.0, D=[2e-2, 1e-2, 5e-3][:d],
                       source=dict(kind="stim", boxes=[W.stim_box([0.0] * d, [0.35] * d, 0.0, 1.5, 1.0)]))
    desc.update(W.DIMENSIONAL_RM)
    desc.update(b=0.05, d_e=1.3, gmres_m=20)
    return desc


def n_dof(desc):
    ns = int(np.prod([n + desc["p"] for n in desc["n_el"]]))
    return ns * (desc["n_el_t"] + desc["p"] - 1)


def compare(P, desc, seed):
    n = n_dof(desc)
    du = dev(W.random_vector(n, seed=seed))
    w_static = empty(n)
    P.wupdate_static(desc, ptr(du), ptr(w_static), stream())
    s = P.Solver(desc, stream())
    w_handle = empty(n)
    s.wupdate(ptr(du), ptr(w_handle))
    a, b = host(w_static), host(w_handle)
    s.close()
    assert np.all(np.isfinite(a))
    assert rel(a, b) < 1e-12
    return a


@pytest.mark.gpu
def test_two_calls_in_a_row_match_st_wupdate():
    P = library()
    compare(P, problem(2, 3, [5, 4], 6), seed=13)
    compare(P, problem(3, 2, [3, 4, 3], 9), seed=14)


@pytest.mark.gpu
def test_scratch_filled_exactly():
    P = library()
    desc = problem(1, 4, [2], 4093)        # N_t = 4096: 2 * 4096 * 9 doubles
    assert 2 * (desc["n_el_t"] + 3) * 9 == P.ST_WUPDATE_STATIC_CAPACITY
    compare(P, desc, seed=15)


def test_oversized_problem_is_rejected():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2311_17500_gb300 import build
    build.build()
    import paper_2311_17500_gb300 as P
    desc = problem(1, 4, [2], 4094)        # N_t = 4097: one time function too many
    with pytest.raises(P.StError) as e:
        P.wupdate_static(desc, 16, 4096, 0)   # nonzero placeholders: rejected before any use
    assert e.value.code == P.ST_ERR_CAPACITY
    assert "ST_WUPDATE_STATIC_CAPACITY" in str(e.value)
