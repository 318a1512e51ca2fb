"""The oracle's full-size Theta-hat and low-rank SU rows (oracle/streamed.py)
equal the assembled oracle's on small meshes: the element maxima taken one
time element at a time with box maxima one axis after the other, against the
dense window loops of oracle/stabilization.py; the SU rows, against rows of
the assembled operator with theta interpolated from the low-rank table."""

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, model
from oracle import rows as OR
from oracle import streamed as S
from oracle.stabilization import low_rank

CASES = [dict(d=1, p=2, n_el=[7], n_el_t=9), dict(d=2, p=3, n_el=[4, 5], n_el_t=6),
         dict(d=3, p=2, n_el=[3, 4, 3], n_el_t=4)]
IDS = [f"d{c['d']}p{c['p']}" for c in CASES]


def problem(c, **over):
    desc = W.base_desc(d=c["d"], p=c["p"], n_el=c["n_el"], n_el_t=c["n_el_t"], T=8.0, C_m=1.0,
                       D=[2e-2, 1e-2, 5e-3][:c["d"]],
                       source=dict(kind="stim", boxes=[W.stim_box([0.0] * c["d"], [0.35] * c["d"], 0.0, 1.5, 1.0)]))
    desc.update(W.DIMENSIONAL_RM)
    desc.update(over)
    return desc


@pytest.mark.parametrize("c", CASES, ids=IDS)
@pytest.mark.parametrize("mode", ["literal", "symmetric"])
def test_streamed_theta_hat_equals_dense_windows(c, mode):
    desc = problem(c, suppext=mode)
    o = Oracle(desc)
    u, w = W.wave_fields(desc, seed=3, speed=0.2, width=0.3)
    info = o.ionic(u, w)
    th, sinfo = S.theta_hat(o.st, desc, u, w, mode)
    assert abs(sinfo["den"] - info["den"]) <= 1e-14 * info["den"]
    assert np.abs(th - info["theta_hat"]).max() <= 1e-13
    if c["d"] < 3:                                                # both branches of the min
        assert 0.0 < th.min() < 1.0 == th.max()
    assert np.abs(sinfo["r_max"] - np.abs(info["R"]).max()) <= 1e-13 * sinfo["r_max"]


@pytest.mark.parametrize("c", CASES, ids=IDS)
def test_su_rows_equal_assembled_rows(c):
    desc = problem(c, eps_theta=0.05)
    o = Oracle(desc)
    st = o.st
    n = st.N_dof
    u, w = W.wave_fields(desc, seed=3, speed=0.2, width=0.3)
    A, info = o.linearization(u, w, "picard")
    assert len(info["s"]) >= 1
    x = W.random_vector(n, seed=3)
    rng = np.random.Generator(np.random.PCG64(4))
    rows = np.unique(np.concatenate([[0, st.N_s - 1, n - 1], rng.integers(0, n, size=12)]))
    th, _ = S.theta_hat(st, desc, u, w)
    U, s, V = low_rank(th, desc["eps_theta"])
    terms = OR.picard_galerkin_terms(st, desc, u, w) + S.su_terms(st, desc, o.tau_q, U, s, V)
    got = OR.apply_rows(st, terms, rows, x)
    ref = (A @ x)[rows]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(A @ x).max()
