"""Selected rows of the oracle's operators (oracle/rows.py) equal the same rows
of the assembled matrices: the row evaluation that the full-size GPU checks use
integrates only over the support of each test function, with the same Gauss
rule and tables as the assembly."""

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, model
from oracle import rows as OR

CASES = [dict(d=1, p=2, n_el=[7], n_el_t=9), dict(d=2, p=3, n_el=[4, 5], n_el_t=5),
         dict(d=2, p=1, n_el=[6, 5], n_el_t=7), dict(d=3, p=2, n_el=[3, 4, 3], n_el_t=4)]


def problem(c):
    desc = W.base_desc(d=c["d"], p=c["p"], n_el=c["n_el"], n_el_t=c["n_el_t"], T=8.0, C_m=1.0,
                       D=[2e-2, 1e-2, 5e-3][:c["d"]], stabilization="galerkin",
                       source=dict(kind="stim", boxes=[W.stim_box([0.0] * c["d"], [0.35] * c["d"], 0.0, 1.5, 1.0)]))
    desc.update(W.DIMENSIONAL_RM)
    return desc


def some_rows(n, N_s, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    fixed = [0, N_s - 1, n - N_s, n - 1, n // 2]
    return np.unique(np.concatenate([fixed, rng.integers(0, n, size=12)]))


@pytest.mark.parametrize("c", CASES, ids=[f"d{c['d']}p{c['p']}" for c in CASES])
def test_rows_equal_assembled_rows(c):
    desc = problem(c)
    o = Oracle(desc)
    st = o.st
    n = st.N_dof
    u = 0.3 * W.random_vector(n, seed=1)
    w = 0.3 * W.random_vector(n, seed=2)
    x = W.random_vector(n, seed=3)
    rows = some_rows(n, st.N_s, seed=4)
    fl = o.fields(u, w)
    A = o.operator(model.reaction_coef(desc, fl["u"], fl["w"]))
    ref = (A @ x)[rows]
    got = OR.apply_rows(st, OR.picard_galerkin_terms(st, desc, u, w), rows, x)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(A @ x).max()
    Ah = o.precond_matrix()
    got = OR.apply_rows(st, OR.precond_terms(st, desc), rows, x)
    assert np.abs(got - (Ah @ x)[rows]).max() <= 1e-13 * np.abs(Ah @ x).max()
    got = OR.load_rows(st, OR.source_fn(st, desc), rows)
    assert np.abs(got - o.F[rows]).max() <= 1e-14 * max(np.abs(o.F).max(), 1e-300)


def test_full_size_checks_on_a_small_mesh():
    """The checks of the full-size GPU test, fed with the assembled oracle's own
    results on a small mesh of the same kind: they pass on exact answers and fail
    on a perturbed one."""
    import scipy.sparse.linalg as spla
    from tests import sampled_rows as SR
    desc = W.config("c2_aniso_2d", scale=dict(n_el=[6, 5], n_el_t=7))
    desc["stabilization"] = "galerkin"
    o = Oracle(desc)
    st = o.st
    inp = SR.linearization_inputs(st.N_dof)
    rows = SR.sample_rows(st, desc, seed=5, n_random=20)
    f = o.F
    f_rows = SR.check_rhs(st, desc, rows, f)
    fl = o.fields(inp["u"], inp["w"])
    A = o.operator(model.reaction_coef(desc, fl["u"], fl["w"]))
    SR.check_apply(st, desc, rows, inp, A @ inp["x"], 1e-12)
    z = spla.spsolve(o.precond_matrix().tocsc(), inp["r"])
    SR.check_precond(st, desc, rows, inp, z, 1e-9)   # exact solve: far below SR.PRECOND_RESIDUAL_TOL
    x = spla.spsolve(A.tocsc(), f)
    SR.check_solution(st, desc, rows, inp, f_rows, np.linalg.norm(f), x, 1e-8)
    bad = A @ inp["x"]
    bad[rows[len(rows) // 2]] *= 1.0 + 1e-9
    with pytest.raises(AssertionError):
        SR.check_apply(st, desc, rows, inp, bad, 1e-12)


@pytest.mark.parametrize("c", CASES, ids=[f"d{c['d']}p{c['p']}" for c in CASES])
def test_local_tables_equal_the_global_ones(c):
    from oracle.spacetime import SpaceTime
    st = SpaceTime(problem(c))
    es = np.arange(st.N_el_s)[::2]
    for ks in [(0,) * st.d] + [st.unit(l, k) for l in range(st.d) for k in (1, 2)]:
        assert np.array_equal(OR.local_table(st, ks, es), st.stab(ks)[es])
    for et in range(st.n_el_t):
        assert np.array_equal(OR.local_glob(st, et, es), st.glob(et)[es])


@pytest.mark.parametrize("name", ["c2_aniso_2d", "c3_cube_3d"])
def test_full_size_oracle_side_runs(name):
    """The oracle's part of the full-size GPU checks at the workloads' real
    sizes (4.43 M and 37.1 M unknowns): the sampled rows of f, of both
    operators and of the preconditioner come out finite, in seconds, and the
    rows hit the stimulus."""
    from oracle.spacetime import SpaceTime
    from tests import sampled_rows as SR
    desc = W.config(name)
    desc.update(stabilization="galerkin", precision="mixed")
    st = SpaceTime(desc)
    rows = SR.sample_rows(st, desc, seed=5)
    inp = SR.linearization_inputs(st.N_dof)
    f = OR.load_rows(st, OR.source_fn(st, desc), rows)
    y = OR.apply_rows(st, OR.picard_galerkin_terms(st, desc, inp["u"], inp["w"]), rows, inp["x"])
    z = OR.apply_rows(st, OR.precond_terms(st, desc), rows, inp["r"])
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(y)) and np.all(np.isfinite(z))
    assert np.abs(f).max() > 0.0 and np.abs(y).max() > 0.0
