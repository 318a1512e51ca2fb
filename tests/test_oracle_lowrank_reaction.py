"""Pins of the oracle's low-rank reaction coefficient (reading A7: the values
of C at the Greville grid, truncated like Theta-hat, interpolated
(d+1)-linearly at the Gauss points)."""

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from oracle.stabilization import greville_values


@pytest.mark.parametrize("d,p", [(1, 2), (2, 3), (3, 2)])
def test_greville_values_reproduce_bilinear_functions(d, p):
    """Linear precision in every direction: the spline whose coefficients are
    the products of Greville abscissae is t * x_0 * ... * x_{d-1}, so its
    values at the Greville grid are those products (the first time function,
    removed from X_t, has abscissa 0 and coefficient 0)."""
    desc = W.base_desc(d=d, p=p, n_el=[4, 5, 3][:d], n_el_t=5, T=3.0, D=[1e-3] * d)
    o = Oracle(desc)
    st = o.st
    gt = st.tdir.greville[1:]
    vec = gt.reshape([-1] + [1] * d)
    for pos in range(d):
        l = d - 1 - pos
        shape = [1] * (d + 1)
        shape[1 + pos] = st.n[l]
        vec = vec * st.sdirs[l].greville.reshape(shape)
    vec = vec.reshape(-1)
    got = greville_values(st, vec)
    assert np.abs(got - vec.reshape(st.N_t, st.N_s)).max() < 1e-13 * np.abs(vec).max()


def test_spatially_uniform_fields_give_rank_one():
    """Coefficients that do not depend on space give Greville values constant
    in space: the coefficient matrix has rank one at any tolerance."""
    desc = W.base_desc(d=2, p=2, n_el=[4, 3], n_el_t=6, T=3.0, D=[1e-3] * 2, eps_reaction=1e-13)
    desc.update(W.DIMENSIONAL_RM)
    o = Oracle(desc)
    st = o.st
    g = np.sin(np.arange(st.N_t) + 1.0)
    u = np.repeat(g, st.N_s)
    w = 0.3 * np.repeat(np.cos(np.arange(st.N_t)), st.N_s)
    _, U, s, V = o.reaction_lowrank(u, w, "picard")
    assert len(s) == 1


@pytest.mark.parametrize("kind", ["picard", "newton"])
def test_full_rank_reaction_converges_to_the_exact_one(kind):
    """With eps_reaction = 0 the coefficient is the (d+1)-linear interpolant of
    the exact one on the Greville grid: for smooth fields the operators differ
    by O(h^2), so the difference falls by about 4 per halving of the mesh (a
    transposed table or a wrong grid would not converge)."""
    errs = []
    for ne in (4, 8, 16):
        base = dict(d=1, p=2, n_el=[ne], n_el_t=ne, T=4.0, D=[1e-2], nonlinear=kind)
        desc = W.base_desc(**base, eps_reaction=0.0, stabilization="galerkin")
        desc.update(W.DIMENSIONAL_RM)
        o = Oracle(desc)
        u, w = W.wave_fields(desc, seed=2, speed=0.2, width=0.6)
        A_lr, _ = o.linearization(u, w, kind)
        exact = dict(desc, eps_reaction=-1.0)
        A_ex, _ = Oracle(exact).linearization(u, w, kind)
        x = W.random_vector(o.st.N_dof, seed=4)
        errs.append(np.linalg.norm((A_lr - A_ex) @ x) / np.linalg.norm(A_ex @ x))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > 1.6, (errs, rates)
