"""Selected rows of the space-time operators and of the load vector, at any
problem size, for the oracle.

Row i of A x (Eq. lin_sys_A) is the integral of the operator's integrand
against the test function v_i = b_{i_t+1}(t) B_{i_s}(x) (the first time
function is removed, Sec. 2).  It involves only the space-time elements in
the support of v_i: (p+1) time elements times (p+1)^d spatial elements.
Evaluating those elements' Gauss-point integrands from the coefficient
vectors gives the row exactly as the assembled matrix of `SpaceTime.assemble`
does: the same Gauss rule and the same tables, restricted to those elements
(local_table, local_glob), so a full-size problem never assembles or stores a
space-time array.

Operators are given as terms (coef_fn, kt_test, ks_test, kt_trial, ks_trial)
like `SpaceTime.assemble`'s, with coef_fn(et, es) returning the integrand
coefficient at the Gauss points of time element et and the spatial elements
es, shape (len(es), nq_t, nq_s).

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np

from . import model


def local_table(st, ks, es):
    """The spatial basis table of `SpaceTime.stab` for the spatial elements es
    only: T[e, qs, ls] = prod_l vals_l[k_l][e_l, q_l, local_l(e_l)[a_l]], with
    es, qs and ls colexicographic (direction 0 fastest)."""
    es = np.asarray(es)
    tab = None
    rem = es.copy()
    for l, dr in enumerate(st.sdirs):
        e_l = rem % dr.n_el
        rem = rem // dr.n_el
        loc = np.array([dr.local[e] for e in e_l])                     # (E, p+1)
        t_l = dr.vals[ks[l]][e_l[:, None], :, loc].transpose(0, 2, 1)  # (E, nq, p+1)
        if tab is None:
            tab = t_l
        else:
            E, Q, A = tab.shape
            tab = np.einsum('eqa,epb->epqba', tab, t_l).reshape(E, t_l.shape[1] * Q, t_l.shape[2] * A)
    return tab


def local_glob(st, et, es):
    """Global dof of (a_t, l_s) on the elements (et, es), -1 where the removed
    first time function would be: (len(es), p+1, L_s)."""
    it = st.tglob[et]
    g = it[None, :, None] * st.N_s + st.sglob[es][:, None, :]
    g[:, it < 0, :] = -1
    return g


def support(st, i):
    """(time index i_t, spatial index i_s, time elements, spatial elements) of
    the support of test function i."""
    it, i_s = divmod(int(i), st.N_s)
    ets = [et for et in range(st.n_el_t) if it in st.tglob[et]]
    ess = np.nonzero((st.sglob == i_s).any(axis=1))[0]
    return it, i_s, ets, ess


def local_field(st, vec, et, es, kt=0, ks=None):
    """Derivative (kt in time, ks per spatial direction) of the spline with
    coefficients `vec` at the Gauss points of (et, es): (len(es), nq_t, nq_s)."""
    ks = (0,) * st.d if ks is None else tuple(ks)
    g = local_glob(st, et, es)                                  # (E, p+1, L_s)
    c = np.where(g >= 0, vec[np.maximum(g, 0)], 0.0)
    return np.einsum('eal,ta,eql->etq', c, st.ttab[kt][et], local_table(st, ks, es))


def apply_rows(st, terms, rows, x):
    """(A x)[rows] for the operator A = sum of the terms (see the module header)."""
    out = np.zeros(len(rows))
    for r, i in enumerate(rows):
        it, i_s, ets, ess = support(st, i)
        acc = 0.0
        for et in ets:
            a_i = int(np.nonzero(st.tglob[et] == it)[0][0])
            l_i = np.array([int(np.nonzero(st.sglob[e] == i_s)[0][0]) for e in ess])
            g = local_glob(st, et, ess)
            xl = np.where(g >= 0, x[np.maximum(g, 0)], 0.0)         # (E, p+1, L_s)
            wt = st.tdir.wq[et]
            for coef_fn, kti, ksi, ktj, ksj in terms:
                W = coef_fn(et, ess) * wt[None, :, None] * st.ws[ess][:, None, :]
                Si = local_table(st, ksi, ess)[np.arange(len(ess)), :, l_i]      # (E, nq_s)
                trial = np.einsum('tb,eqm,ebm->etq', st.ttab[ktj][et], local_table(st, ksj, ess), xl)
                acc += np.einsum('etq,t,eq,etq->', W, st.ttab[kti][et][:, a_i], Si, trial)
        out[r] = acc
    return out


def load_rows(st, coef_fn, rows, kt=0, ks=None):
    """(int int coef v_i)[rows] with coef_fn as in the operator terms."""
    ks = (0,) * st.d if ks is None else tuple(ks)
    out = np.zeros(len(rows))
    for r, i in enumerate(rows):
        it, i_s, ets, ess = support(st, i)
        for et in ets:
            a_i = int(np.nonzero(st.tglob[et] == it)[0][0])
            l_i = np.array([int(np.nonzero(st.sglob[e] == i_s)[0][0]) for e in ess])
            W = coef_fn(et, ess) * st.tdir.wq[et][None, :, None] * st.ws[ess][:, None, :]
            Si = local_table(st, ks, ess)[np.arange(len(ess)), :, l_i]
            out[r] += np.einsum('etq,t,eq->', W, st.ttab[kt][et][:, a_i], Si)
    return out


def constant(st, value):
    return lambda et, es: np.full((len(es), st.nq_t, st.nq_s), float(value))


def linear_terms(st, C_m, D):
    """int int C_m d_t u v + grad u . D grad v (the linear part of A, Sec. 3)."""
    z = (0,) * st.d
    terms = [(constant(st, C_m), 0, z, 1, z)]
    for l in range(st.d):
        terms.append((constant(st, D[l]), 0, st.unit(l, 1), 0, st.unit(l, 1)))
    return terms


def picard_galerkin_terms(st, desc, u, w):
    """A of the fixed-point step without stabilization (Eq. lin_sys_A with the
    SU term left out): the linear part plus int int C_r(u, w) u v, with C_r of
    Eq. reaction evaluated at the Gauss points from the coefficient vectors."""
    z = (0,) * st.d

    def reaction(et, es):
        return model.reaction_coef(desc, local_field(st, u, et, es), local_field(st, w, et, es))

    return linear_terms(st, desc["C_m"], desc["D"]) + [(reaction, 0, z, 0, z)]


def precond_terms(st, desc):
    """A-hat of Eq. preconditioner with the conductivity scaling D_ll."""
    z = (0,) * st.d
    return linear_terms(st, desc["C_m"], desc["D"]) + [(constant(st, desc["a"] * desc["c1"]), 0, z, 0, z)]


def source_fn(st, desc):
    """f at the Gauss points of (et, es) (the stimulus or manufactured source)."""
    def f(et, es):
        xs = [x[es][:, None, :] for x in st.xs]                  # (E, 1, nq_s)
        t = st.tdir.xq[et][None, :, None]                         # (1, nq_t, 1)
        return model.source(desc, xs, t) * np.ones((len(es), st.nq_t, st.nq_s))
    return f
