"""C^0-in-time SUPG with shock capturing: the comparison method of Sec. 4.2.

Discrete space: splines of degree p of maximal regularity in space and of
continuity C^0 in time (every interior time breakpoint repeated p times in the
knot vector, so N_t = p n_el_t once the first time function is removed).  The
SU term of the fixed-point scheme (Eq. solverSU_approx) is replaced by

  S_SUPG(u~, v) = h / (2p+1) int int (C_m d_t u~ - div(D grad u~)
                                      + C_r(u^k, w^k) u~ - f) d_t v,
  S_SC(u~, v)   = c h^2 / 4 int int |R(u^k, w^k)| / (C_m (||u^k||_inf / T
                                      + ||d_t u^k||_inf)) d_t u~ d_t v,

with R the residual of eq. 3.1 at the iterate.  The f part of S_SUPG moves to
the right-hand side: F = int int f v + h / (2p+1) int int f d_t v.

Readings where the paper is silent:
  * h is the length of the time element (physical units).  The SUPG direction
    is the time direction, the one the test derivative d_t v follows.
  * c = 1: the constant of the shock-capturing term is not given.
  * The S_SC coefficient is taken pointwise at the Gauss points.  Its
    denominator uses the maxima over all Gauss points, as Theta-hat does, and
    the coefficient is 0 where that denominator vanishes (the zero iterate,
    which has no front to capture).
  * The low-rank replacement of C_r and of the S_SC coefficient, which the
    paper uses to speed up its fixed point, is not taken here: the oracle
    keeps the plain definition.

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np


def time_h(st):
    """Length of each time element in physical units, shape (n_el_t,)."""
    return np.diff(st.tdir.br) * st.T


def _per_time_element(st, s):
    """Scale per time element broadcast to the Gauss-point layout of `assemble`."""
    return s[:, None, None, None] * np.ones((st.n_el_t, st.N_el_s, st.nq_t, st.nq_s))


def supg_terms(st, C_m, D, cr_q):
    """Terms of S_SUPG without its f part: test function d_t v, trial functions
    C_m d_t u, -D_ll d_ll u (l = 1..d) and C_r u."""
    s = _per_time_element(st, time_h(st) / (2 * st.p + 1))
    z = (0,) * st.d
    terms = [(C_m * s, 1, z, 1, z)]
    for l in range(st.d):
        terms.append((-D[l] * s, 1, z, 0, st.unit(l, 2)))
    terms.append((s * cr_q, 1, z, 0, z))
    return terms


def supg_load(st, f_q):
    """The f part of S_SUPG on the right-hand side: h/(2p+1) int int f d_t v."""
    s = _per_time_element(st, time_h(st) / (2 * st.p + 1))
    return st.load(s * f_q, kt=1)


def sc_coefficient(R, u_q, ut_q, C_m, T):
    """|R| / (C_m (max|u| / T + max|d_t u|)) at every Gauss point; 0 where the
    denominator vanishes."""
    den = C_m * (np.abs(u_q).max() / T + np.abs(ut_q).max())
    if not den > 0.0:
        return np.zeros_like(R), den
    return np.abs(R) / den, den


def sc_terms(st, coef_q, c=1.0):
    """Terms of S_SC: c h^2/4 int int coef d_t u d_t v."""
    h = time_h(st)
    s = _per_time_element(st, c * h * h / 4.0)
    z = (0,) * st.d
    return [(s * coef_q, 1, z, 1, z)]
