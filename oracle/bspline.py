"""Univariate splines for the oracle (Sec. 2 of the paper).

Open knot vectors, B-splines by the Cox-de Boor recursion (values and
derivatives through the degree recursion), Greville abscissae, Gauss-Legendre
rules per knot span, and the per-direction tables the space-time assembly uses.

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np


def open_uniform_knots(n_el, p):
    """Open knot vector on [0, 1] with n_el equal spans: p+1 repeated end knots
    (Sec. 2, the knot vector Xi-hat).  Length n + p + 1 with n = n_el + p."""
    inner = np.arange(1, n_el, dtype=float) / n_el
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def _ratio(num, den):
    """num / den with the B-spline convention 0/0 := 0 (den == 0 only when a
    repeated knot makes the lower-degree function vanish identically)."""
    if den == 0.0:
        return np.zeros_like(num)
    return num / den


def bspline_all(knots, p, x, deriv=0):
    """All B-splines b_{i,p} of the knot vector (i = 0..n-1), or their `deriv`-th
    derivative, at the points x.  Returns an array of shape (len(x), n).

    Degree 0: indicator of [xi_i, xi_{i+1}), the last non-empty span closed on
    the right so that the basis is complete at x = xi_end.
    Degree q > 0, value: the Cox-de Boor convex combination
        b_{i,q} = (x - xi_i)/(xi_{i+q} - xi_i) b_{i,q-1}
                + (xi_{i+q+1} - x)/(xi_{i+q+1} - xi_{i+1}) b_{i+1,q-1}.
    Degree q > 0, k-th derivative:
        b_{i,q}^(k) = q [ b_{i,q-1}^(k-1)/(xi_{i+q} - xi_i)
                        - b_{i+1,q-1}^(k-1)/(xi_{i+q+1} - xi_{i+1}) ].
    """
    knots = np.asarray(knots, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    m = len(knots) - 1  # number of degree-0 functions

    def rec(q, k):
        if q == 0:
            if k > 0:
                return np.zeros((len(x), m))
            out = np.zeros((len(x), m))
            last = max(i for i in range(m) if knots[i] < knots[i + 1])
            for i in range(m):
                if knots[i] < knots[i + 1]:
                    inside = (x >= knots[i]) & (x < knots[i + 1])
                    if i == last:
                        inside |= x == knots[i + 1]
                    out[:, i] = inside
            return out
        nfun = m - q
        out = np.zeros((len(x), nfun))
        if k == 0:
            low = rec(q - 1, 0)
            for i in range(nfun):
                left = _ratio(x - knots[i], knots[i + q] - knots[i]) * low[:, i]
                right = _ratio(knots[i + q + 1] - x, knots[i + q + 1] - knots[i + 1]) * low[:, i + 1]
                out[:, i] = left + right
        else:
            low = rec(q - 1, k - 1)
            for i in range(nfun):
                out[:, i] = q * (_ratio(low[:, i], knots[i + q] - knots[i])
                                 - _ratio(low[:, i + 1], knots[i + q + 1] - knots[i + 1]))
        return out

    return rec(p, deriv)


def greville(knots, p):
    """Greville abscissae gamma_i = (xi_{i+1} + ... + xi_{i+p}) / p (Sec. 2)."""
    knots = np.asarray(knots, dtype=float)
    n = len(knots) - p - 1
    return np.array([knots[i + 1:i + p + 1].mean() for i in range(n)])


def gauss_rule(nq):
    """Gauss-Legendre nodes and weights on [-1, 1] (library routine)."""
    return np.polynomial.legendre.leggauss(nq)


def breakpoints(knots):
    return np.unique(np.asarray(knots, dtype=float))


class Direction:
    """Quadrature tables of one parametric direction.

    Each knot span e = 0..n_el-1 gets nq Gauss points.  `scale` maps the
    parametric coordinate to the physical one (T for time, 1 in space):
    physical points scale*x, weights scale*w, and the k-th derivative of a
    basis function in physical units is scale**(-k) times the parametric one.

    Attributes
      xq[e, q], wq[e, q]        physical points and weights
      vals[k][e, q, i]          k-th derivative of basis i (full basis, dense)
      local[e]                  indices of the basis functions non-zero on span e
    """

    def __init__(self, n_el, p, nq=None, scale=1.0, knots=None, max_deriv=None):
        self.p = p
        self.knots = open_uniform_knots(n_el, p) if knots is None else np.asarray(knots, float)
        self.br = breakpoints(self.knots)
        self.n_el = len(self.br) - 1
        self.n = len(self.knots) - p - 1
        self.scale = float(scale)
        nq = p + 1 if nq is None else nq
        self.nq = nq
        gx, gw = gauss_rule(nq)
        a, b = self.br[:-1], self.br[1:]
        xp = 0.5 * (a[:, None] + b[:, None]) + 0.5 * (b - a)[:, None] * gx[None, :]
        wp = 0.5 * (b - a)[:, None] * gw[None, :]
        self.xq_par = xp
        self.xq = scale * xp
        self.wq = scale * wp
        kmax = p if max_deriv is None else max_deriv
        flat = xp.reshape(-1)
        self.vals = []
        for k in range(kmax + 1):
            v = bspline_all(self.knots, p, flat, k) * scale ** (-k)
            self.vals.append(v.reshape(self.n_el, nq, self.n))
        nz = np.abs(self.vals[0]).sum(axis=1) > 0
        self.local = [np.nonzero(nz[e])[0] for e in range(self.n_el)]
        self.greville = scale * greville(self.knots, p)
