"""Space-time discretization for the oracle: assembled sparse matrices by a
direct loop over (d+1)-dimensional elements with Gauss quadrature.

Discrete space (Sec. 2): tensor-product B-splines of degree p in each of the d
spatial directions and in time, maximal regularity (or C^0 in time with
time_continuity = "c0", the space of the comparison method of Sec. 4.2), the
first time function b_1 removed to impose the zero initial condition, so
N_t = n_t - 1 and
N_dof = N_s * N_t.  Unknowns are ordered colexicographically: x fastest, then
y, z, and time slowest, i.e. index = i_t * N_s + i_s with
i_s = i_x + n_x (i_y + n_y i_z).

Every matrix here is assembled entry by entry from its integral definition on
the space-time elements (no Kronecker products of assembled 1D matrices): row
index = test function, column index = trial function.

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np
import scipy.sparse as sp

from .bspline import Direction


def open_knots(breaks, p):
    """Open knot vector of maximal regularity on the breakpoints (None: uniform,
    left to Direction): p+1 copies of each end, the interior breakpoints once."""
    if breaks is None:
        return None
    b = np.asarray(breaks, dtype=float)
    return np.concatenate([np.full(p, b[0]), b, np.full(p, b[-1])])


def c0_time_knots(n_el_t, p, breaks=None):
    """Knot vector on [0, 1] of degree p and continuity C^0 (the time space of
    the comparison method of Sec. 4.2): p+1 copies of each end, every interior
    breakpoint p times; uniform breakpoints unless given."""
    b = np.linspace(0.0, 1.0, n_el_t + 1) if breaks is None else np.asarray(breaks, dtype=float)
    inner = np.repeat(b[1:-1], p)
    return np.concatenate([np.full(p + 1, b[0]), inner, np.full(p + 1, b[-1])])


def _spatial_table(dirs, kk):
    """Tensor-product table of the spatial basis on spatial elements.

    Returns S[es, qs, ls] = prod_l vals_l[k_l][e_l, q_l, local_l(e_l)[a_l]] with
    es, qs, ls colexicographic (direction 0 fastest)."""
    tab = None
    for l, dr in enumerate(dirs):
        loc = np.array([dr.local[e] for e in range(dr.n_el)])          # (n_el, p+1)
        v = dr.vals[kk[l]]                                              # (n_el, nq, n)
        t1 = np.take_along_axis(v, loc[:, None, :].repeat(dr.nq, axis=1), axis=2)
        if tab is None:
            tab = t1
        else:
            e0, q0, a0 = tab.shape
            e1, q1, a1 = t1.shape
            tab = np.einsum('eqa,fpb->fepqba', tab, t1).reshape(e1 * e0, q1 * q0, a1 * a0)
    return tab


def _spatial_weights(dirs):
    w = None
    for dr in dirs:
        if w is None:
            w = dr.wq
        else:
            w = np.einsum('eq,fp->fepq', w, dr.wq).reshape(dr.n_el * w.shape[0], dr.nq * w.shape[1])
    return w


def _spatial_points(dirs):
    """Physical coordinates of the spatial Gauss points: list of d arrays (N_el_s, nq_s)."""
    d = len(dirs)
    out = []
    for l in range(d):
        arr = None
        for m, dr in enumerate(dirs):
            c = dr.xq if m == l else np.ones_like(dr.xq)
            if arr is None:
                arr = c
            else:
                arr = np.einsum('eq,fp->fepq', arr, c).reshape(dr.n_el * arr.shape[0], dr.nq * arr.shape[1])
        out.append(arr)
    return out


def _spatial_glob(dirs):
    """Global spatial index of local function ls on spatial element es: (N_el_s, L)."""
    glob = None
    stride = 1
    for dr in dirs:
        loc = np.array([dr.local[e] for e in range(dr.n_el)]) * stride   # (n_el, p+1)
        if glob is None:
            glob = loc
        else:
            glob = (glob[None, :, None, :] + loc[:, None, :, None]).reshape(
                dr.n_el * glob.shape[0], loc.shape[1] * glob.shape[1])
        stride *= dr.n
    return glob


class SpaceTime:
    """Tables and assembly routines for one problem description (see workloads)."""

    def __init__(self, desc, nq=None):
        self.desc = desc
        self.d = desc["d"]
        self.p = desc["p"]
        p = self.p
        self.T = float(desc["T"])
        breaks = desc.get("breaks") or [None] * self.d
        self.sdirs = [Direction(ne, p, nq=nq, scale=1.0, max_deriv=2, knots=open_knots(breaks[l], p))
                      for l, ne in enumerate(desc["n_el"])]
        if desc.get("time_continuity", "max") == "c0":
            tknots = c0_time_knots(desc["n_el_t"], p, desc.get("breaks_t"))
        else:
            tknots = open_knots(desc.get("breaks_t"), p)
        self.tdir = Direction(desc["n_el_t"], p, nq=nq, scale=self.T, max_deriv=p, knots=tknots)
        self.n = [dr.n for dr in self.sdirs]
        self.N_s = int(np.prod(self.n))
        self.n_t = self.tdir.n
        self.N_t = self.n_t - 1
        self.N_dof = self.N_s * self.N_t
        self.N_el_s = int(np.prod([dr.n_el for dr in self.sdirs]))
        self.n_el_t = self.tdir.n_el
        self.nq_t = self.tdir.nq
        self.ws = _spatial_weights(self.sdirs)                 # (N_el_s, nq_s)
        self.nq_s = self.ws.shape[1]
        self.xs = _spatial_points(self.sdirs)                  # d x (N_el_s, nq_s)
        self.sglob = _spatial_glob(self.sdirs)                 # (N_el_s, L_s)
        self._stab = {}
        tloc = np.array([self.tdir.local[e] for e in range(self.n_el_t)])  # full time index
        self.tglob = tloc - 1                                   # X_t index, -1 = removed b_1
        self.ttab = [np.take_along_axis(self.tdir.vals[k], tloc[:, None, :].repeat(self.nq_t, axis=1), axis=2)
                     for k in range(p + 1)]                     # [k][et, qt, at]

    # ---------------------------------------------------------------- tables
    def stab(self, kk):
        kk = tuple(kk)
        if kk not in self._stab:
            self._stab[kk] = _spatial_table(self.sdirs, kk)
        return self._stab[kk]

    def unit(self, l, k):
        kk = [0] * self.d
        kk[l] = k
        return tuple(kk)

    def glob(self, et):
        """Global dof of (at, ls) on space-time element (et, es): (N_el_s, p+1, L_s), -1 = removed."""
        it = self.tglob[et]
        g = it[None, :, None] * self.N_s + self.sglob[:, None, :]
        g[:, it < 0, :] = -1
        return g

    # ---------------------------------------------------------------- fields
    def field(self, vec, kt=0, ks=None):
        """Derivative (kt in time, ks = per-direction orders in space) of the
        spline with coefficient vector `vec` at every Gauss point:
        array (n_el_t, N_el_s, nq_t, nq_s)."""
        ks = (0,) * self.d if ks is None else ks
        S = self.stab(ks)
        out = np.zeros((self.n_el_t, self.N_el_s, self.nq_t, self.nq_s))
        for et in range(self.n_el_t):
            g = self.glob(et)
            c = np.where(g >= 0, vec[np.maximum(g, 0)], 0.0)          # (es, at, ls)
            out[et] = np.einsum('eal,ta,eql->etq', c, self.ttab[kt][et], S)
        return out

    def time_points(self):
        return self.tdir.xq                                          # (n_el_t, nq_t)

    # ---------------------------------------------------------------- assembly
    def assemble(self, terms):
        """Sparse matrix of sum_terms int int coef * (d test) * (d trial).

        Each term is (coef, kt_test, ks_test, kt_trial, ks_trial) with coef an
        array (n_el_t, N_el_s, nq_t, nq_s) of integrand coefficients at the
        Gauss points (quadrature weights are applied here)."""
        rows, cols, vals = [], [], []
        for et in range(self.n_el_t):
            g = self.glob(et).reshape(self.N_el_s, -1)                # (es, at*ls)
            loc = 0.0
            wt = self.tdir.wq[et]
            for coef, kti, ksi, ktj, ksj in terms:
                W = coef[et] * wt[None, :, None] * self.ws[:, None, :]  # (es, qt, qs)
                Ti, Tj = self.ttab[kti][et], self.ttab[ktj][et]
                Si, Sj = self.stab(ksi), self.stab(ksj)
                loc = loc + np.einsum('etq,ta,eql,tb,eqm->ealbm', W, Ti, Si, Tj, Sj, optimize=True)
            nl = g.shape[1]
            loc = loc.reshape(self.N_el_s, nl, nl)
            r = np.repeat(g[:, :, None], nl, axis=2)
            c = np.repeat(g[:, None, :], nl, axis=1)
            keep = (r >= 0) & (c >= 0)
            rows.append(r[keep]); cols.append(c[keep]); vals.append(loc[keep])
        rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.N_dof, self.N_dof))

    def load(self, coef, kt=0, ks=None):
        """Vector of int int coef * (d test): coef at the Gauss points as in `assemble`."""
        ks = (0,) * self.d if ks is None else ks
        out = np.zeros(self.N_dof)
        S = self.stab(ks)
        for et in range(self.n_el_t):
            g = self.glob(et).reshape(self.N_el_s, -1)
            W = coef[et] * self.tdir.wq[et][None, :, None] * self.ws[:, None, :]
            loc = np.einsum('etq,ta,eql->eal', W, self.ttab[kt][et], S).reshape(self.N_el_s, -1)
            keep = g >= 0
            np.add.at(out, g[keep], loc[keep])
        return out

    def const(self, value):
        return np.full((self.n_el_t, self.N_el_s, self.nq_t, self.nq_s), float(value))

    # ------------------------------------------------------- named operators
    def linear_terms(self, C_m, D):
        """Terms of int int C_m d_t u v + grad u . D grad v (the linear part of A, Sec. 3)."""
        one = self.const(1.0)
        z = (0,) * self.d
        terms = [(C_m * one, 0, z, 1, z)]
        for l in range(self.d):
            terms.append((D[l] * one, 0, self.unit(l, 1), 0, self.unit(l, 1)))
        return terms

    def mass_terms(self, coef):
        z = (0,) * self.d
        return [(coef, 0, z, 0, z)]

    def su_terms(self, C_m, tau_q, theta_q):
        """Terms of C_m sum_k int int tau_k theta d_t^k u d_t^k v (Sec. 3, SU term).

        tau_q[k-1] is tau_k at the time Gauss points (n_el_t, nq_t); theta_q is
        theta at all Gauss points."""
        z = (0,) * self.d
        out = []
        for k in range(1, self.p + 1):
            coef = C_m * tau_q[k - 1][:, None, :, None] * theta_q
            out.append((coef, k, z, k, z))
        return out

    # ------------------------------------------------------------ 1D helpers
    def matrices_1d(self):
        """1D matrices by quadrature on each direction (used by the pins and the
        Kronecker identity tests): M_l, K_l per spatial direction, M_t, W_t on X_t."""
        out = {}
        for l, dr in enumerate(self.sdirs):
            B0 = dr.vals[0].reshape(-1, dr.n)
            B1 = dr.vals[1].reshape(-1, dr.n)
            w = dr.wq.reshape(-1)
            out[f"M{l}"] = (B0 * w[:, None]).T @ B0
            out[f"K{l}"] = (B1 * w[:, None]).T @ B1
        dr = self.tdir
        B0 = dr.vals[0].reshape(-1, dr.n)[:, 1:]
        B1 = dr.vals[1].reshape(-1, dr.n)[:, 1:]
        w = dr.wq.reshape(-1)
        out["Mt"] = (B0 * w[:, None]).T @ B0
        out["Wt"] = (B0 * w[:, None]).T @ B1     # [i, j] = int b_j' b_i
        return out
