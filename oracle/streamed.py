"""Theta-hat and the low-rank SU rows of problems too large to assemble, for
the oracle.

Theta-hat (Eq. theta_ce_u) needs the residual R = C_m d_t u - div(D grad u)
+ I_ion(u, w) - f at every Gauss point.  Here R is evaluated one time element
at a time (the same tables and Gauss rule as `SpaceTime.field`, restricted to
that element), and only its maximum over each space-time element is kept, with
the global maxima of |u|, |d_t u| and |R|.  The numerator of Theta-hat is the
maximum of those element maxima over the support extension of each basis
function (Eq. suppext); a box maximum is taken one axis after the other, which
gives the same value as the maximum over the box.

The SU term of Eq. (tildeS) with the low-rank theta is given as operator terms
for `rows.apply_rows`: theta at the Gauss points of the support elements is
sum_r s_r theta_{t,r}(t) theta_{s,r}(x), the product of the linear
interpolant of U[:, r] in time and the d-linear interpolant of V[:, r] in
space (Sec. 3.1), which is the (d+1)-linear interpolant of U diag(s) V^T.

Both are checked against the assembled oracle on small meshes
(tests/test_oracle_streamed.py).

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np

from . import model
from .stabilization import hat_weights, support_window


def _coeffs(st, vec, et):
    g = st.glob(et)                                               # (N_el_s, p+1, L_s)
    return np.where(g >= 0, vec[np.maximum(g, 0)], 0.0)


def _at_gauss(st, c, et, kt, ks):
    """Derivative (kt, ks) at the Gauss points of time element et: (N_el_s, nq_t, nq_s)."""
    return np.einsum('eal,ta,eql->etq', c, st.ttab[kt][et], st.stab(ks), optimize=True)


def element_maxima(st, desc, u, w):
    """max |R| over the Gauss points of every space-time element, (n_el_t, N_el_s),
    and the maxima of |u|, |d_t u| and |R| over all Gauss points."""
    d, C_m, D = st.d, desc["C_m"], desc["D"]
    z = (0,) * d
    elem = np.zeros((st.n_el_t, st.N_el_s))
    umax = utmax = rmax = 0.0
    xs = [x[:, None, :] for x in st.xs]                           # (N_el_s, 1, nq_s)
    for et in range(st.n_el_t):
        cu, cw = _coeffs(st, u, et), _coeffs(st, w, et)
        uq = _at_gauss(st, cu, et, 0, z)
        utq = _at_gauss(st, cu, et, 1, z)
        lap = sum(D[l] * _at_gauss(st, cu, et, 0, st.unit(l, 2)) for l in range(d))
        wq = _at_gauss(st, cw, et, 0, z)
        f = model.source(desc, xs, st.tdir.xq[et][None, :, None])
        R = C_m * utq - lap + model.ionic_current(desc, uq, wq) - f
        aR = np.abs(R)
        elem[et] = aR.max(axis=(1, 2))
        umax = max(umax, np.abs(uq).max())
        utmax = max(utmax, np.abs(utq).max())
        rmax = max(rmax, aR.max())
    return elem, dict(u_max=umax, ut_max=utmax, r_max=rmax)


def _window_max(a, axis, n_out, p, shift, mode):
    """out[.., i, ..] = max of `a` over the spans of the support extension of
    basis i + shift (0-based full index) along `axis`."""
    n_el = a.shape[axis]
    shape = list(a.shape)
    shape[axis] = n_out
    out = np.empty(shape)
    for i in range(n_out):
        lo, hi = support_window(i + shift, p, n_el, mode)
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(lo, hi + 1)
        dst = [slice(None)] * a.ndim
        dst[axis] = i
        out[tuple(dst)] = a[tuple(sl)].max(axis=axis)
    return out


def theta_hat(st, desc, u, w, mode="literal"):
    """Theta-hat of Eq. (theta_ce_u) as an (N_t, N_s) matrix, with the
    denominator C_m (max|u| / T + max|d_t u|) and the maxima."""
    p, d = st.p, st.d
    elem, info = element_maxima(st, desc, u, w)
    ne = [dr.n_el for dr in st.sdirs]
    a = elem.reshape([st.n_el_t] + ne[::-1])                       # (t, z, y, x)
    a = _window_max(a, 0, st.N_t, p, 1, mode)                      # X_t index i is basis i + 1
    for pos in range(d):
        l = d - 1 - pos
        a = _window_max(a, 1 + pos, st.n[l], p, 0, mode)
    num = a.reshape(st.N_t, st.N_s)
    den = desc["C_m"] * (info["u_max"] / st.T + info["ut_max"])
    if den > 0:
        th = np.minimum(num / den, 1.0)
    else:
        th = np.where(num > 0, 1.0, 0.0)
    info["den"] = den
    return th, info


def theta_lowrank_at(st, U, s, V):
    """theta(x, t) = sum_r s_r theta_{t,r}(t) theta_{s,r}(x) at the Gauss points of
    (et, es): a function (et, es) -> (len(es), nq_t, nq_s)."""
    grid_t = st.tdir.greville[1:]
    Vt = V.reshape(st.n[::-1] + [V.shape[1]])                      # (z, y, x, R)

    def theta(et, es):
        es = np.asarray(es)
        it, lt = hat_weights(grid_t, st.tdir.xq[et])               # (nq_t,)
        Tt = U[it] * (1.0 - lt)[:, None] + U[it + 1] * lt[:, None]  # (nq_t, R)
        hats = [hat_weights(st.sdirs[l].greville, st.xs[l][es]) for l in range(st.d)]   # (E, nq_s) each
        Sx = np.zeros((len(es), st.nq_s, V.shape[1]))
        for corner in range(2 ** st.d):
            wgt = np.ones((len(es), st.nq_s))
            idx = []
            for l in range(st.d - 1, -1, -1):
                c = (corner >> l) & 1
                i_l, lam = hats[l]
                wgt = wgt * (lam if c else 1.0 - lam)
                idx.append(i_l + c)
            Sx += wgt[:, :, None] * Vt[tuple(idx)]
        return np.einsum('tr,r,eqr->etq', Tt, s, Sx)

    return theta


def su_terms(st, desc, tau_q, U, s, V):
    """Terms of C_m sum_l int int tau_l theta d_t^l u d_t^l v with the low-rank
    theta (Eq. tildeS), for rows.apply_rows."""
    theta = theta_lowrank_at(st, U, s, V)
    z = (0,) * st.d
    out = []
    for l in range(1, st.p + 1):
        def coef(et, es, l=l):
            return desc["C_m"] * tau_q[l - 1][et][None, :, None] * theta(et, es)
        out.append((coef, l, z, l, z))
    return out
