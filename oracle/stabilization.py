"""Spline Upwind ingredients for the oracle (Sec. 3 of the paper).

* tau_k, k = 1..p: splines of degree p-k on the time mesh fixed by the
  conditions of Eq. (tau): the strict upper band (offsets 1..p) of
  W_t + sum_k int tau_k b^(k) b^(k) vanishes.
* Theta-hat (Eq. theta_ce_u): the L-infinity norm of the residual over the
  support extension (Eq. suppext) of each basis function, divided by
  C_m (||u||_inf / T + ||d_t u||_inf), capped at 1.
* The low-rank approximation U R V^T of Theta-hat at relative Frobenius
  tolerance eps (Eq. tol), and theta at the Gauss points as the
  (d+1)-linear interpolant on the Greville grid (Sec. 3.1).
* The values of a spline at the Greville grid, from which the low-rank
  reaction coefficient of reading A7 is formed the same way.

Readings where the paper is silent: tau is the
minimum-norm solution in the scaled coefficients c_{k,m} / h_{k,m}^(2k-1), with
h_{k,m} the largest element in the support of the m-th B-spline of tau_k (h_t
on a uniform mesh); the support
extension is taken literally with the underlying b-hat index in time; the
L-infinity norms are maxima over Gauss points; Theta = 1 when the denominator
vanishes with a non-zero residual and 0 when both vanish; the low-rank factors
are the truncated SVD with the smallest rank meeting Eq. (tol).

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np

from .bspline import bspline_all
from .bspline import greville as greville_param


def tau_solve(st):
    """Coefficients of tau_k and their values at the time Gauss points.

    Unknowns: B-spline coefficients c_{k,m} of tau_k in S^{p-k} (maximal
    regularity on the time breakpoints).  Conditions, for X_t indices
    i = 0..N_t-2 and l = 1..min(p, N_t-1-i), j = i+l:
        int b_j' b_i dt + sum_k int tau_k b_j^(k) b_i^(k) dt = 0.
    Returns (coeffs, tau_q) with coeffs[k-1] the coefficient vector of tau_k and
    tau_q[k-1] the values (n_el_t, nq_t)."""
    p = st.p
    td = st.tdir
    n_el = td.n_el
    xpar = td.xq_par.reshape(-1)
    w = td.wq.reshape(-1)
    B = [td.vals[k].reshape(-1, td.n)[:, 1:] for k in range(p + 1)]     # X_t basis, physical derivs
    beta = []
    for k in range(1, p + 1):
        # degree p-k on the breakpoints of the time mesh
        kn = np.concatenate([np.full(p - k, td.br[0]), td.br, np.full(p - k, td.br[-1])])
        beta.append(bspline_all(kn, p - k, xpar, 0))                      # (nq_total, n_k)
    sizes = [bb.shape[1] for bb in beta]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rows, rhs = [], []
    N_t = st.N_t
    for i in range(N_t - 1):
        for l in range(1, min(p, N_t - 1 - i) + 1):
            j = i + l
            row = np.zeros(offs[-1])
            for k in range(1, p + 1):
                row[offs[k - 1]:offs[k]] = (w * B[k][:, j] * B[k][:, i]) @ beta[k - 1]
            rows.append(row)
            rhs.append(-np.sum(w * B[1][:, j] * B[0][:, i]))
    C = np.array(rows)
    rhs = np.array(rhs)
    # unknowns scaled by h^(2k-1), h the largest element in the support of the
    # coefficient's B-spline (h_t itself on a uniform mesh)
    hel = st.T * np.diff(td.br)
    scale = []
    for k in range(1, p + 1):
        q = p - k
        for m in range(sizes[k - 1]):
            scale.append(hel[max(0, m - q):min(n_el - 1, m) + 1].max() ** (2 * k - 1))
    scale = np.array(scale)
    y, *_ = np.linalg.lstsq(C * scale[None, :], rhs, rcond=None)
    c = y * scale
    coeffs = [c[offs[k - 1]:offs[k]] for k in range(1, p + 1)]
    tau_q = [(beta[k - 1] @ coeffs[k - 1]).reshape(n_el, td.nq) for k in range(1, p + 1)]
    return coeffs, tau_q


def support_window(i_full, p, n_el, mode="literal"):
    """Knot-span indices (0-based) inside the support extension of the basis
    function with 0-based full index i_full, clamped to the mesh.

    Eq. (suppext) gives (xi_{i-p}, xi_{i+p+1}) for the 1-based basis index i,
    i.e. spans i-2p .. i (1-based spans [xi_{p+e}, xi_{p+e+1}]), which in
    0-based indices is i_full-2p .. i_full.  mode="symmetric" takes
    (xi_{i-p}, xi_{i+2p+1}) instead: spans i_full-2p .. i_full+p."""
    lo = i_full - 2 * p
    hi = i_full if mode == "literal" else i_full + p
    return max(lo, 0), min(hi, n_el - 1)


def theta_hat(st, R_q, u_q, dtu_q, C_m, mode="literal"):
    """Theta-hat of Eq. (theta_ce_u) as an (N_t, N_s) matrix.

    R_q, u_q, dtu_q: residual, u and d_t u at all Gauss points, arrays
    (n_el_t, N_el_s, nq_t, nq_s).  The numerator of basis (i_s, i_t) is the
    largest |R| over the Gauss points of the space-time elements inside its
    support extension; the denominator C_m (max|u| / T + max|d_t u|) is taken
    over all Gauss points."""
    p, d = st.p, st.d
    elem = np.abs(R_q).max(axis=(2, 3))                                  # (n_el_t, N_el_s)
    ne = [dr.n_el for dr in st.sdirs]
    elem = elem.reshape([st.n_el_t] + ne[::-1])                            # (t, z, y, x)
    den = C_m * (np.abs(u_q).max() / st.T + np.abs(dtu_q).max())
    n_rev = st.n[::-1]
    num = np.zeros([st.N_t] + n_rev)
    for it in range(st.N_t):
        t0, t1 = support_window(it + 1, p, st.n_el_t, mode)
        for idx in np.ndindex(*n_rev):
            sl = [slice(t0, t1 + 1)]
            for pos, i in enumerate(idx):
                l = d - 1 - pos
                a, b = support_window(i, p, ne[l], mode)
                sl.append(slice(a, b + 1))
            num[(it,) + idx] = elem[tuple(sl)].max()
    num = num.reshape(st.N_t, st.N_s)
    if den > 0:
        th = np.minimum(num / den, 1.0)
    else:
        th = np.where(num > 0, 1.0, 0.0)
    return th, dict(elem_max=elem.reshape(st.n_el_t, -1), den=den)


def low_rank(theta, eps):
    """Truncated SVD of Theta-hat with the smallest R meeting Eq. (tol):
    ||Theta - U diag(s) V^T||_F <= eps ||Theta||_F.  Returns (U, s, V) with
    U (N_t, R), s (R,), V (N_s, R); R = 0 for Theta = 0."""
    U, s, Vt = np.linalg.svd(theta, full_matrices=False)
    fro = np.sqrt(np.sum(s ** 2))
    if fro == 0.0:
        return U[:, :0], s[:0], Vt[:0].T
    tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))  # tail[r] = ||s[r:]||
    R = next(r for r in range(1, len(s) + 1) if tail[r] <= eps * fro)
    return U[:, :R], s[:R], Vt[:R].T


def greville_values(st, vec):
    """Values of the space-time spline with coefficient vector `vec` at the
    Greville grid (time: the Greville points of b_2 .. b_{n_t}, the functions of
    X_t; space: all Greville points), as an (N_t, N_s) matrix: the
    tensor-product spline evaluated with the 1D B-splines at those points."""
    tdir = st.tdir
    Gt = bspline_all(tdir.knots, st.p, greville_param(tdir.knots, st.p)[1:], 0)[:, 1:]   # (N_t, N_t)
    X = vec.reshape([st.N_t] + st.n[::-1])                                             # (t, z, y, x)
    X = np.tensordot(Gt, X, axes=(1, 0))
    for pos in range(st.d):
        l = st.d - 1 - pos
        dr = st.sdirs[l]
        G = bspline_all(dr.knots, st.p, greville_param(dr.knots, st.p), 0)             # (n_l, n_l)
        X = np.moveaxis(np.tensordot(G, X, axes=(1, 1 + pos)), 0, 1 + pos)
    return X.reshape(st.N_t, st.N_s)


def hat_weights(grid, x):
    """Linear interpolation on the sorted grid: left index and weight of the
    right neighbour; constant outside [grid[0], grid[-1]]."""
    idx = np.clip(np.searchsorted(grid, x, side="right") - 1, 0, len(grid) - 2)
    lam = (x - grid[idx]) / (grid[idx + 1] - grid[idx])
    return idx, np.clip(lam, 0.0, 1.0)


def interpolate_at_gauss(st, theta_mat):
    """(d+1)-linear interpolant of an (N_t, N_s) table given at the Greville
    grid (time: Greville points of b_2..b_{n_t}; space: all Greville points),
    evaluated at every Gauss point: array (n_el_t, N_el_s, nq_t, nq_s)."""
    d = st.d
    grid_t = st.tdir.greville[1:]
    tab = theta_mat.reshape([st.N_t] + st.n[::-1])                        # (t, z, y, x)
    it, lt = hat_weights(grid_t, st.tdir.xq)                              # (n_el_t, nq_t)
    sp_idx, sp_lam = [], []
    for l in range(d):
        i, lam = hat_weights(st.sdirs[l].greville, st.xs[l])              # (N_el_s, nq_s)
        sp_idx.append(i); sp_lam.append(lam)
    out = np.zeros((st.n_el_t, st.N_el_s, st.nq_t, st.nq_s))
    for corner in range(2 ** (d + 1)):
        ct = corner & 1
        wt = (lt if ct else 1.0 - lt)[:, None, :, None]
        ti = (it + ct)[:, None, :, None]
        wgt = wt
        index = [np.broadcast_to(ti, out.shape)]
        for l in range(d):
            cl = (corner >> (l + 1)) & 1
            wl = (sp_lam[l] if cl else 1.0 - sp_lam[l])[None, :, None, :]
            wgt = wgt * wl
            index.append(None)
        for l in range(d - 1, -1, -1):
            cl = (corner >> (l + 1)) & 1
            index[d - l] = np.broadcast_to((sp_idx[l] + cl)[None, :, None, :], out.shape)
        out += wgt * tab[tuple(index)]
    return out
