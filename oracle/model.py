"""Monodomain + Rogers-McCulloch model terms for the oracle (Sec. 3, eq. 3.1).

    C_m d_t u - div(D grad u) + c1 u (u - a)(u - 1) + c2 u w = f
    d_t w - b (u - d_e w) = 0,   Neumann on the boundary, u = w = 0 at t = 0.

The fixed-point linearization (Eq. reaction) uses
    C_r(u, w) = c1 (u - a)(u - 1) + c2 w,
and the Newton variant differentiates the ionic current in u:
    C_J(u, w) = c1 (3 u^2 - 2 (1 + a) u + a) + c2 w.

Sources (f at arbitrary points): stimulus boxes (closed in space, [t0, t1) in
time), the smooth 1D solution of Sec. 4.1, and a Neumann-compatible linear heat
manufactured solution.

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np


def ionic_current(desc, u, w):
    return desc["c1"] * u * (u - desc["a"]) * (u - 1.0) + desc["c2"] * u * w


def reaction_coef(desc, u, w):
    return desc["c1"] * (u - desc["a"]) * (u - 1.0) + desc["c2"] * w


def jacobian_coef(desc, u, w):
    a = desc["a"]
    return desc["c1"] * (3.0 * u * u - 2.0 * (1.0 + a) * u + a) + desc["c2"] * w


def e1_exact(x, t):
    """u_ex = 10 sin(pi x) sin(pi t) (1 - e^-x)(1 - e^(x-1))(1 - e^(t-1)) (Sec. 4.1)
    with d_t u and d_xx u.  Returns (u, u_t, u_xx)."""
    pi = np.pi
    s, s1, s2 = np.sin(pi * x), pi * np.cos(pi * x), -pi * pi * np.sin(pi * x)
    A, A1, A2 = 1 - np.exp(-x), np.exp(-x), -np.exp(-x)
    B, B1, B2 = 1 - np.exp(x - 1), -np.exp(x - 1), -np.exp(x - 1)
    g = s * A * B
    g2 = s2 * A * B + s * A2 * B + s * A * B2 + 2 * (s1 * A1 * B + s1 * A * B1 + s * A1 * B1)
    h = np.sin(pi * t) * (1 - np.exp(t - 1))
    h1 = pi * np.cos(pi * t) * (1 - np.exp(t - 1)) - np.sin(pi * t) * np.exp(t - 1)
    return 10 * g * h, 10 * g * h1, 10 * g2 * h


def heat_exact(xs, t):
    """u = prod_l cos(pi x_l) sin(t): returns (u, u_t, [u_{x_l x_l}])."""
    c = np.ones_like(t)
    for x in xs:
        c = c * np.cos(np.pi * x)
    u = c * np.sin(t)
    return u, c * np.cos(t), [-np.pi ** 2 * u for _ in xs]


def exact_solution(desc, xs, t):
    kind = desc["source"]["kind"]
    if kind == "e1_mms":
        return e1_exact(xs[0], t)[0]
    if kind == "heat_mms":
        return heat_exact(xs, t)[0]
    raise ValueError(f"no exact solution for source {kind}")


def source(desc, xs, t):
    """f at points: xs list of d coordinate arrays, t times (broadcastable)."""
    src = desc["source"]
    kind = src["kind"]
    C_m, D = desc["C_m"], desc["D"]
    if kind == "zero":
        return np.zeros(np.broadcast(t, *xs).shape)
    if kind == "stim":
        out = np.zeros(np.broadcast(t, *xs).shape)
        for bx in src["boxes"]:
            ind = ((t >= bx["t0"]) & (t < bx["t1"])).astype(float)
            for l, x in enumerate(xs):
                ind = ind * ((x >= bx["lo"][l]) & (x <= bx["hi"][l]))
            out = out + bx["amp"] * ind
        return out
    if kind == "e1_mms":
        u, ut, uxx = e1_exact(xs[0], t)
        return C_m * ut - D[0] * uxx + ionic_current(desc, u, 0.0)
    if kind == "heat_mms":
        u, ut, uxx = heat_exact(xs, t)
        lap = sum(D[l] * uxx[l] for l in range(len(xs)))
        return C_m * ut - lap + ionic_current(desc, u, 0.0)
    raise ValueError(kind)
