"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds problem descriptions (plain dictionaries of numbers) and seeded
random draws only.  It contains none of the method's arithmetic: no basis
functions, no quadrature, no operators.  Both the CPU oracle and the CUDA path
read the same dictionaries, so a parity test compares the two on identical
inputs.

Problem description keys (all plain Python numbers / lists / strings):

  d, p            spatial dimension (1..3) and spline degree p_s = p_t = p
  n_el, n_el_t    elements per spatial direction (list of d ints), time elements
  T, C_m, D       final time, membrane capacitance, diagonal conductivity (list of d)
  a, b, c1, c2, d_e   dimensionless Rogers-McCulloch constants (monodomain eq. 3.1)
  source          {"kind": "stim", "boxes": [...]} | {"kind": "heat_mms"} |
                  {"kind": "e1_mms"} | {"kind": "zero"}
                  a box is {"lo": [d], "hi": [d], "t0": t0, "t1": t1, "amp": A};
                  it contributes A on the closed box [lo, hi] for t0 <= t < t1
  stabilization   "galerkin" | "su"
  suppext         "literal" | "symmetric"   (support-extension reading, see DESIGN)
  eps_theta       relative Frobenius tolerance of the low-rank theta (Sec. 3.1)
  eps_reaction    < 0: exact reaction coefficient at the Gauss points; >= 0: its
                  Greville-grid values in low rank at that tolerance
  nonlinear       "picard" (fixed point with relaxation) | "newton"
  alpha, delta, max_fp   relaxation, stopping tolerance, iteration cap
  fix_w_zero      True: recovery variable held at zero (smooth 1D test, Sec. 4.1)
  precision       "fp64" | "mixed"
  gmres_m, rtol, max_it  Krylov restart length, relative residual target, cap
  breaks, breaks_t  None (uniform) or the n_el + 1 increasing breakpoints from 0 to
                  1 of each spatial direction (a list of d lists or None) and of
                  time (parametric, scaled by T)
  operator_form   "auto" | "bands" | "lean"   (how the device stores the
                  reaction + SU part of the operator; results are the same)
  inner_op        "auto" | "fp32" | "df"   (arithmetic of the operator inside
                  the mixed mode's FP32 Krylov solve)
  precond_arith   "auto" | "tf32" | "fp32" | "fp64"   (the preconditioner inside
                  the mixed mode's FP32 Krylov solve)
"""

import copy
import numpy as np

# Dimensionless Rogers-McCulloch constants of the paper's numerical section (Sec. 4).
PAPER_RM = dict(a=0.13, b=0.013, c1=0.26, c2=0.1, d_e=1.0)

# The dimensional set G=1.5, v_th=13, v_p=100, eta1=4.4, eta2=0.012, eta3=1 and
# I_app=100 rewritten for u = v / v_p:  a = v_th/v_p, c1 = G v_p / v_th,
# c2 = eta1, b = eta2, d_e = eta3, stimulus amplitude I_app / v_p.
DIMENSIONAL_RM = dict(a=0.13, b=0.012, c1=1.5 * 100.0 / 13.0, c2=4.4, d_e=1.0)
DIMENSIONAL_STIM_AMP = 100.0 / 100.0


def base_desc(**over):
    """Defaults shared by every workload; keyword arguments override."""
    desc = dict(
        d=2, p=2, n_el=[4, 4], n_el_t=8, T=1.0, C_m=1.0, D=[1e-3, 1e-3],
        source=dict(kind="zero"),
        stabilization="su", suppext="literal", eps_theta=0.1, eps_reaction=-1.0,
        nonlinear="picard", alpha=0.5, delta=1e-4, max_fp=60, fix_w_zero=False,
        precision="fp64", gmres_m=100, rtol=1e-8, max_it=2000, operator_form="auto", inner_op="auto", precond_arith="auto",
    )
    desc.update(PAPER_RM)
    for k, v in over.items():
        desc[k] = v
    return copy.deepcopy(desc)


def stim_box(lo, hi, t0, t1, amp):
    return dict(lo=list(map(float, lo)), hi=list(map(float, hi)),
                t0=float(t0), t1=float(t1), amp=float(amp))


def corner_box(d, seed, side_range=(0.05, 0.15)):
    """Square (cube) stimulus of random side at a random corner of the unit domain.

    numpy PCG64 with the given seed draws the side ~ U[side_range] and the corner
    index uniformly from the 2**d corners."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = float(rng.uniform(*side_range))
    corner = int(rng.integers(0, 2 ** d))
    lo, hi = [], []
    for l in range(d):
        if (corner >> l) & 1:
            lo.append(1.0 - side); hi.append(1.0)
        else:
            lo.append(0.0); hi.append(side)
    return lo, hi


def config(name, scale=None):
    """Problem description of a named workload.

    c1_newton_2d   2D, p=2, 16x16 x 32 elements, T=50, D=1e-3, RM (dimensional
                   set), stimulus [0,0.1]^2 for t<1, Newton, FP64.
    c2_aniso_2d    2D, p=3, 128x128 x 256 elements, T=50, D=diag(1e-3,2.5e-4),
                   seeded corner stimulus (seed 2), Picard, FP64 (and mixed).
    c3_cube_3d     3D, p=2, 64^3 x 128 elements, D=1e-3 I, planar stimulus x<0.05,
                   mixed precision.
    c5_cube_3d     3D, p=3, 96^3 x 192 elements (188,238,006 unknowns),
                   D=diag(1e-3,5e-4,2.5e-4), two staggered stimuli ([0,0.1]^3 for
                   t<1 and [0.9,1]^3 for 10<=t<11), mixed precision.
    heat_mms_2d    linear heat manufactured solution cos(pi x)cos(pi y)sin(t), T=1.
    e1_mms_1d      smooth 1D test of Sec. 4.1 (Omega=(0,1), T=1, D=1e-4).

    `scale` (optional) replaces the element counts with smaller ones of the same
    shape: a dict {"n_el": [...], "n_el_t": int}.
    """
    if name == "c1_newton_2d":
        desc = base_desc(d=2, p=2, n_el=[16, 16], n_el_t=32, T=50.0, C_m=1.0,
                         D=[1e-3, 1e-3], nonlinear="newton", precision="fp64",
                         source=dict(kind="stim", boxes=[stim_box([0, 0], [0.1, 0.1], 0.0, 1.0,
                                                                  DIMENSIONAL_STIM_AMP)]))
        desc.update(DIMENSIONAL_RM)
    elif name == "c2_aniso_2d":
        lo, hi = corner_box(2, seed=2)
        desc = base_desc(d=2, p=3, n_el=[128, 128], n_el_t=256, T=50.0, C_m=1.0,
                         D=[1e-3, 2.5e-4], nonlinear="picard", precision="fp64",
                         source=dict(kind="stim", boxes=[stim_box(lo, hi, 0.0, 1.0,
                                                                  DIMENSIONAL_STIM_AMP)]))
        desc.update(DIMENSIONAL_RM)
    elif name == "c3_cube_3d":
        desc = base_desc(d=3, p=2, n_el=[64, 64, 64], n_el_t=128, T=50.0, C_m=1.0,
                         D=[1e-3, 1e-3, 1e-3], nonlinear="picard", precision="mixed",
                         source=dict(kind="stim", boxes=[stim_box([0, 0, 0], [0.05, 1, 1], 0.0, 1.0,
                                                                  DIMENSIONAL_STIM_AMP)]))
        desc.update(DIMENSIONAL_RM)
    elif name == "c5_cube_3d":
        desc = base_desc(d=3, p=3, n_el=[96, 96, 96], n_el_t=192, T=50.0, C_m=1.0,
                         D=[1e-3, 5e-4, 2.5e-4], nonlinear="picard", precision="mixed",
                         source=dict(kind="stim", boxes=[
                             stim_box([0, 0, 0], [0.1, 0.1, 0.1], 0.0, 1.0, DIMENSIONAL_STIM_AMP),
                             stim_box([0.9, 0.9, 0.9], [1, 1, 1], 10.0, 11.0, DIMENSIONAL_STIM_AMP)]))
        desc.update(DIMENSIONAL_RM)
    elif name == "heat_mms_2d":
        desc = base_desc(d=2, p=2, n_el=[8, 8], n_el_t=8, T=1.0, C_m=1.0, D=[1e-3, 2.5e-4],
                         a=0.13, b=0.0, c1=0.0, c2=0.0, d_e=1.0, stabilization="galerkin",
                         source=dict(kind="heat_mms"), fix_w_zero=True)
    elif name == "e1_mms_1d":
        desc = base_desc(d=1, p=2, n_el=[8], n_el_t=8, T=1.0, C_m=1.0, D=[1e-4],
                         stabilization="su", source=dict(kind="e1_mms"), fix_w_zero=True,
                         alpha=1.0)
    else:
        raise KeyError(name)
    if scale is not None:
        desc["n_el"] = list(scale["n_el"])
        desc["n_el_t"] = int(scale["n_el_t"])
    return desc


def n_dofs(desc):
    """Number of unknowns N_s * N_t (counting only; n_l = n_el + p, N_t = n_t - 1)."""
    p = desc["p"]
    n_s = 1
    for ne in desc["n_el"]:
        n_s *= ne + p
    return n_s * (desc["n_el_t"] + p - 1)


def wave_fields(desc, seed=7, speed=0.03, width=0.05):
    """Smooth synthetic linearization inputs (u, w), coefficient vectors in the
    layout [t][z][y][x]: an excitation front spreading from a seeded point.
    Closed-form values on a uniform index grid (x_i = i / (n_l - 1), t_j =
    (j + 1) T / N_t) are used directly as coefficients; nothing here evaluates a
    basis function.  u = (1 + tanh((speed t - r) / width)) / 2 with r the
    distance to the point, w = 0.3 times the same front five time units later."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d, p = desc["d"], desc["p"]
    n = [ne + p for ne in desc["n_el"]]
    n_t = desc["n_el_t"] + p - 1
    c = rng.uniform(0.0, 0.3, size=d)
    axes = [np.linspace(0.0, 1.0, n[l]) for l in range(d)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")              # (z, y, x) order
    r2 = sum((grids[d - 1 - l] - c[l]) ** 2 for l in range(d))
    r = np.sqrt(r2)[None]
    t = (np.arange(n_t) + 1.0) * desc["T"] / n_t
    t = t.reshape((n_t,) + (1,) * d)
    u = 0.5 * (1.0 + np.tanh((speed * t - r) / width))
    w = 0.3 * 0.5 * (1.0 + np.tanh((speed * (t - 5.0) - r) / width))
    return u.reshape(-1), w.reshape(-1)


def clustered_breaks(n_el, centers, p, T=1.0, spread=0.125):
    """Breakpoints on [0, 1] (parametric; physical times are T times these):
    p + 1 of them clustered at spacing spread / n_el around each physical time
    in `centers`, the rest spread almost uniformly over the gaps between the
    clusters and the ends, in proportion to the gap lengths; cluster points
    outside (0, 1) are dropped (the time knots
    clustered where the source switches on and off, same number of elements,
    Sec. 4.2).  Plain arithmetic on a list of numbers."""
    h = 1.0 / n_el
    fixed = [0.0, 1.0]
    for c in centers:
        x = c / T
        fixed += [x + (k - p / 2.0) * spread * h for k in range(p + 1)]
    # cluster points must lie strictly inside (0, 1), once each
    fixed = sorted(set(v for v in fixed if 0.0 < v < 1.0) | {0.0, 1.0})
    left = n_el + 1 - len(fixed)
    gaps = np.diff(fixed)
    share = gaps / gaps.sum() * left
    count = np.floor(share).astype(int)
    for i in np.argsort(-(share - count))[:left - count.sum()]:
        count[i] += 1
    out = list(fixed)
    for i, m in enumerate(count):
        a, b = fixed[i], fixed[i + 1]
        out += [a + (b - a) * (k + 1) / (m + 1) for k in range(m)]
    return sorted(float(v) for v in out)


def graded_breaks(n_el, power=1.3):
    """Breakpoints (i / n_el)^power on [0, 1]: elements growing smoothly from
    0 to 1 (plain arithmetic on a list of numbers)."""
    return [float((i / n_el) ** power) for i in range(n_el + 1)]


def random_vector(n, seed, lo=-1.0, hi=1.0):
    """x ~ U(lo, hi) from numpy PCG64(seed), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=n)


def serving_requests(n_req=256, seed=4, rate=None):
    """The serving stream: seeded 2D requests with ragged shapes.

    p in {2,3}; n_el_x, n_el_y ~ U{32..256}; n_el_t ~ U{64..512};
    D = d I with log10 d ~ U[log10 2e-4, log10 2e-3]; a 0.1-square stimulus
    with lower-left corner uniform in [0, 0.9]^2 for t < 1; Poisson arrivals
    (exponential gaps of mean 1/rate seconds) when `rate` is given."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    t = 0.0
    for i in range(n_req):
        p = int(rng.integers(2, 4))
        nx = int(rng.integers(32, 257))
        ny = int(rng.integers(32, 257))
        nt = int(rng.integers(64, 513))
        dval = float(10 ** rng.uniform(np.log10(2e-4), np.log10(2e-3)))
        cx, cy = (float(v) for v in rng.uniform(0.0, 0.9, size=2))
        gap = float(rng.exponential(1.0 / rate)) if rate else 0.0
        t += gap
        desc = base_desc(d=2, p=p, n_el=[nx, ny], n_el_t=nt, T=50.0, D=[dval, dval],
                         nonlinear="picard", precision="mixed",
                         source=dict(kind="stim", boxes=[stim_box([cx, cy], [cx + 0.1, cy + 0.1],
                                                                  0.0, 1.0, DIMENSIONAL_STIM_AMP)]))
        desc.update(DIMENSIONAL_RM)
        reqs.append(dict(id=i, arrival=t, desc=desc))
    return reqs
