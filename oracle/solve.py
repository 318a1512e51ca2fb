"""The oracle's solver: assembled FP64 space-time systems and direct solves.

Follows Sec. 3 of the paper:
  * fixed-point scheme (Eq. solverSU_approx) with the low-rank SU term,
    relaxation alpha (Sec. 3.1) and the stopping rule ||u^{k+1}-u^k||_inf <= delta
    (Sec. 4);
  * the u-system A u = f (Eq. lin_sys_A) with
        A = int int C_m d_t u v + grad u . D grad v + C_r(u^k, w^k) u v
            + C_m sum_k tau_k theta d_t^k u d_t^k v,
    assembled directly on the space-time elements;
  * the w-system L w = g (Eq. lin_sys_L) with L from
        int int d_t w z + b d_e w z   and g from int int b u^k z;
  * the preconditioner matrix A-hat (Eq. preconditioner), here with the
    conductivity scaling D_ll on each direction (the unit-D form of the paper
    is available with unit_D=True);
  * a Newton variant on the u-equation (Jacobian coefficient C_J, w lagged,
    theta frozen at the current iterate, no relaxation);
  * optionally (eps_reaction >= 0) the reaction coefficient in low rank:
    its values at the Greville grid truncated like Theta-hat (reading A7);
  * the comparison method of Sec. 4.2 (stabilization = "supg_sc", on C^0
    time splines): SUPG plus shock capturing in place of the SU term, with
    the f part of SUPG on the right-hand side (oracle/supg.py).

Linear systems are solved with scipy's sparse direct solver (SuperLU).

Test infrastructure only: nothing in the product path imports this package.
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import model
from . import supg
from .spacetime import SpaceTime
from .stabilization import tau_solve, theta_hat, low_rank, interpolate_at_gauss, greville_values


class Oracle:
    def __init__(self, desc):
        self.desc = desc
        self.st = SpaceTime(desc)
        st = self.st
        self.supg = desc["stabilization"] == "supg_sc"
        # tau belongs to SU, whose splines are C^(p-1) in time
        self.tau_coeffs, self.tau_q = (None, None) if self.supg else tau_solve(st)
        tq = st.time_points()[:, None, :, None]
        xs = [x[None, :, None, :] for x in st.xs]
        self.f_q = model.source(desc, xs, tq) * np.ones((st.n_el_t, st.N_el_s, st.nq_t, st.nq_s))
        self.F = st.load(self.f_q)
        if self.supg:
            self.F = self.F + supg.supg_load(st, self.f_q)
        self.lin_terms = st.linear_terms(desc["C_m"], desc["D"])

    # ------------------------------------------------------------ pieces
    def fields(self, u, w):
        st = self.st
        out = dict(u=st.field(u), ut=st.field(u, kt=1), w=st.field(w))
        out["lap"] = sum(self.desc["D"][l] * st.field(u, ks=st.unit(l, 2)) for l in range(st.d))
        return out

    def residual_q(self, fl):
        """R = C_m d_t u - div(D grad u) + I_ion(u, w) - f at every Gauss point."""
        d = self.desc
        return d["C_m"] * fl["ut"] - fl["lap"] + model.ionic_current(d, fl["u"], fl["w"]) - self.f_q

    def ionic(self, u, w, eps=None):
        """Everything the linearization at (u, w) needs: the fields, the
        residual, Theta-hat, its low-rank factors and theta at the Gauss points."""
        d = self.desc
        eps = d["eps_theta"] if eps is None else eps
        fl = self.fields(u, w)
        R = self.residual_q(fl)
        th, info = theta_hat(self.st, R, fl["u"], fl["ut"], d["C_m"], d.get("suppext", "literal"))
        U, s, V = low_rank(th, eps)
        approx = (U * s[None, :]) @ V.T
        theta_q = interpolate_at_gauss(self.st, approx)
        return dict(fields=fl, R=R, theta_hat=th, U=U, s=s, V=V, theta_lr=approx,
                    theta_q=theta_q, **info)

    def operator(self, coef_q, theta_q=None, sc_q=None):
        """Assembled A with reaction coefficient coef_q at the Gauss points and,
        for SU, theta at the Gauss points; for SUPG + shock capturing, the
        SUPG terms with the same reaction coefficient and the shock-capturing
        coefficient sc_q."""
        st = self.st
        d = self.desc
        terms = list(self.lin_terms) + st.mass_terms(coef_q)
        if d["stabilization"] == "su" and theta_q is not None:
            terms += st.su_terms(d["C_m"], self.tau_q, theta_q)
        if self.supg:
            terms += supg.supg_terms(st, d["C_m"], d["D"], coef_q)
            if sc_q is not None:
                terms += supg.sc_terms(st, sc_q, d.get("sc_c", 1.0))
        return st.assemble(terms)

    def supg_ionic(self, u, w):
        """Fields, residual and shock-capturing coefficient at (u, w)."""
        d = self.desc
        fl = self.fields(u, w)
        R = self.residual_q(fl)
        sc_q, den = supg.sc_coefficient(R, fl["u"], fl["ut"], d["C_m"], self.st.T)
        return dict(fields=fl, R=R, sc_q=sc_q, den=den, s=np.zeros(0))

    def reaction_lowrank(self, u, w, kind):
        """Low-rank reaction coefficient (reading A7, the SUPG variant's
        low-rank C_r of Sec. 4.2 carried over to SU): the coefficient (C_r of
        Eq. reaction, or C_J for Newton) of the splines' values at the Greville
        grid, truncated like Theta-hat at the relative Frobenius tolerance
        eps_reaction (Eq. tol), and its (d+1)-linear interpolant at the Gauss
        points.  Returns (coefficient at the Gauss points, U, s, V)."""
        d = self.desc
        ug, wg = greville_values(self.st, u), greville_values(self.st, w)
        C = model.jacobian_coef(d, ug, wg) if kind == "newton" else model.reaction_coef(d, ug, wg)
        U, s, V = low_rank(C, d["eps_reaction"])
        return interpolate_at_gauss(self.st, (U * s[None, :]) @ V.T), U, s, V

    def linearization(self, u, w, kind=None):
        """(A, ionic info) of one nonlinear step at (u, w)."""
        d = self.desc
        kind = d["nonlinear"] if kind is None else kind
        if self.supg:
            if kind != "picard" or d.get("eps_reaction", -1.0) >= 0.0:
                raise NotImplementedError("SUPG + shock capturing: fixed point with the exact reaction only")
            info = self.supg_ionic(u, w)
            coef = model.reaction_coef(d, info["fields"]["u"], info["fields"]["w"])
            info["coef_q"] = coef
            return self.operator(coef, sc_q=info["sc_q"]), info
        info = self.ionic(u, w)
        fl = info["fields"]
        if d.get("eps_reaction", -1.0) >= 0.0:
            coef, Uc, sc, Vc = self.reaction_lowrank(u, w, kind)
            info.update(Uc=Uc, sc=sc, Vc=Vc)
        elif kind == "newton":
            coef = model.jacobian_coef(d, fl["u"], fl["w"])
        else:
            coef = model.reaction_coef(d, fl["u"], fl["w"])
        theta_q = info["theta_q"] if d["stabilization"] == "su" else None
        info["coef_q"] = coef
        return self.operator(coef, theta_q), info

    def precond_matrix(self, unit_D=False):
        """A-hat = int int C_m d_t u v + sum_l D_ll d_l u d_l v + a c1 u v."""
        d, st = self.desc, self.st
        Dp = [1.0] * st.d if unit_D else d["D"]
        terms = st.linear_terms(d["C_m"], Dp) + st.mass_terms(st.const(d["a"] * d["c1"]))
        return st.assemble(terms)

    def w_matrix(self):
        d, st = self.desc, self.st
        z = (0,) * st.d
        return st.assemble([(st.const(1.0), 0, z, 1, z), (st.const(d["b"] * d["d_e"]), 0, z, 0, z)])

    def w_rhs(self, u):
        return self.st.load(self.desc["b"] * self.st.field(u))

    def w_update(self, u):
        """w-tilde = L^{-1} g(u) (Eq. lin_sys_L)."""
        return spla.spsolve(self.w_matrix().tocsc(), self.w_rhs(u))

    def ionic_load(self, u, w):
        """Vector int int I_ion(u, w) v at the Gauss points."""
        fl = self.fields(u, w)
        return self.st.load(model.ionic_current(self.desc, fl["u"], fl["w"]))

    # ------------------------------------------------------------ loops
    def solve(self, max_fp=None, record=False):
        """Nonlinear loop from u^0 = w^0 = 0.  Returns (u, w, history)."""
        d = self.desc
        st = self.st
        max_fp = d["max_fp"] if max_fp is None else max_fp
        u = np.zeros(st.N_dof)
        w = np.zeros(st.N_dof)
        hist = []
        for k in range(max_fp):
            A, info = self.linearization(u, w)
            if d["nonlinear"] == "newton":
                rhs = self.F - self.operator(st.const(0.0), info["theta_q"] if d["stabilization"] == "su" else None) @ u \
                      - self.ionic_load(u, w)
                du = spla.spsolve(A.tocsc(), rhs)
                u_new = u + du
                w_new = np.zeros_like(w) if d["fix_w_zero"] else self.w_update(u)
            else:
                ut = spla.spsolve(A.tocsc(), self.F)
                wt = np.zeros_like(w) if d["fix_w_zero"] else self.w_update(u)
                al = d["alpha"]
                u_new = al * ut + (1 - al) * u
                w_new = al * wt + (1 - al) * w
            diff = np.abs(u_new - u).max()
            if record:
                hist.append(dict(k=k, diff=diff, rank=len(info["s"]), u=u_new.copy(), w=w_new.copy()))
            else:
                hist.append(dict(k=k, diff=diff, rank=len(info["s"])))
            u, w = u_new, w_new
            if diff <= d["delta"]:
                break
        return u, w, hist

    def l2_error(self, u, nq=None):
        """L2(Omega x (0,T)) error of the spline u against the exact solution,
        with a Gauss rule of p+3 points per direction."""
        fine = SpaceTime(self.desc, nq=self.st.p + 3 if nq is None else nq)
        uh = fine.field(u)
        tq = fine.time_points()[:, None, :, None]
        xs = [x[None, :, None, :] for x in fine.xs]
        ue = model.exact_solution(self.desc, xs, tq)
        W = fine.tdir.wq[:, None, :, None] * fine.ws[None, :, None, :]
        err = np.sqrt(np.sum(W * (uh - ue) ** 2))
        nrm = np.sqrt(np.sum(W * ue ** 2 * np.ones_like(uh)))
        return err, nrm
