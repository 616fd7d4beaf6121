"""Symbolic model of the QSS source term and its analytic Jacobian.

Builds, on one hash-consed DAG (``expr.Graph``):

* per-species NASA-7 thermo functions of T (g/RT, h/RT, c_p/R);
* rate constants: Arrhenius, third-body, Troe falloff (Section 2.1 names
  "any elementary reaction type"; the forms are the CHEMKIN ones);
* the rates of progress and production rates, Eqs. (progRates, ReacMech),
  with the QSS concentrations as placeholders C_Q;
* the QSS linear system: A = d omega_Q / d C_Q and b = omega_Q(C_Q = 0),
  obtained by symbolic differentiation of the production rates (the exact
  content of Eq. (full_QSSsystem), whose printed form is garbled), then solved
  in the condensed SCC order of the QSS digraph (Section 2.3, Appendix B):
  singletons by division, groups by Gaussian elimination;
* the analytic Jacobian of phi = (C_1..C_N, T), Eq. (JacExptr), through the
  chain rule of Eq. (JQSS):  J = dw/dphi|_{C_Q} + dw/dC_Q * dC_Q/dphi, with
  dC_Q/dphi = -A^{-1} d omega_Q/dphi|_{C_Q} solved in the same SCC order.
  Third-body concentrations [M]_j are placeholders as well, and their
  dependence on C enters as one more chain-rule level (d[M]_j/dC_k is the
  collision efficiency), which keeps the dense third-body contributions to a
  rank-one update per row;
* the simplified Jacobians of Section 3.2.1 (constant-QSS and zero-QSS) and
  the finite-difference temperature column of Section 3.2.2 as build options;
* the temperature row from Tdot = -T sum_k (h_k/RT - 1) w_k / sum_k C_k (c_p,k/R - 1)
  (constant volume), differentiated with the production rates as
  placeholders and closed with the rows of J.

Elimination inside an SCC group uses no pivoting: -A restricted to a group is
a nonsingular M-matrix (nonpositive off-diagonal after the sign change,
column diagonally dominant), for which Gaussian elimination in natural order
is stable.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List

from .expr import Graph
from .graph import tarjan_scc
from .mech import MechIR, P_STD, R_GAS, MechanismError

LN10 = math.log(10.0)


@dataclass
class Model:
    ir: MechIR
    g: Graph
    C: List[int]
    T: int
    wdot: List[int]
    Tdot: int
    jac: List[List[int]]            # (N+1) x (N+1), row i, column j
    bind: Dict[int, int]            # placeholder VAR -> value node
    groups: List[List[int]]         # QSS solve order (QSS indices)
    cq_value: List[int]
    stats: dict = field(default_factory=dict)
    parts: dict = field(default_factory=dict)
    fd_vars: tuple = None           # (T + h, T - h, 1/(2h)) inputs of the FD T column
    jac_variant: str = "exact"
    t_column: str = "analytic"


JAC_VARIANTS = ("exact", "const_qss", "zero_qss")
T_COLUMNS = ("analytic", "fd")


class _Builder:
    def __init__(self, ir: MechIR, jac_variant="exact", t_column="analytic"):
        if jac_variant not in JAC_VARIANTS or t_column not in T_COLUMNS:
            raise ValueError(f"unknown Jacobian variant {jac_variant!r} / T column {t_column!r}")
        self.jac_variant = jac_variant
        self.t_column = t_column
        self.ir = ir
        g = self.g = Graph()
        N, Q = ir.N, ir.Q
        self.C = [g.var(f"C{k}") for k in range(N)]
        self.T = g.var("T")
        self.CQ = [g.var(f"CQ{m}") for m in range(Q)]
        T = self.T
        self.lnT = g.log(T)
        self.invT = g.recip(T)
        self.Tp = {1: T}
        self.Tp[2] = g.mul(T, T)
        self.Tp[3] = g.mul(self.Tp[2], T)
        self.Tp[4] = g.mul(self.Tp[3], T)
        self._thermo = {}
        self._G = {}
        self.bind: Dict[int, int] = {}
        self.Mvar: Dict[tuple, int] = {}
        self.Mval: Dict[tuple, int] = {}
        self.Ctot = None

    # ------------------------------------------------------------- thermo
    def _poly(self, coeffs):
        """c0 + c1 T + c2 T^2 + ... + cl lnT + ci invT over shared T powers."""
        g = self.g
        c0, cT, cT2, cT3, cT4, cinv, cln = coeffs
        terms = [g.const(c0)]
        for k, c in ((1, cT), (2, cT2), (3, cT3), (4, cT4)):
            if c != 0.0:
                terms.append(g.mul(g.const(c), self.Tp[k]))
        if cinv != 0.0:
            terms.append(g.mul(g.const(cinv), self.invT))
        if cln != 0.0:
            terms.append(g.mul(g.const(cln), self.lnT))
        return g.sum(terms)

    def thermo(self, s, what):
        key = (s, what)
        if key in self._thermo:
            return self._thermo[key]
        ir = self.ir

        def coeffs(a):
            a1, a2, a3, a4, a5, a6, a7 = a
            if what == "gRT":   # h/RT - s/R
                return (a1 - a7, -a2 / 2.0, -a3 / 6.0, -a4 / 12.0, -a5 / 20.0, a6, -a1)
            if what == "hRT":
                return (a1, a2 / 2.0, a3 / 3.0, a4 / 4.0, a5 / 5.0, a6, 0.0)
            if what == "cpR":
                return (a1, a2, a3, a4, a5, 0.0, 0.0)
            raise KeyError(what)

        lo, hi = ir.nasa_lo[s], ir.nasa_hi[s]
        if lo == hi:
            node = self._poly(coeffs(lo))
        else:
            cond = self.g.lt(self.T, ir.Tmid[s])
            node = self.g.select(cond, self._poly(coeffs(lo)), self._poly(coeffs(hi)))
        self._thermo[key] = node
        return node

    def Gfac(self, s, sign):
        """exp(+g_s/RT) (sign=+1) or exp(-g_s/RT) (sign=-1)."""
        key = (s, sign)
        if key not in self._G:
            x = self.thermo(s, "gRT")
            self._G[key] = self.g.exp(x if sign > 0 else self.g.neg(x))
        return self._G[key]

    # -------------------------------------------------------------- rates
    def arrhenius_arg(self, lnA, b, EaR):
        g = self.g
        terms = [g.const(lnA)]
        if b != 0.0:
            terms.append(g.mul(g.const(b), self.lnT))
        if EaR != 0.0:
            terms.append(g.mul(g.const(-EaR), self.invT))
        return g.sum(terms)

    def third_body(self, rx):
        """Placeholder [M] for the reaction's efficiency table; its value is
        sum_k C_k + sum_k (eff_k - 1) C_k over transported species."""
        g = self.g
        key = tuple(sorted(rx.eff.items()))
        if key not in self.Mvar:
            v = g.var(f"M{len(self.Mvar)}")
            if self.Ctot is None:
                self.Ctot = g.sum(self.C)
            val = self.Ctot
            for k, e in key:
                val = g.add(val, g.mul(g.const(e - 1.0), self.C[k]))
            self.Mvar[key] = v
            self.Mval[key] = val
            self.bind[v] = val
        return self.Mvar[key], key

    def rates(self, rx):
        """(k_f, k_b) including falloff and third-body factors."""
        g = self.g
        arg = self.arrhenius_arg(rx.lnA, rx.b, rx.EaR)
        kinf = g.exp(arg)
        if rx.kind == 1:
            M, _ = self.third_body(rx)
            kf = g.mul(kinf, M)
        elif rx.kind == 2:
            M, _ = self.third_body(rx)
            arg0 = self.arrhenius_arg(rx.lnA0, rx.b0, rx.Ea0R)
            lnPr0 = g.sub(arg0, arg)                   # ln(k0/kinf)
            Pr = g.mul(g.exp(lnPr0), M)
            alpha, T3, T1, T2 = rx.troe
            terms = []
            if alpha != 1.0:
                terms.append(g.mul(g.const(1.0 - alpha), g.exp(g.mul(g.const(-1.0 / T3), self.T))))
            if alpha != 0.0:
                terms.append(g.mul(g.const(alpha), g.exp(g.mul(g.const(-1.0 / T1), self.T))))
            terms.append(g.exp(g.mul(g.const(-T2), self.invT)))
            Fcent = g.sum(terms)
            lFc = g.mul(g.const(1.0 / LN10), g.log(Fcent))
            lPr = g.mul(g.const(1.0 / LN10), g.add(lnPr0, g.log(M)))
            c = g.add(g.const(-0.4), g.mul(g.const(-0.67), lFc))
            nn = g.add(g.const(0.75), g.mul(g.const(-1.27), lFc))
            x = g.add(lPr, c)
            den = g.sub(nn, g.mul(g.const(0.14), x))
            den2 = g.mul(den, den)
            # log10 F = log10 Fcent / (1 + (x/den)^2) = log10 Fcent den^2 / (den^2 + x^2)
            lF = g.mul(g.mul(lFc, den2), g.recip(g.add(den2, g.mul(x, x))))
            F = g.exp(g.mul(g.const(LN10), lF))
            kf = g.mul(g.mul(kinf, g.mul(Pr, g.recip(g.add(g.ONE, Pr)))), F)
        else:
            kf = kinf
        kb = None
        if rx.reversible:
            # 1/K_c = exp(sum_s nu_s g_s/RT) (R T / P0)^dnu, as a product of
            # per-species factors; its logarithm carries the derivative.
            facs = []
            lnarg = []
            dnu = 0
            for s, nu in rx.rhs:
                facs += [self.Gfac(s, +1)] * nu
                lnarg.append(g.mul(g.const(float(nu)), self.thermo(s, "gRT")))
                dnu += nu
            for s, nu in rx.lhs:
                facs += [self.Gfac(s, -1)] * nu
                lnarg.append(g.mul(g.const(-float(nu)), self.thermo(s, "gRT")))
                dnu -= nu
            if dnu > 0:
                facs += [g.mul(g.const(R_GAS / P_STD), self.T)] * dnu
            elif dnu < 0:
                facs += [g.mul(g.const(P_STD / R_GAS), self.invT)] * (-dnu)
            if dnu != 0:
                lnarg.append(g.mul(g.const(float(dnu)), g.add(self.lnT, g.const(math.log(R_GAS / P_STD)))))
            inv_kc = g.fact(g.prod(facs), g.sum(lnarg))
            kb = g.mul(kf, inv_kc)
        return kf, kb

    # ------------------------------------------------------------- build
    def build(self) -> Model:
        g, ir = self.g, self.ir
        N, Q = ir.N, ir.Q
        nsp = N + Q
        Qj = []
        for rx in ir.rxns:
            kf, kb = self.rates(rx)
            pf = g.prod([g.powi(self.C[s], nu) for s, nu in rx.lhs if s < N])
            qf = g.mul(kf, pf)
            if rx.qss_l >= 0:
                qf = g.mul(qf, self.CQ[rx.qss_l])
            if not rx.forward:
                qf = g.ZERO          # reverse-only: k_b = k_f / K_c is kept
            if kb is not None:
                pb = g.prod([g.powi(self.C[s], nu) for s, nu in rx.rhs if s < N])
                qb = g.mul(kb, pb)
                if rx.qss_r >= 0:
                    qb = g.mul(qb, self.CQ[rx.qss_r])
                Qj.append(g.sub(qf, qb))
            else:
                Qj.append(qf)
        # production rates of all species (QSS placeholders and [M] unbound)
        omega = [g.ZERO] * nsp
        for j, rx in enumerate(ir.rxns):
            nu = {}
            for s, v in rx.lhs:
                nu[s] = nu.get(s, 0) - v
            for s, v in rx.rhs:
                nu[s] = nu.get(s, 0) + v
            for s, v in sorted(nu.items()):
                if v != 0:
                    omega[s] = g.add(omega[s], g.mul(g.const(float(v)), Qj[j]))
        # ---- QSS system A C_Q + b = 0 -------------------------------------
        A = [[g.d(omega[N + m], self.CQ[n]) for n in range(Q)] for m in range(Q)]
        zero_map = {v: g.ZERO for v in self.CQ}
        bvec = [g.subs(omega[N + m], zero_map) if Q else None for m in range(Q)]
        for m in range(Q):
            for n in range(Q):
                for p in range(Q):
                    if g.depends_on(A[m][n], self.CQ[p]):
                        raise MechanismError("QSS relations are not linear in C_Q")
        adj = [[n for n in range(Q) if n != m and A[m][n] != g.ZERO] for m in range(Q)]
        groups = tarjan_scc(adj)
        for m in range(Q):
            if A[m][m] == g.ZERO:
                raise MechanismError(f"QSS species {ir.names[N + m]} has no consumption channel")
        cqv = [None] * Q
        elim = {}   # per group: (order, multipliers, pivots-recip, U)
        for comp in groups:
            rhs = {}
            for m in comp:
                acc = bvec[m]
                for n in range(Q):
                    if n not in comp and A[m][n] != g.ZERO:
                        acc = g.add(acc, g.mul(A[m][n], cqv[n]))
                rhs[m] = g.neg(acc)
            sol, fac = self._group_solve(comp, A, rhs, None)
            elim[tuple(comp)] = fac
            for m in comp:
                cqv[m] = sol[m]
        for m in range(Q):
            self.bind[self.CQ[m]] = cqv[m]
        # ---- Jacobian ------------------------------------------------------
        n = N + 1
        phi = self.C + [self.T]
        Mkeys = list(self.Mvar.keys())
        Gm = [[None] * n for _ in range(nsp)]
        for r in range(nsp):
            dM = [g.d(omega[r], self.Mvar[key]) for key in Mkeys]
            U = g.sum(dM)
            for k in range(N):
                acc = g.add(g.d(omega[r], self.C[k]), U)
                for mi, key in enumerate(Mkeys):
                    if dM[mi] == g.ZERO:
                        continue
                    e = dict(key).get(k)
                    if e is not None:
                        acc = g.add(acc, g.mul(g.const(e - 1.0), dM[mi]))
                Gm[r][k] = acc
            Gm[r][N] = g.d(omega[r], self.T)
        # X = dC_Q/dphi = -A^{-1} G_Q, in the same SCC order
        X = [[None] * n for _ in range(Q)]
        for comp in groups:
            for c in range(n):
                rhs = {}
                for m in comp:
                    acc = Gm[N + m][c]
                    for q in range(Q):
                        if q not in comp and A[m][q] != g.ZERO:
                            acc = g.add(acc, g.mul(A[m][q], X[q][c]))
                    rhs[m] = g.neg(acc)
                sol, _ = self._group_solve(comp, A, rhs, elim[tuple(comp)])
                for m in comp:
                    X[m][c] = sol[m]
        P = [[g.d(omega[i], self.CQ[m]) for m in range(Q)] for i in range(N)]
        J = [[None] * n for _ in range(n)]
        zero_q = {v: g.ZERO for v in self.CQ}
        for i in range(N):
            for c in range(n):
                acc = Gm[i][c]
                if self.jac_variant == "exact":
                    for m in range(Q):
                        if P[i][m] != g.ZERO and X[m][c] != g.ZERO:
                            acc = g.add(acc, g.mul(P[i][m], X[m][c]))
                elif self.jac_variant == "zero_qss" and Q:
                    acc = g.subs(acc, zero_q)
                J[i][c] = acc
        fd_vars = None
        if self.t_column == "fd":
            # Section 3.2.2: dw/dT by a central difference of the production
            # rates at T + h and T - h (h an exact power of two, so that both
            # shifted temperatures and 1/(2h) are exact); the full QSS
            # evaluation, C_Q included, is repeated at each temperature.
            fd_vars = (g.var("Tp"), g.var("Tm"), g.var("inv2h"))
            cq_full = {self.CQ[m]: cqv[m] for m in range(Q)}
            for i in range(N):
                full = g.subs(omega[i], cq_full) if Q else omega[i]
                up = g.subs(full, {self.T: fd_vars[0]})
                dn = g.subs(full, {self.T: fd_vars[1]})
                J[i][N] = g.mul(g.sub(up, dn), fd_vars[2])
        # ---- temperature equation and row ------------------------------------
        Wv = [g.var(f"W{i}") for i in range(N)]
        Su = g.sum([g.mul(g.sub(self.thermo(k, "hRT"), g.ONE), Wv[k]) for k in range(N)])
        Scv = g.sum([g.mul(self.C[k], g.sub(self.thermo(k, "cpR"), g.ONE)) for k in range(N)])
        Tdot_ph = g.neg(g.mul(g.mul(self.T, Su), g.recip(Scv)))
        for i in range(N):
            self.bind[Wv[i]] = omega[i]
        for c in range(n):
            acc = g.d(Tdot_ph, phi[c])
            for i in range(N):
                dW = g.d(Tdot_ph, Wv[i])
                if dW != g.ZERO and J[i][c] != g.ZERO:
                    acc = g.add(acc, g.mul(dW, J[i][c]))
            J[N][c] = acc
        model = Model(ir=ir, g=g, C=self.C, T=self.T, wdot=omega[:N], Tdot=Tdot_ph, jac=J,
                      bind=self.bind, groups=groups, cq_value=cqv, fd_vars=fd_vars,
                      jac_variant=self.jac_variant, t_column=self.t_column)
        model.parts = {"G": Gm, "X": X, "P": P, "A": A}
        model.stats = {"nodes": len(g.op), "n_third_body_tables": len(Mkeys),
                       "groups": [len(c) for c in groups]}
        return model

    def _group_solve(self, comp, A, rhs, fac):
        """Solve A[comp, comp] x = rhs by Gaussian elimination in natural order.
        ``fac`` reuses the multipliers/pivot reciprocals of an earlier solve."""
        g = self.g
        s = len(comp)
        if s == 1:
            m = comp[0]
            piv = g.recip(A[m][m]) if fac is None else fac["piv"][0]
            return {m: g.mul(rhs[m], piv)}, {"piv": [piv]}
        if fac is None:
            U = [[A[comp[i]][comp[j]] for j in range(s)] for i in range(s)]
            L = [[g.ZERO] * s for _ in range(s)]
            piv = [None] * s
            for k in range(s):
                piv[k] = g.recip(U[k][k])
                for i in range(k + 1, s):
                    if U[i][k] == g.ZERO:
                        continue
                    L[i][k] = g.mul(U[i][k], piv[k])
                    for j in range(k + 1, s):
                        if U[k][j] != g.ZERO:
                            U[i][j] = g.sub(U[i][j], g.mul(L[i][k], U[k][j]))
                    U[i][k] = g.ZERO
            fac = {"piv": piv, "L": L, "U": U}
        L, U, piv = fac["L"], fac["U"], fac["piv"]
        y = [rhs[m] for m in comp]
        for k in range(s):
            for i in range(k + 1, s):
                if L[i][k] != g.ZERO and y[k] != g.ZERO:
                    y[i] = g.sub(y[i], g.mul(L[i][k], y[k]))
        x = [None] * s
        for k in range(s - 1, -1, -1):
            acc = y[k]
            for j in range(k + 1, s):
                if U[k][j] != g.ZERO and x[j] != g.ZERO:
                    acc = g.sub(acc, g.mul(U[k][j], x[j]))
            x[k] = g.mul(acc, piv[k])
        return {comp[i]: x[i] for i in range(s)}, fac


def build_model(ir: MechIR, jac_variant: str = "exact", t_column: str = "analytic") -> Model:
    """``jac_variant``: "exact" (Eq. JQSS with the chain rule through C_Q),
    "const_qss" (the second term of Eq. JQSS dropped: C_Q held at its solved
    value) or "zero_qss" (that term dropped and C_Q set to zero inside the
    Jacobian), Section 3.2.1.  ``t_column``: "analytic" or "fd" (central
    difference in T, Section 3.2.2).  The temperature row always follows from
    the species rows by the chain rule; wdot and Tdot are exact in every
    variant."""
    return _Builder(ir, jac_variant, t_column).build()
