"""CPU oracle for the QSS source term, analytic Jacobian and implicit step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline leg may import this package; the product path
never does.  The numerics live in ``qss_oracle.cpp`` (plain FP64 C++ with
OpenMP over cells, templated so that the same code runs in complex and
binary128 arithmetic); this module only marshals a mechanism dictionary and
NumPy arrays across ctypes.  It shares no code with the CUDA path.

Parity status of each function (see the test files named beside them):
  eval (wdot, Tdot, C_QSS, J) ..... pinned: closed forms, invariants,
                                     complex-step, central and one-sided FD,
                                     binary128 rerun (tests/test_oracle_*.py);
                                     the Troe broadening by its centre value,
                                     its pole and the affine law of 1/f1 in
                                     1/x; Tdot by a single-coefficient closed
                                     form and conservation of the internal
                                     energy along an integration
  be_step ......................... pinned: closed-form linear case, mass
                                     invariant, Newton residual
  eval_variant (constant-QSS, zero-QSS, FD T column)
                                    pinned: complex step at fixed C_Q (the
                                     definition of the simplified Jacobians),
                                     complex step of the T column
  jac_fd / jac_fd_errbound ........ pinned: first- and second-order
                                     convergence to the complex-step Jacobian
  qss_groups / tarjan ............. pinned: the paper's Fig. 2 example graph
  integrate (backward Euler, BDF2)  pinned: A <=> B relaxation (global error
                                     ~ tol^(1/2) and tol^(2/3)), two BDF2
                                     substeps against the closed-form linear
                                     solves, one substep = one BE step, mass
                                     (tests/test_integrate_oracle.py)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "qss_oracle.cpp")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (OpenMP, libquadmath)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", _LIB_PATH + ".tmp",
               _SRC, "-lquadmath"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.oracle_mech_create.restype = ctypes.c_void_p
        L.oracle_mech_create.argtypes = [ctypes.c_int] * 3 + [_dp] * 4 + [_ip] * 8 + [_dp] * 4
        L.oracle_mech_free.argtypes = [ctypes.c_void_p]
        L.oracle_qss_groups.argtypes = [ctypes.c_void_p, _ip, _ip]
        L.oracle_tarjan.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip, _ip]
        ev = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_eval.argtypes = ev + [ctypes.c_int, ctypes.c_int]
        L.oracle_eval_q128.argtypes = ev + [ctypes.c_int]
        L.oracle_eval_errbound.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, _dp, _dp, _dp,
                                           ctypes.c_int]
        L.oracle_eval_phi.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, ctypes.c_int]
        L.oracle_jac_complex_step.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp,
                                              ctypes.c_double, _dp, ctypes.c_int]
        L.oracle_jac_fd.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int]
        L.oracle_jac_fd_errbound.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.oracle_eval_variant.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, ctypes.c_int,
                                          ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.oracle_jac_cs_fixed_cq.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, _dp,
                                             ctypes.c_double, _dp, ctypes.c_int]
        L.oracle_integrate.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, ctypes.c_int, _dp, _dp, _dp] + \
            [ctypes.c_double] * 5 + [ctypes.c_int] + [ctypes.c_double] * 3 + [ctypes.c_int, ctypes.c_int, _ip, _ip,
                                                                               ctypes.c_int]
        L.oracle_qss_residual.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp, _dp, _dp,
                                          ctypes.c_int]
        L.oracle_qss_newton_q128.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, _dp, _dp,
                                             ctypes.c_int, _dp, ctypes.c_int]
        L.oracle_be_step.argtypes = [ctypes.c_void_p, _i64, _i64, _dp, ctypes.c_int, _dp, _dp, _dp,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, _ip, _ip, ctypes.c_int]
        _lib = L
    return _lib


def _p(a, t=_dp):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def tarjan(n_vertices, edges):
    """SCCs of a digraph given as (u, v) pairs meaning "u needs v".
    Returns the components in solve order (each after those it needs)."""
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    comp_of = np.zeros(n_vertices, dtype=np.int32)
    order = np.zeros(n_vertices, dtype=np.int32)
    nc = lib().oracle_tarjan(n_vertices, len(edges), _p(eu, _ip), _p(ev, _ip), _p(comp_of, _ip),
                             _p(order, _ip))
    comps = [[] for _ in range(nc)]
    for v in order:
        comps[comp_of[v]].append(int(v))
    return comps


class OracleMech:
    """A mechanism dictionary loaded into the C++ oracle."""

    def __init__(self, mech: dict):
        sp = mech["species"]
        tr = [s for s in sp if not s["qss"]]
        qs = [s for s in sp if s["qss"]]
        order = tr + qs
        self.names = [s["name"] for s in order]
        idx = {nm: i for i, nm in enumerate(self.names)}
        self.N, self.Q, self.M = len(tr), len(qs), len(mech["reactions"])
        N, Q, M = self.N, self.Q, self.M
        self.W = np.array([s["W"] for s in tr], dtype=np.float64)
        nlo = np.array([s["nasa_lo"] for s in order], dtype=np.float64).reshape(-1)
        nhi = np.array([s["nasa_hi"] for s in order], dtype=np.float64).reshape(-1)
        tmid = np.array([s.get("Tmid", 1000.0) for s in order], dtype=np.float64)
        nl = np.zeros(M, np.int32); nr = np.zeros(M, np.int32)
        lsp = np.zeros(4 * M, np.int32); lnu = np.zeros(4 * M, np.int32)
        rsp = np.zeros(4 * M, np.int32); rnu = np.zeros(4 * M, np.int32)
        rev = np.zeros(M, np.int32); kind = np.zeros(M, np.int32)
        arr = np.zeros(3 * M); low = np.zeros(3 * M); troe = np.zeros(4 * M)
        troe[1::4] = 1.0; troe[2::4] = 1.0; troe[3::4] = 1.0
        eff = np.ones(N * M)
        for j, r in enumerate(mech["reactions"]):
            for i, (s, nu) in enumerate(r["reactants"].items()):
                lsp[4 * j + i] = idx[s]; lnu[4 * j + i] = nu
            nl[j] = len(r["reactants"])
            for i, (s, nu) in enumerate(r["products"].items()):
                rsp[4 * j + i] = idx[s]; rnu[4 * j + i] = nu
            nr[j] = len(r["products"])
            rev[j] = (1 if r["reversible"] else 0) | (0 if r.get("forward", True) else 2)
            arr[3 * j:3 * j + 3] = (r["A"], r["b"], r["Ea"])
            if r.get("third_body"):
                kind[j] = 1
                for s, e in r["third_body"]["efficiencies"].items():
                    if idx[s] < N:
                        eff[j * N + idx[s]] = e
            if r.get("falloff"):
                kind[j] = 2
                lo = r["falloff"]["low"]
                low[3 * j:3 * j + 3] = (lo["A"], lo["b"], lo["Ea"])
                troe[4 * j:4 * j + 4] = r["falloff"]["troe"]
        self._keep = (self.W, nlo, nhi, tmid, nl, lsp, lnu, nr, rsp, rnu, rev, kind, arr, low, troe, eff)
        self.h = lib().oracle_mech_create(N, Q, M, _p(self.W), _p(nlo), _p(nhi), _p(tmid),
                                          _p(nl, _ip), _p(lsp, _ip), _p(lnu, _ip), _p(nr, _ip),
                                          _p(rsp, _ip), _p(rnu, _ip), _p(rev, _ip), _p(kind, _ip),
                                          _p(arr), _p(low), _p(troe), _p(eff))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.oracle_mech_free(self.h)
            self.h = None

    @property
    def n(self):
        return self.N + 1

    def qss_groups(self):
        sizes = np.zeros(max(self.Q, 1), np.int32)
        members = np.zeros(max(self.Q, 1), np.int32)
        ng = lib().oracle_qss_groups(self.h, _p(sizes, _ip), _p(members, _ip))
        out, pos = [], 0
        for g in range(ng):
            out.append([int(x) for x in members[pos:pos + sizes[g]]])
            pos += sizes[g]
        return out

    def _state(self, rho, T, Y):
        rho, T, Y = _f64(rho), _f64(T), _f64(Y)
        ld = T.shape[0]
        assert Y.shape == (self.N, ld) and rho.shape == (ld,)
        return rho, T, Y, ld

    def eval(self, rho, T, Y, ncells=None, jac=True, ordered=True, cq=False, nthreads=0):
        rho, T, Y, ld = self._state(rho, T, Y)
        nc = ld if ncells is None else ncells
        w = np.zeros((self.N, ld)); td = np.zeros(ld)
        J = np.zeros((self.n * self.n, ld)) if jac else None
        C = np.zeros((max(self.Q, 1), ld)) if cq else None
        nf = lib().oracle_eval(self.h, nc, ld, _p(rho), _p(T), _p(Y), _p(w), _p(td), _p(J), _p(C),
                               1 if ordered else 0, nthreads)
        if nf:
            raise RuntimeError(f"oracle evaluation failed in {nf} cells")
        return {"wdot": w, "Tdot": td, "jac": J, "cq": C}

    def eval_q128(self, rho, T, Y, ncells=None, jac=True, cq=False, nthreads=0):
        rho, T, Y, ld = self._state(rho, T, Y)
        nc = ld if ncells is None else ncells
        w = np.zeros((self.N, ld)); td = np.zeros(ld)
        J = np.zeros((self.n * self.n, ld)) if jac else None
        C = np.zeros((max(self.Q, 1), ld)) if cq else None
        nf = lib().oracle_eval_q128(self.h, nc, ld, _p(rho), _p(T), _p(Y), _p(w), _p(td), _p(J),
                                    _p(C), nthreads)
        if nf:
            raise RuntimeError(f"oracle evaluation failed in {nf} cells")
        return {"wdot": w, "Tdot": td, "jac": J, "cq": C}

    def errbound(self, rho, T, Y, ncells=None, jac=True, nthreads=0):
        """First-order rounding-error bounds of ``eval``'s FP64 results, as
        absolute values (running error analysis, multiplied by u = 2^-53)."""
        rho, T, Y, ld = self._state(rho, T, Y)
        nc = ld if ncells is None else ncells
        w = np.zeros((self.N, ld)); td = np.zeros(ld)
        J = np.zeros((self.n * self.n, ld)) if jac else None
        nf = lib().oracle_eval_errbound(self.h, nc, ld, _p(rho), _p(T), _p(Y), _p(w), _p(td), _p(J),
                                        nthreads)
        if nf:
            raise RuntimeError(f"oracle evaluation failed in {nf} cells")
        u = 2.0 ** -53
        return {"wdot": w * u, "Tdot": td * u, "jac": (J * u) if jac else None}

    def eval_phi(self, phi, jac=True, nthreads=0, strict=True):
        """f = (wdot, Tdot) and J at phi = (C, T) given per cell.  With
        strict=False, cells whose evaluation fails are returned as NaN."""
        phi = _f64(phi)
        ld = phi.shape[1]
        f = np.full((self.n, ld), np.nan)
        J = np.full((self.n * self.n, ld), np.nan) if jac else None
        nf = lib().oracle_eval_phi(self.h, ld, ld, _p(phi), _p(f), _p(J), nthreads)
        if nf and strict:
            raise RuntimeError(f"oracle evaluation failed in {nf} cells")
        return f, J

    def jac_complex_step(self, rho, T, Y, hrel=1e-30, nthreads=0):
        rho, T, Y, ld = self._state(rho, T, Y)
        J = np.zeros((self.n * self.n, ld))
        nf = lib().oracle_jac_complex_step(self.h, ld, ld, _p(rho), _p(T), _p(Y), hrel, _p(J), nthreads)
        if nf:
            raise RuntimeError("complex-step failed")
        return J

    def jac_fd(self, rho, T, Y, dC, dT, central=True, nthreads=0):
        rho, T, Y, ld = self._state(rho, T, Y)
        J = np.zeros((self.n * self.n, ld))
        nf = lib().oracle_jac_fd(self.h, ld, ld, _p(rho), _p(T), _p(Y), dC, dT, 2 if central else 1,
                                 _p(J), nthreads)
        if nf:
            raise RuntimeError("finite differences failed")
        return J

    def jac_fd_errbound(self, rho, T, Y, dC, dT, central=True, nthreads=0):
        """``jac_fd`` in the running-error type: (J, absolute rounding bound)."""
        rho, T, Y, ld = self._state(rho, T, Y)
        J = np.zeros((self.n * self.n, ld)); E = np.zeros_like(J)
        nf = lib().oracle_jac_fd_errbound(self.h, ld, ld, _p(rho), _p(T), _p(Y), dC, dT,
                                          2 if central else 1, _p(J), _p(E), nthreads)
        if nf:
            raise RuntimeError("finite differences failed")
        return J, E * 2.0 ** -53

    JAC_VARIANTS = {"exact": 0, "const_qss": 1, "zero_qss": 2}

    def eval_variant(self, rho, T, Y, jac_variant="exact", t_column="analytic", nthreads=0):
        """The Jacobian of a simplified construction (Section 3.2.1) and/or
        with the finite-difference T column (Section 3.2.2), with running
        error bounds: {"wdot", "Tdot", "jac", "jac_err"} (bounds absolute)."""
        rho, T, Y, ld = self._state(rho, T, Y)
        w = np.zeros((self.N, ld)); td = np.zeros(ld)
        J = np.zeros((self.n * self.n, ld)); E = np.zeros_like(J)
        nf = lib().oracle_eval_variant(self.h, ld, ld, _p(rho), _p(T), _p(Y),
                                       self.JAC_VARIANTS[jac_variant], 1 if t_column == "fd" else 0,
                                       _p(w), _p(td), _p(J), _p(E), nthreads)
        if nf:
            raise RuntimeError(f"oracle evaluation failed in {nf} cells")
        return {"wdot": w, "Tdot": td, "jac": J, "jac_err": E * 2.0 ** -53}

    def jac_cs_fixed_cq(self, rho, T, Y, cq, hrel=1e-30, nthreads=0):
        """Complex-step Jacobian of (wdot, Tdot) with the QSS concentrations
        held at the given values cq [Q][ld] (no QSS solve)."""
        rho, T, Y, ld = self._state(rho, T, Y)
        cq = _f64(cq if self.Q else np.zeros((1, ld)))
        J = np.zeros((self.n * self.n, ld))
        nf = lib().oracle_jac_cs_fixed_cq(self.h, ld, ld, _p(rho), _p(T), _p(Y), _p(cq), hrel, _p(J),
                                          nthreads)
        if nf:
            raise RuntimeError("complex-step failed")
        return J

    def qss_residual(self, rho, T, Y, nthreads=0):
        rho, T, Y, ld = self._state(rho, T, Y)
        r = np.zeros((max(self.Q, 1), ld)); m = np.zeros((max(self.Q, 1), ld))
        nf = lib().oracle_qss_residual(self.h, ld, ld, _p(rho), _p(T), _p(Y), _p(r), _p(m), nthreads)
        if nf:
            raise RuntimeError("qss residual failed")
        return r, m

    def qss_newton_q128(self, rho, T, Y, iters=4, nthreads=0):
        rho, T, Y, ld = self._state(rho, T, Y)
        C = np.zeros((max(self.Q, 1), ld))
        nf = lib().oracle_qss_newton_q128(self.h, ld, ld, _p(rho), _p(T), _p(Y), iters, _p(C), nthreads)
        if nf:
            raise RuntimeError("qss newton failed")
        return C

    def be_step(self, rho, T, Y, dt, ncells=None, rtol=1e-12, atol_C=1e-20, atol_T=1e-10,
                max_iter=50, nthreads=0):
        """One backward-Euler step; returns (T_new, Y_new, iters, status)."""
        rho, T, Y, ld = self._state(rho, T, Y)
        nc = ld if ncells is None else ncells
        T2, Y2 = T.copy(), Y.copy()
        dt = np.atleast_1d(_f64(dt))
        stride = 1 if dt.shape[0] > 1 else 0
        it = np.zeros(ld, np.int32); st = np.zeros(ld, np.int32)
        lib().oracle_be_step(self.h, nc, ld, _p(dt), stride, _p(rho), _p(T2), _p(Y2), rtol, atol_C,
                             atol_T, max_iter, _p(it, _ip), _p(st, _ip), nthreads)
        return T2, Y2, it, st

    def conc(self, rho, Y):
        """C_k = rho Y_k / W_k (the oracle's first step), for tests."""
        return _f64(rho)[None, :] * _f64(Y) / self.W[:, None]

    def integrate(self, rho, T, Y, dt_total, rtol=1e-4, atol_C=1e-10, atol_T=1e-4, h0=0.0, h_min=1e-14,
                  max_rounds=400, newton_rtol=1e-12, newton_atol_C=1e-20, newton_atol_T=1e-10,
                  max_iter=6, order=1, nthreads=0):
        """Integration over dt_total by error-controlled substeps of order 1
        (backward Euler) or 2 (variable-step BDF2); returns (T_new, Y_new,
        nsteps, status)."""
        rho, T, Y, ld = self._state(rho, T, Y)
        T2, Y2 = T.copy(), Y.copy()
        dt = np.atleast_1d(_f64(dt_total))
        ns = np.zeros(ld, np.int32); st = np.zeros(ld, np.int32)
        lib().oracle_integrate(self.h, ld, ld, _p(dt), 1 if dt.size > 1 else 0, _p(rho), _p(T2), _p(Y2),
                               rtol, atol_C, atol_T, h0, h_min, max_rounds, newton_rtol, newton_atol_C,
                               newton_atol_T, max_iter, int(order), _p(ns, _ip), _p(st, _ip), nthreads)
        return T2, Y2, ns, st

