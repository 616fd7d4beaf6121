"""Python binding of libqss.so (ctypes; argument marshalling only).

Every computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no fallback: if the shared library or the
mechanism artefact is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqss.so")

QSS_OK = 0
QSS_ERRORS = {-1: "INVALID_ARG", -2: "MECH_FORMAT", -3: "CUDA", -4: "OOM", -5: "NOT_CONVERGED",
              -6: "TIMEOUT", -7: "BUDGET", -8: "UNIMPLEMENTED"}
QSS_LU_FP64 = 0
QSS_LU_FP32_IR = 1
QSS_LU_MIXED = 2

_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


class QSSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qss error {code} ({QSS_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class NewtonOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("rtol", ctypes.c_double), ("atol_C", ctypes.c_double),
                ("atol_T", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("jac_reuse", ctypes.c_int)]


def newton_opts(max_iter=None, rtol=1e-12, atol_C=1e-20, atol_T=1e-10, max_refine=10, refine_tol=1e-8,
                jac_reuse=0) -> NewtonOpts:
    """qss_newton_opts with the library's defaults (full Newton, at most 20
    iterations).  With jac_reuse the default cap is 40: iterations that keep
    the Jacobian converge linearly, and each costs a source-term evaluation
    instead of a Jacobian."""
    if max_iter is None:
        max_iter = 40 if jac_reuse else 20
    return NewtonOpts(max_iter, rtol, atol_C, atol_T, max_refine, refine_tol, jac_reuse)


class IntegrateOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol_C", ctypes.c_double), ("atol_T", ctypes.c_double),
                ("h0", ctypes.c_double), ("h_min", ctypes.c_double), ("max_rounds", ctypes.c_int),
                ("newton", NewtonOpts), ("order", ctypes.c_int)]


def integrate_opts(rtol=1e-4, atol_C=1e-10, atol_T=1e-4, h0=0.0, h_min=1e-14, max_rounds=400,
                   newton: Optional["NewtonOpts"] = None, order=1) -> IntegrateOpts:
    """order 1: backward-Euler substeps; 2: variable-step BDF2 substeps.  The
    substep Newton defaults to at most 6 iterations (the library's default)."""
    return IntegrateOpts(rtol, atol_C, atol_T, h0, h_min, max_rounds,
                         newton if newton is not None else NewtonOpts(6, 1e-12, 1e-20, 1e-10, 10, 1e-8),
                         order)


class ServeOpts(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("max_batch_cells", ctypes.c_int64),
                ("newton", ctypes.POINTER(NewtonOpts)), ("graphs", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_uint64) for nm in ("submitted", "completed", "rejected", "queued",
                                                 "in_flight", "batches", "cells_completed",
                                                 "bytes_in_use", "bytes_peak")] + \
               [(nm, ctypes.c_double) for nm in ("p50_latency_us", "p99_latency_us",
                                                 "mean_latency_us", "cells_per_s")] + \
               [(nm, ctypes.c_uint64) for nm in ("graph_batches", "graphs_captured", "graphs_cached",
                                                 "in_flight_peak")]

    def as_dict(self):
        return {nm: getattr(self, nm) for nm, _ in self._fields_}


def lib():
    """The loaded libqss.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2405_05974_b300.build_ext`")
        L = ctypes.CDLL(LIB_PATH)
        L.qss_last_error.restype = ctypes.c_char_p
        L.qss_mech_load.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(_vp)]
        L.qss_mech_free.argtypes = [_vp]
        L.qss_mech_free.restype = None
        L.qss_mech_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
        L.qss_wdot.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
        L.qss_jacobian.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.qss_jacobian_mixed.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.qss_mech_set_frontier_bytes.argtypes = [_vp, ctypes.c_size_t]
        L.qss_jacobian_launches.argtypes = [_vp, _i64, ctypes.POINTER(_i64)]
        L.qss_mech_set_newton_bytes.argtypes = [_vp, ctypes.c_size_t]
        L.qss_debug_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
        L.qss_mech_jac_pattern.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                                           ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))]
        L.qss_jacobian_fd.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                      _vp, _vp]
        L.qss_jacobian_host.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp]
        L.qss_implicit_step.argtypes = [_vp, _i64, _i64, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int,
                                        ctypes.POINTER(NewtonOpts), _vp, _vp, _vp]
        L.qss_integrate.argtypes = [_vp, _i64, _i64, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int,
                                    ctypes.POINTER(IntegrateOpts), _vp, _vp, _vp]
        L.qss_measure_fp64_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.qss_selftest_math.argtypes = [ctypes.c_int, ctypes.c_int, _i64, _vp, _vp, _vp]
        L.qss_measure_fp64_pipe.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_double)] * 2
        L.qss_serve_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(ServeOpts),
                                       ctypes.POINTER(_vp)]
        L.qss_serve_submit.argtypes = [_vp, _vp, _i64, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                       _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]
        L.qss_serve_wait.argtypes = [_vp, ctypes.c_uint64, _i64, ctypes.POINTER(ctypes.c_int)]
        L.qss_serve_stats.argtypes = [_vp, ctypes.POINTER(ServeStats)]
        L.qss_serve_destroy.argtypes = [_vp]
        L.qss_serve_destroy.restype = None
        _lib = L
    return _lib


def check(rc):
    if rc != QSS_OK:
        raise QSSError(rc, lib().qss_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def measure_fp64_peak(device: int = 0, millis: int = 200) -> float:
    out = ctypes.c_double()
    check(lib().qss_measure_fp64_peak(device, millis, ctypes.byref(out)))
    return out.value


def measure_fp64_pipe(warps_per_sm: int, active_lanes: int = 32, dependent: bool = False,
                      device: int = 0):
    """(TFLOP/s over the active lanes, SM sub-partition cycles per warp-wide
    FMA) of the FP64 pipe probe (qss_measure_fp64_pipe)."""
    t, c = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(lib().qss_measure_fp64_pipe(device, warps_per_sm, active_lanes, int(dependent), ctypes.byref(t),
                                      ctypes.byref(c)))
    return t.value, c.value


def selftest_math(fn: int, x: torch.Tensor, device: int = 0) -> torch.Tensor:
    """Device math routine `fn` (0 table exp, 1 library exp, 2 log, 3 rcp) on x."""
    y = torch.empty_like(x)
    check(lib().qss_selftest_math(device, fn, x.numel(), _ptr(x), _ptr(y), _stream(None)))
    return y


class Mechanism:
    """A compiled mechanism loaded on one GPU."""

    def __init__(self, artefact_dir: str, device: int = 0):
        self.dir = artefact_dir
        self.device = device
        h = _vp()
        check(lib().qss_mech_load(artefact_dir.encode(), device, ctypes.byref(h)))
        self.h = h
        N, Q, M = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        W = ctypes.POINTER(ctypes.c_double)()
        check(lib().qss_mech_info(h, ctypes.byref(N), ctypes.byref(Q), ctypes.byref(M), ctypes.byref(W)))
        self.N, self.Q, self.M = N.value, Q.value, M.value
        self.W = [W[i] for i in range(self.N)]
        nnz = _i64()
        rp, ci = ctypes.POINTER(ctypes.c_int32)(), ctypes.POINTER(ctypes.c_int32)()
        check(lib().qss_mech_jac_pattern(h, ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)))
        # stored Jacobian entries per cell and their CSR pattern (dense: all)
        self.jac_nnz = nnz.value
        self.jac_row_ptr = [rp[i] for i in range(self.N + 2)]
        self.jac_col = [ci[i] for i in range(self.jac_nnz)]
        # the artefact carries the mixed-precision Jacobian kernel (jac32)
        with open(os.path.join(artefact_dir, "meta.txt")) as f:
            self.has_jac32 = any(ln.split()[:2] == ["jac32", "1"] for ln in f)

    @classmethod
    def from_dict(cls, mech: dict, device: int = 0, **build_kw):
        from .qssc.build import build_mechanism
        return cls(build_mechanism(mech, **build_kw), device)

    @property
    def n(self):
        return self.N + 1

    def close(self):
        if getattr(self, "h", None):
            lib().qss_mech_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ checks
    def _check_state(self, rho, T, Y, ncells):
        for nm, t in (("rho", rho), ("T", T), ("Y", Y)):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError(f"{nm} must be a contiguous float64 CUDA tensor")
        ld = T.shape[0]
        if rho.shape != (ld,) or Y.shape != (self.N, ld):
            raise ValueError("shape mismatch: rho[ld], T[ld], Y[N][ld]")
        nc = ld if ncells is None else int(ncells)
        return nc, ld

    def _out(self, t, shape, like):
        if t is None:
            return torch.empty(shape, dtype=torch.float64, device=like.device)
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"output must be a contiguous float64 CUDA tensor of shape {shape}")
        return t

    # -------------------------------------------------------------- calls
    def wdot(self, rho, T, Y, wdot=None, Tdot=None, ncells=None, stream=None, want_Tdot=True):
        nc, ld = self._check_state(rho, T, Y, ncells)
        wdot = self._out(wdot, (self.N, ld), T)
        if want_Tdot:
            Tdot = self._out(Tdot, (ld,), T)
        check(lib().qss_wdot(self.h, nc, ld, _ptr(rho), _ptr(T), _ptr(Y), _ptr(wdot), _ptr(Tdot),
                             _stream(stream)))
        return wdot, Tdot

    def jacobian(self, rho, T, Y, jac=None, wdot=None, Tdot=None, ncells=None, stream=None,
                 want_rates=True, mixed=False):
        """qss_jacobian, or with mixed=True qss_jacobian_mixed (derivative
        terms in FP32)."""
        nc, ld = self._check_state(rho, T, Y, ncells)
        jac = self._out(jac, (self.jac_nnz, ld), T)
        if want_rates:
            wdot = self._out(wdot, (self.N, ld), T)
            Tdot = self._out(Tdot, (ld,), T)
        fn = lib().qss_jacobian_mixed if mixed else lib().qss_jacobian
        check(fn(self.h, nc, ld, _ptr(rho), _ptr(T), _ptr(Y), _ptr(jac), _ptr(wdot), _ptr(Tdot), _stream(stream)))
        return jac, wdot, Tdot

    def jac_dense(self, jac):
        """A stored Jacobian [jac_nnz][ld] as the dense [(N+1)^2][ld] array
        (zeros off the pattern); a dense artefact's output is returned as is."""
        n = self.n
        if self.jac_nnz == n * n:
            return jac
        out = torch.zeros((n * n, jac.shape[1]), dtype=jac.dtype, device=jac.device)
        rows = [i * n + self.jac_col[p] for i in range(n) for p in range(self.jac_row_ptr[i], self.jac_row_ptr[i + 1])]
        out[torch.tensor(rows, device=jac.device)] = jac
        return out

    def jacobian_launches(self, ncells: int) -> int:
        """Kernel launches of one qss_jacobian call over ncells cells."""
        v = _i64()
        check(lib().qss_jacobian_launches(self.h, int(ncells), ctypes.byref(v)))
        return v.value

    def set_newton_bytes(self, nbytes: int):
        """Size limit of the Newton scratch of the implicit step and the
        interval integrator (default 1/16 of the device's memory)."""
        check(lib().qss_mech_set_newton_bytes(self.h, int(nbytes)))

    def debug_status(self) -> int:
        """First bounds-check code recorded by a QSS_DEBUG artefact's kernels
        since the last call (0: none); the word is cleared."""
        v = ctypes.c_int(0)
        check(lib().qss_debug_status(self.h, ctypes.byref(v)))
        return v.value

    def set_frontier_bytes(self, nbytes: int):
        """Size limit of the partitioned Jacobian's frontier buffer."""
        check(lib().qss_mech_set_frontier_bytes(self.h, int(nbytes)))

    def jacobian_fd(self, rho, T, Y, dC, dT, jac=None, ncells=None, stream=None):
        """Central finite-difference Jacobian (absolute steps dC, dT)."""
        nc, ld = self._check_state(rho, T, Y, ncells)
        jac = self._out(jac, (self.n * self.n, ld), T)
        check(lib().qss_jacobian_fd(self.h, nc, ld, _ptr(rho), _ptr(T), _ptr(Y), float(dC), float(dT),
                                    _ptr(jac), _stream(stream)))
        return jac

    def jacobian_host(self, rho, T, Y, jac=None, wdot=None, Tdot=None, chunk=0):
        """Host (CPU, ideally pinned) float64 tensors; synchronous."""
        for nm, t in (("rho", rho), ("T", T), ("Y", Y)):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous float64 host tensor")
        nc = T.shape[0]
        if jac is None:
            jac = torch.empty((self.jac_nnz, nc), dtype=torch.float64, pin_memory=True)
        check(lib().qss_jacobian_host(self.h, nc, _ptr(rho), _ptr(T), _ptr(Y), _ptr(jac), _ptr(wdot),
                                      _ptr(Tdot), chunk, None))
        return jac, wdot, Tdot

    def integrate(self, rho, T, Y, dt_total, precision=QSS_LU_FP32_IR, ncells=None, nsteps=None,
                  status=None, opts: Optional[IntegrateOpts] = None, stream=None):
        """Advance (T, Y) in place over dt_total by error-controlled
        backward-Euler substeps; returns (nsteps, status) device tensors."""
        nc, ld = self._check_state(rho, T, Y, ncells)
        if not isinstance(dt_total, torch.Tensor):
            dt_total = torch.full((1,), float(dt_total), dtype=torch.float64, device=T.device)
        stride = 1 if dt_total.numel() > 1 else 0
        if nsteps is None:
            nsteps = torch.empty(ld, dtype=torch.int32, device=T.device)
        if status is None:
            status = torch.empty(ld, dtype=torch.int32, device=T.device)
        check(lib().qss_integrate(self.h, nc, ld, _ptr(dt_total), stride, _ptr(rho), _ptr(T), _ptr(Y),
                                  precision, ctypes.byref(opts) if opts is not None else None,
                                  _ptr(nsteps), _ptr(status), _stream(stream)))
        return nsteps, status

    def implicit_step(self, rho, T, Y, dt, precision=QSS_LU_FP64, ncells=None, iters=None,
                      status=None, opts: Optional[NewtonOpts] = None, stream=None):
        """Advance (T, Y) in place by one backward-Euler step of size dt."""
        nc, ld = self._check_state(rho, T, Y, ncells)
        if not isinstance(dt, torch.Tensor):
            dt = torch.full((1,), float(dt), dtype=torch.float64, device=T.device)
        if not (dt.is_cuda and dt.dtype == torch.float64):
            raise ValueError("dt must be a float64 CUDA tensor")
        stride = 1 if dt.numel() > 1 else 0
        if stride and dt.shape[0] < ld:
            raise ValueError("dt must have ld entries or one")
        if iters is None:
            iters = torch.empty(ld, dtype=torch.int32, device=T.device)
        if status is None:
            status = torch.empty(ld, dtype=torch.int32, device=T.device)
        check(lib().qss_implicit_step(self.h, nc, ld, _ptr(dt), stride, _ptr(rho), _ptr(T), _ptr(Y),
                                      precision, ctypes.byref(opts) if opts is not None else None,
                                      _ptr(iters), _ptr(status), _stream(stream)))
        return iters, status


class Server:
    """Continuous-batching server of implicit-step requests (host arrays)."""

    def __init__(self, device: int = 0, budget_bytes: int = 8 << 30, n_streams: int = 4,
                 max_batch_cells: int = 1 << 18, newton: Optional[NewtonOpts] = None,
                 graphs: bool = True):
        """graphs: replay CUDA graphs captured per (mechanism, precision,
        size bucket) instead of launching each batch's kernels directly."""
        self._newton = newton
        o = ServeOpts(n_streams, max_batch_cells,
                      ctypes.pointer(newton) if newton is not None else None, 1 if graphs else -1)
        h = _vp()
        check(lib().qss_serve_create(device, budget_bytes, ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, mech: Mechanism, rho, T, Y, dt: float, precision=QSS_LU_FP64, iters=None,
               status=None) -> int:
        """Queue one request; rho[n], T[n], Y[N][n] are host float64 tensors
        (T, Y updated in place on completion).  Returns the request id."""
        for nm, t in (("rho", rho), ("T", T), ("Y", Y)):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous float64 host tensor")
        n = T.shape[0]
        if rho.shape != (n,) or Y.shape != (mech.N, n):
            raise ValueError("shape mismatch")
        rid = ctypes.c_uint64()
        check(lib().qss_serve_submit(self.h, mech.h, n, _ptr(rho), _ptr(T), _ptr(Y), float(dt), precision,
                                     _ptr(iters), _ptr(status), ctypes.byref(rid)))
        self._keep[rid.value] = (rho, T, Y, iters, status)
        return rid.value

    def wait(self, rid: int, timeout_us: int = -1) -> int:
        st = ctypes.c_int()
        rc = lib().qss_serve_wait(self.h, rid, timeout_us, ctypes.byref(st))
        if rc != -6:
            self._keep.pop(rid, None)
        check(rc)
        return st.value

    def stats(self) -> dict:
        s = ServeStats()
        check(lib().qss_serve_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            lib().qss_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
