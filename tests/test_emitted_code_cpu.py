"""The mechanism compiler's generated code, compiled as plain C++ on the CPU,
against the oracle (no GPU).

The CUDA kernels inline the generated straight-line body (qss_eval_jac).  Here
the same generated source is compiled with g++ (fma, exp, log and 1/x from the
C++ library in place of the device's table-driven functions) and evaluated on
seeded workload states, so that build options that change only the emitted
code -- Alg. 2's common-subexpression replacement (replace_nop, Sec. 4.1),
the emission order (Alg. 3's recycling on or off) and the placement of the
most-reloaded values in shared memory (smem_slots) -- are checked for
correctness without a GPU, through the same parity gate as the GPU tests
(the hydrocarbon variants too, whose CUDA builds take up to 1.5 hours to
compile and are only timed on the GPU, by the benchmark's memory study).
The two emission orders must also emit the same statements, only reordered.
"""
import collections
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2405_05974_b300 import mechgen, workloads
from paper_2405_05974_b300.qssc import emit
from paper_2405_05974_b300.qssc import mech as qmech
from paper_2405_05974_b300.qssc import model as qmodel
from tests.parity import assert_gate

_SHIM = r"""
#include <cmath>
#define __device__
#define __forceinline__ inline
#define __constant__ static const
#define __restrict__ __restrict
#define __shared__
#define QSS_BLOCK 1
static struct { unsigned x; } threadIdx = {0};
double qss_smem_dyn[16384];
static inline double qss_exp(double x) { return std::exp(x); }
static inline double qss_log(double x) { return std::log(x); }
static inline double qss_rcp(double x) { return 1.0 / x; }
using std::fma;
"""

_DRIVER = r"""
extern "C" void eval_cells(long long n, const double* C, const double* T, double* wdot, double* Tdot,
                           double* jac) {
  for (long long c = 0; c < n; ++c) {
    double Cc[QSS_N];
    for (int k = 0; k < QSS_N; ++k) Cc[k] = C[k * n + c];
    qss_eval_jac(Cc, T[c], wdot + c, Tdot + c, jac + c, n, n);
  }
}
"""

_models = {}


def _model(key):
    if key not in _models:
        _models[key] = qmodel.build_model(qmech.parse(workloads.mechanism(key)))
    return _models[key]


def _compile(src):
    d = tempfile.mkdtemp(prefix="qss_emit_")
    iw = src.index("__device__ __forceinline__ void qss_eval_wdot")
    ij = src.index("__device__ __forceinline__ void qss_eval_jac")
    cpp = os.path.join(d, "gen.cpp")
    with open(cpp, "w") as f:
        f.write(_SHIM + src[:iw] + src[ij:] + _DRIVER)
    so = os.path.join(d, "gen.so")
    subprocess.check_call(["g++", "-O0", "-shared", "-fPIC", "-ffp-contract=off", "-o", so, cpp])
    L = ctypes.CDLL(so)
    p = ctypes.POINTER(ctypes.c_double)
    L.eval_cells.argtypes = [ctypes.c_longlong, p, p, p, p, p]
    return L


def _run(L, C, T, n_out):
    n = T.shape[0]
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    C = np.ascontiguousarray(C)
    T = np.ascontiguousarray(T)
    w = np.zeros((C.shape[0], n))
    td = np.zeros(n)
    J = np.zeros((n_out, n))
    L.eval_cells(n, p(C), p(T), p(w), p(td), p(J))
    return w, td, J


@pytest.mark.parametrize("key,opts", [("tiny", {}), ("tiny", {"replace_nop": 10}),
                                      ("tiny", {"replace_nop": 20}), ("tiny", {"emit_order": "all_first"}),
                                      ("tiny", {"smem_slots": 24}), ("hydrocarbon", {}),
                                      ("hydrocarbon", {"replace_nop": 10}), ("hydrocarbon", {"replace_nop": 20}),
                                      ("hydrocarbon", {"emit_order": "all_first"}),
                                      ("hydrocarbon", {"smem_slots": 100})])
def test_generated_code_matches_oracle(key, opts):
    model = _model(key)
    src, meta = emit.emit_mechanism_source(model, **opts)
    L = _compile(src)
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 256)
    om = oracle.OracleMech(m)
    C = om.conc(rho, Y)
    n = meta["N"] + 1
    w, td, J = _run(L, C, T, n * n)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])
    assert_gate("jac", J, ref["jac"], eb["jac"])
    if opts.get("replace_nop"):
        # Alg. 2 trades stored values for recomputation: fewer stored
        # subexpressions, more operations in the emitted code
        base = emit.emit_mechanism_source(model)[1]
        assert meta["ops_jac"]["fma"] + meta["ops_jac"].get("mul", 0) > \
            base["ops_jac"]["fma"] + base["ops_jac"].get("mul", 0)
        assert meta["flops_jac"] == base["flops_jac"]


@pytest.mark.parametrize("key", ["tiny", "hydrocarbon"])
def test_emission_orders_emit_the_same_statements(key):
    """Alg. 3 on/off changes only the order: the same value definitions and
    the same stores; with recycling off every store follows every value."""
    model = _model(key)
    a = emit.emit_mechanism_source(model)[0]
    b = emit.emit_mechanism_source(model, emit_order="all_first")[0]

    def body(src):
        ij = src.index("__device__ __forceinline__ void qss_eval_jac")
        return [ln.strip() for ln in src[ij:].splitlines() if ln.strip().startswith(("const double t", "jac[",
                                                                                     "if (wdot)", "if (Tdot)"))]
    la, lb = body(a), body(b)
    assert collections.Counter(la) == collections.Counter(lb)
    first_store = min(i for i, ln in enumerate(lb) if not ln.startswith("const double t"))
    assert all(not ln.startswith("const double t") for ln in lb[first_store:])
    assert la != lb


_SHIM32 = r"""
#include <math.h>
float qss_smem32_dyn[65536];
#include "qss_convert.h"
static inline float __frcp_rn(float x) { return 1.0f / x; }
using std::fmaf;
"""

_DRIVER32 = _DRIVER.replace("qss_eval_jac(", "qss_eval_jac32(")


@pytest.mark.parametrize("key,slots", [("tiny", 0), ("hydrocarbon", 0), ("hydrocarbon", 200)])
def test_mixed_precision_jacobian_within_fp32_bound(key, slots):
    """The mixed-precision Jacobian (derivative terms in FP32, the source
    term in FP64), compiled on the CPU with the kernels' own bit-pattern
    conversions: wdot and Tdot pass the FP64 gate, and every Jacobian entry
    is within 2^29 (= u_32 / u_64) times the oracle's FP64 running-error
    bound (plus the 1e-20 floor), i.e. within the first-order rounding
    bound of the same evaluation carried out entirely in FP32; also with
    FP32 values placed in (emulated) shared memory."""
    from paper_2405_05974_b300.qssc.build import CSRC
    model = _model(key)
    src, meta = emit.emit_mechanism_source(model)
    s32, m32 = emit.emit_jac32_source(model, smem_slots=slots)
    assert m32["jac32_slots"] == slots   # (the hydrocarbon body reloads far more than 200 values)
    iw = src.index("__device__ __forceinline__ void qss_eval_wdot")
    d = tempfile.mkdtemp(prefix="qss_emit32_")
    cpp = os.path.join(d, "gen.cpp")
    with open(cpp, "w") as f:
        f.write(_SHIM + _SHIM32 + src[:iw] + s32 + _DRIVER32)
    so = os.path.join(d, "gen.so")
    subprocess.check_call(["g++", "-O0", "-shared", "-fPIC", "-ffp-contract=off", "-I", CSRC, "-o", so, cpp])
    L = ctypes.CDLL(so)
    p = ctypes.POINTER(ctypes.c_double)
    L.eval_cells.argtypes = [ctypes.c_longlong, p, p, p, p, p]
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 256)
    om = oracle.OracleMech(m)
    n = meta["N"] + 1
    w, td, J = _run(L, om.conc(rho, Y), T, n * n)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])
    err = np.abs(J - ref["jac"])
    assert np.all(np.isfinite(J))
    assert np.all(err <= 2.0 ** 29 * eb["jac"] + 1e-20), float(np.max(err / (2.0 ** 29 * eb["jac"] + 1e-20)))
    # the FP64 part is the source term's: the same FP64 operation count
    assert m32["fp64_instr_jac32"] == meta["fp64_instr_wdot"]
    assert m32["flops_jac32"] == meta["flops_jac"]


@pytest.mark.parametrize("key,K", [("tiny", 2), ("hydrocarbon", 4)])
def test_partitioned_mixed_precision_jacobian_within_fp32_bound(key, K):
    """The partitioned form of the mixed-precision Jacobian (prefix kernel in
    FP64 for the source term and FP32 for its shared derivative values, the
    column groups in FP32 from the narrowed frontier), compiled on the CPU:
    the same FP32 bound as the single function, and the same source term."""
    from paper_2405_05974_b300.qssc.build import CSRC
    model = _model(key)
    src, meta = emit.emit_mechanism_source(model)
    prefix, groups, pmeta = emit.emit_partitioned_source(model, K, mixed=True)
    n = meta["N"] + 1
    nfr = pmeta["frontier"]
    iw = src.index("__device__ __forceinline__ void qss_eval_wdot")
    body = src[:iw] + prefix + "".join(f"namespace g{i} {{\n{g}}}\n" for i, g in enumerate(groups))
    calls = "".join(f"    g{i}::qss_jac_group(fr, 1, jac + c, n);\n" for i in range(K))
    drv = ("extern \"C\" void eval_cells(long long n, const double* C, const double* T, double* wdot,"
           " double* Tdot, double* jac) {\n"
           f"  static double fr[{nfr}];\n"
           "  for (long long c = 0; c < n; ++c) {\n"
           "    double Cc[QSS_N];\n"
           "    for (int k = 0; k < QSS_N; ++k) Cc[k] = C[k * n + c];\n"
           "    qss_jac_prefix(Cc, T[c], wdot + c, Tdot + c, n, fr, 1);\n" + calls + "  }\n}\n")
    d = tempfile.mkdtemp(prefix="qss_emitp32_")
    cpp = os.path.join(d, "gen.cpp")
    with open(cpp, "w") as f:
        f.write(_SHIM + _SHIM32 + body + drv)
    so = os.path.join(d, "gen.so")
    subprocess.check_call(["g++", "-O0", "-shared", "-fPIC", "-ffp-contract=off", "-I", CSRC, "-o", so, cpp])
    L = ctypes.CDLL(so)
    p = ctypes.POINTER(ctypes.c_double)
    L.eval_cells.argtypes = [ctypes.c_longlong, p, p, p, p, p]
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 128)
    om = oracle.OracleMech(m)
    w, td, J = _run(L, om.conc(rho, Y), T, n * n)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])
    err = np.abs(J - ref["jac"])
    assert np.all(np.isfinite(J))
    assert np.all(err <= 2.0 ** 29 * eb["jac"] + 1e-20), float(np.max(err / (2.0 ** 29 * eb["jac"] + 1e-20)))


@pytest.mark.parametrize("key,K,slots", [("tiny", 2, 16), ("hydrocarbon", 4, 60)])
def test_partitioned_jacobian_with_shared_memory_values(key, K, slots):
    """The FP64 partitioned Jacobian with its most-reloaded values kept in
    shared memory (smem_slots in the prefix and in every column group),
    compiled on the CPU: the same gate against the oracle as the GPU tests.
    A kernel whose values all fit the simulated register file gets no slots
    (the tiny mechanism's column groups)."""
    model = _model(key)
    src, meta = emit.emit_mechanism_source(model)
    prefix, groups, pmeta = emit.emit_partitioned_source(model, K, smem_slots=slots)
    assert len(pmeta["smem_slots_parts"]) == K + 1
    assert all(0 <= u <= slots for u in pmeta["smem_slots_parts"]) and pmeta["smem_slots_parts"][0] > 0
    for u, s_ in zip(pmeta["smem_slots_parts"], [prefix] + groups):
        assert ("qss_sm[" in s_) == (u > 0)
    n = meta["N"] + 1
    nfr = pmeta["frontier"]
    iw = src.index("__device__ __forceinline__ void qss_eval_wdot")
    # each group is its own kernel (its own dynamic shared memory): one array
    # per namespace here
    body = src[:iw] + prefix + "".join(f"namespace g{i} {{\ndouble qss_smem_dyn[16384];\n{g}}}\n"
                                       for i, g in enumerate(groups))
    calls = "".join(f"    g{i}::qss_jac_group(fr, 1, jac + c, n);\n" for i in range(K))
    drv = ("extern \"C\" void eval_cells(long long n, const double* C, const double* T, double* wdot,"
           " double* Tdot, double* jac) {\n"
           f"  static double fr[{nfr}];\n"
           "  for (long long c = 0; c < n; ++c) {\n"
           "    double Cc[QSS_N];\n"
           "    for (int k = 0; k < QSS_N; ++k) Cc[k] = C[k * n + c];\n"
           "    qss_jac_prefix(Cc, T[c], wdot + c, Tdot + c, n, fr, 1);\n" + calls + "  }\n}\n")
    d = tempfile.mkdtemp(prefix="qss_emitps_")
    cpp = os.path.join(d, "gen.cpp")
    with open(cpp, "w") as f:
        f.write(_SHIM + body + drv)
    so = os.path.join(d, "gen.so")
    subprocess.check_call(["g++", "-O0", "-shared", "-fPIC", "-ffp-contract=off", "-o", so, cpp])
    L = ctypes.CDLL(so)
    p = ctypes.POINTER(ctypes.c_double)
    L.eval_cells.argtypes = [ctypes.c_longlong, p, p, p, p, p]
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 128)
    om = oracle.OracleMech(m)
    w, td, J = _run(L, om.conc(rho, Y), T, n * n)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])
    assert_gate("jac", J, ref["jac"], eb["jac"])


_DRIVER2 = r"""
extern "C" void eval_cells2(long long n, const double* C, const double* T, double* wdot, double* Tdot,
                            double* jac) {
  // cells c and c + h per call (the kernel's two-cells-per-thread form); an
  // odd last cell is computed twice, its copy's Jacobian stores skipped
  const long long h = (n + 1) / 2;
  for (long long c = 0; c < h; ++c) {
    const long long d = c + h < n ? c + h : c;
    double Ca[QSS_N], Cb[QSS_N];
    for (int k = 0; k < QSS_N; ++k) { Ca[k] = C[k * n + c]; Cb[k] = C[k * n + d]; }
    qss_eval_jac2(Ca, T[c], wdot + c, Tdot + c, jac + c, Cb, T[d], wdot + d, Tdot + d,
                  d != c ? jac + d : nullptr, n, n);
  }
}
"""


@pytest.mark.parametrize("key,ncells", [("tiny", 255), ("hydrocarbon", 129)])
def test_two_cells_per_thread_body_matches_oracle(key, ncells):
    """The two-cells-per-thread Jacobian body (cells_per_thread = 2: the
    one-cell body and its renamed copy interleaved), compiled on the CPU for
    an odd number of cells (the last one evaluated as both cells with the
    second copy's Jacobian stores skipped): the oracle's gate for every cell,
    and bit for bit the one-cell body's results (the same operations)."""
    model = _model(key)
    src1, meta = emit.emit_mechanism_source(model)
    src, meta2 = emit.emit_mechanism_source(model, cells_per_thread=2)
    assert meta2["cells_per_thread"] == 2 and "qss_eval_jac2" in src
    iw = src.index("__device__ __forceinline__ void qss_eval_wdot")
    ij = src.index("__device__ __forceinline__ void qss_eval_jac")
    d = tempfile.mkdtemp(prefix="qss_emit2_")
    cpp = os.path.join(d, "gen.cpp")
    with open(cpp, "w") as f:
        f.write(_SHIM + src[:iw] + src[ij:] + _DRIVER2)
    so = os.path.join(d, "gen.so")
    subprocess.check_call(["g++", "-O0", "-shared", "-fPIC", "-ffp-contract=off", "-o", so, cpp])
    L = ctypes.CDLL(so)
    p = ctypes.POINTER(ctypes.c_double)
    L.eval_cells2.argtypes = [ctypes.c_longlong, p, p, p, p, p]
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    om = oracle.OracleMech(m)
    C = np.ascontiguousarray(om.conc(rho, Y))
    T = np.ascontiguousarray(T)
    n = meta["N"] + 1
    w = np.zeros((meta["N"], ncells))
    td = np.zeros(ncells)
    J = np.zeros((n * n, ncells))
    q = lambda a: a.ctypes.data_as(p)  # noqa: E731
    L.eval_cells2(ncells, q(C), q(T), q(w), q(td), q(J))
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])
    assert_gate("jac", J, ref["jac"], eb["jac"])
    w1, td1, J1 = _run(_compile(src1), C, T, n * n)
    assert np.array_equal(J, J1) and np.array_equal(w, w1) and np.array_equal(td, td1)
