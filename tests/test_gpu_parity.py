"""GPU parity of wdot, Tdot and the analytic Jacobian against the CPU oracle.

All calls go through the C ABI (libqss.so) via the ctypes binding.  Inputs are
the seeded synthetic workloads; the oracle is evaluated on the same inputs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests.parity import assert_gate, assert_gate_exact

pytestmark = pytest.mark.gpu

_mechs = {}


def mech(key):
    if key not in _mechs:
        m = workloads.mechanism(key)
        _mechs[key] = (m, binding.Mechanism(build_mechanism(m, **workloads.build_options(key)), 0), oracle.OracleMech(m))
    return _mechs[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gpu(key, rho, T, Y, ncells=None, jac=True):
    _, gm, _ = mech(key)
    r, t, y = dev(rho), dev(T), dev(Y)
    if jac:
        J, w, td = gm.jacobian(r, t, y, ncells=ncells)
    else:
        w, td = gm.wdot(r, t, y, ncells=ncells)
        J = None
    torch.cuda.synchronize()
    return (J.cpu().numpy() if J is not None else None), w.cpu().numpy(), td.cpu().numpy()


@pytest.mark.parametrize("key,ncells", [("tiny", 4096), ("hydrocarbon", 2048), ("large", 256)])
def test_jacobian_parity(key, ncells):
    m, gm, om = mech(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    J, w, td = run_gpu(key, rho, T, Y)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)

    def q128(name):
        return lambda cells: om.eval_q128(rho[cells], T[cells], np.ascontiguousarray(Y[:, cells]))[name]
    rw = assert_gate_exact("wdot", w, ref["wdot"], eb["wdot"], q128("wdot"))
    rt = assert_gate_exact("Tdot", td, ref["Tdot"], eb["Tdot"], q128("Tdot"))
    rj = assert_gate_exact("jac", J, ref["jac"], eb["jac"], q128("jac"))
    print(key, "wdot", rw, "Tdot", rt, "jac", rj)


@pytest.mark.parametrize("key,ncells", [("tiny", 4096), ("hydrocarbon", 2048)])
def test_wdot_kernel_parity(key, ncells):
    m, gm, om = mech(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    _, w, td = run_gpu(key, rho, T, Y, jac=False)
    ref = om.eval(rho, T, Y, jac=False)
    eb = om.errbound(rho, T, Y, jac=False)
    assert_gate("wdot", w, ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td, ref["Tdot"], eb["Tdot"])


def test_ragged_tail_and_padding_untouched():
    """ncells not a multiple of the block, ld > ncells: the padding columns of
    every output keep their previous contents."""
    key = "tiny"
    m, gm, om = mech(key)
    ncells, ld = 4096 - 37, 4096
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells, ld=ld)
    r, t, y = dev(rho), dev(T), dev(Y)
    n = gm.n
    J = torch.full((n * n, ld), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((gm.N, ld), 7.0, dtype=torch.float64, device="cuda")
    td = torch.full((ld,), 9.0, dtype=torch.float64, device="cuda")
    gm.jacobian(r, t, y, jac=J, wdot=w, Tdot=td, ncells=ncells)
    torch.cuda.synchronize()
    J, w, td = J.cpu().numpy(), w.cpu().numpy(), td.cpu().numpy()
    assert np.isnan(J[:, ncells:]).all()
    assert (w[:, ncells:] == 7.0).all() and (td[ncells:] == 9.0).all()
    ref = om.eval(rho, T, Y, ncells=ncells)
    eb = om.errbound(rho, T, Y, ncells=ncells)
    assert_gate("jac", J[:, :ncells], ref["jac"][:, :ncells], eb["jac"][:, :ncells])
    assert_gate("wdot", w[:, :ncells], ref["wdot"][:, :ncells], eb["wdot"][:, :ncells])


@pytest.mark.parametrize("ncells", [0, 1, 31, 129])
def test_small_and_empty_batches(ncells):
    key = "tiny"
    m, gm, om = mech(key)
    ld = max(ncells, 1)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], max(ncells, 1), ld=ld)
    J, w, td = run_gpu(key, rho, T, Y, ncells=ncells)
    if ncells == 0:
        return
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("jac", J, ref["jac"], eb["jac"])


def test_paper_sampling_protocols():
    """The paper's composition-space samples (Section 3.2.1: C ~ U[1e-4, 1];
    Appendix C: C ~ U[0.1, 1.1]; T ~ U[300, 1300] K), including low
    temperatures outside the workload ranges."""
    key = "hydrocarbon"
    m, gm, om = mech(key)
    rng = np.random.default_rng(5)
    for lo, hi in ((1e-4, 1.0), (0.1, 1.1)):
        C = rng.uniform(lo, hi, size=(gm.N, 512))
        Tt = rng.uniform(300.0, 1300.0, size=512)
        rho, T, Y = mechgen.concentrations_to_state(m, C, Tt)
        J, w, td = run_gpu(key, rho, T, Y)
        ref = om.eval(rho, T, Y)
        eb = om.errbound(rho, T, Y)
        assert_gate("wdot", w, ref["wdot"], eb["wdot"])
        assert_gate("jac", J, ref["jac"], eb["jac"])


@pytest.mark.parametrize("key", ["hydrocarbon", "large"])
def test_full_size_sampled_cells(key):
    """The workload at its full size (2^20 cells) in the benchmark's launch
    configuration (the autotuned Jacobian variant; for the large mechanism
    the partitioned Jacobian in several frontier chunks): a seeded sample of
    cells checked against the oracle."""
    from paper_2405_05974_b300 import autotune
    m, _, om = mech(key)
    nc = workloads.NCELLS[key]
    gm = binding.Mechanism(autotune.artefact(m, torch.cuda.get_device_name(0), defaults=workloads.build_options(key),
                                             ncells=nc), 0)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], nc)
    r, t, y = dev(rho), dev(T), dev(Y)
    J, w, td = gm.jacobian(r, t, y)
    idx_np = np.sort(np.random.default_rng(9).choice(nc, size=256, replace=False))
    idx = torch.from_numpy(idx_np).cuda()
    Js = J.index_select(1, idx).cpu().numpy()
    ws = w.index_select(1, idx).cpu().numpy()
    del J
    torch.cuda.empty_cache()
    rs, ts, ys = rho[idx_np], T[idx_np], np.ascontiguousarray(Y[:, idx_np])
    ref = om.eval(rs, ts, ys)
    eb = om.errbound(rs, ts, ys)

    def q128(name):
        return lambda cells: om.eval_q128(rs[cells], ts[cells], np.ascontiguousarray(ys[:, cells]))[name]
    print(key, "jac", assert_gate_exact("jac", Js, ref["jac"], eb["jac"], q128("jac")))
    print(key, "wdot", assert_gate_exact("wdot", ws, ref["wdot"], eb["wdot"], q128("wdot")))


def test_deterministic_and_host_path_identical():
    key = "hydrocarbon"
    m, gm, om = mech(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 3000)
    J1, w1, t1 = run_gpu(key, rho, T, Y)
    J2, w2, t2 = run_gpu(key, rho, T, Y)
    assert np.array_equal(J1, J2) and np.array_equal(w1, w2)
    rh = torch.from_numpy(rho).pin_memory()
    th = torch.from_numpy(T).pin_memory()
    yh = torch.from_numpy(np.ascontiguousarray(Y)).pin_memory()
    Jh = torch.empty((gm.n ** 2, 3000), dtype=torch.float64).pin_memory()
    wh = torch.empty((gm.N, 3000), dtype=torch.float64).pin_memory()
    gm.jacobian_host(rh, th, yh, jac=Jh, wdot=wh, chunk=1024)
    assert np.array_equal(Jh.numpy(), J1)
    assert np.array_equal(wh.numpy(), w1)


def test_invalid_arguments_rejected():
    key = "tiny"
    _, gm, _ = mech(key)
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    Y = torch.zeros((gm.N, 64), dtype=torch.float64, device="cuda")
    J = torch.zeros((gm.n ** 2, 64), dtype=torch.float64, device="cuda")
    lib = binding.lib()
    rc = lib.qss_jacobian(gm.h, 65, 64, x.data_ptr(), x.data_ptr(), Y.data_ptr(), J.data_ptr(),
                          None, None, None)
    assert rc == -1
    rc = lib.qss_jacobian(gm.h, 8, 64, None, x.data_ptr(), Y.data_ptr(), J.data_ptr(), None, None, None)
    assert rc == -1
    assert b"null" in lib.qss_last_error()


def _tuned_cases():
    """(workload, size bucket) of every choice the table records for this
    GPU; the bucket's cell count selects it through autotune.artefact."""
    from paper_2405_05974_b300 import autotune
    out = []
    for key in ("tiny", "hydrocarbon", "large"):
        sizes = sorted({int(n) for gpu in autotune.load_table().values() for rec in gpu.values()
                        if rec.get("name", "").startswith(workloads.mechanism(key)["name"])
                        for n in (rec.get("choice_by_size") or {})}) or [None]
        out += [(key, n) for n in sizes]
    return out


@pytest.mark.parametrize("key,bucket", _tuned_cases())
def test_tuned_variant_matches_default(key, bucket):
    """The Jacobian kernel variant the autotuner records for this GPU and
    size bucket (block size, register budget, shared-memory placement of
    values, column partition) computes the same DAG: its wdot, Tdot and J
    pass the gate against the oracle on a sample of a ragged batch larger
    than one wave, and an implicit step gives the default artefact's
    statuses and a state within the implicit step's gate (the variants may
    differ from the default build in the compiler's multiply-add
    contraction only)."""
    from paper_2405_05974_b300 import autotune
    m, gm, om = mech(key)
    art = autotune.artefact(m, torch.cuda.get_device_name(0), defaults=workloads.build_options(key), ncells=bucket)
    gt = binding.Mechanism(art, 0)
    nc = {"tiny": 40001, "hydrocarbon": 40001, "large": 9001}[key]
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], nc)
    J, w, td = gt.jacobian(dev(rho), dev(T), dev(Y))
    idx_np = np.sort(np.random.default_rng(3).choice(nc, size=256, replace=False))
    idx = torch.from_numpy(idx_np).cuda()
    rs, ts, ys = rho[idx_np], T[idx_np], np.ascontiguousarray(Y[:, idx_np])
    ref, eb = om.eval(rs, ts, ys), om.errbound(rs, ts, ys)
    assert_gate("jac", J.index_select(1, idx).cpu().numpy(), ref["jac"], eb["jac"])
    assert_gate("wdot", w.index_select(1, idx).cpu().numpy(), ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td.index_select(0, idx).cpu().numpy(), ref["Tdot"], eb["Tdot"])
    del J
    res = []
    for g in (gm, gt):
        t, y = dev(T), dev(Y)
        it, st = g.implicit_step(dev(rho), t, y, 1e-9, precision=binding.QSS_LU_FP32_IR)
        torch.cuda.synchronize()
        res.append((t.cpu().numpy(), y.cpu().numpy(), st.cpu().numpy()))
    (t0, y0, s0), (t1, y1, s1) = res
    assert np.mean(s0 == s1) >= 0.999
    both = (s0 == 0) & (s1 == 0)
    W = np.array(gm.W)[:, None]
    p0 = np.vstack([rho[None] * y0 / W, t0[None]])[:, both]
    p1 = np.vstack([rho[None] * y1 / W, t1[None]])[:, both]
    atol = np.r_[np.full(gm.N, 1e-20), 1e-10][:, None]
    assert np.all(np.abs(p1 - p0) <= 1e-10 * np.abs(p0) + 10 * atol)
