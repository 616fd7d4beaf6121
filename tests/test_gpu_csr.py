"""Artefacts that store only the structural nonzeros of the Jacobian (CSR
order, qss_mech_jac_pattern) on the GPU.

The generated code is the dense artefact's with the stores of identically
zero entries dropped and the others renumbered, so every stored value must be
bit-identical to the dense artefact's entry at the same (row, column), and
the dense artefact must hold exact zeros off the pattern; the implicit step
(which scatters the CSR values into the dense Newton matrix) must be
bit-identical too.  The oracle gate is applied to the densified output.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests.parity import assert_gate

pytestmark = pytest.mark.gpu
_cache = {}


def gpu_mech(key, fmt="dense", parts=0):
    k = (key, fmt, parts)
    if k not in _cache:
        # the dense single-kernel form: the workload's own artefact (its FP64
        # kernels are those of the plain build)
        kw = {"jac_format": fmt, "jac_parts": parts} if (fmt, parts) != ("dense", 0) else workloads.build_options(key)
        _cache[k] = binding.Mechanism(build_mechanism(workloads.mechanism(key), **kw), 0)
    return _cache[k]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dense_rows(gm):
    n = gm.n
    return np.array([i * n + gm.jac_col[p] for i in range(n)
                     for p in range(gm.jac_row_ptr[i], gm.jac_row_ptr[i + 1])])


@pytest.mark.parametrize("key,parts,ncells", [("tiny", 0, 3001), ("tiny", 2, 3001), ("hydrocarbon", 0, 2047)])
def test_csr_values_equal_dense(key, parts, ncells):
    m = workloads.mechanism(key)
    gd, gc = gpu_mech(key, "dense", parts), gpu_mech(key, "csr", parts)   # same kernels but the stores
    n = gd.n
    assert gd.jac_nnz == n * n and gc.jac_nnz < n * n
    assert len(gc.jac_row_ptr) == n + 1 and gc.jac_row_ptr[-1] == gc.jac_nnz
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    r, t, y = dev(rho), dev(T), dev(Y)
    Jd, wd, tdd = gd.jacobian(r, t, y)
    Jc, wc, tdc = gc.jacobian(r, t, y)
    Jd, Jc = Jd.cpu().numpy(), Jc.cpu().numpy()
    rows = dense_rows(gc)
    assert Jc.shape == (gc.jac_nnz, ncells)
    assert np.array_equal(Jc, Jd[rows])
    off = np.setdiff1d(np.arange(n * n), rows)
    assert np.all(Jd[off] == 0.0)
    assert torch.equal(wd, wc) and torch.equal(tdd, tdc)
    om = oracle.OracleMech(m)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("jac", gc.jac_dense(torch.from_numpy(Jc)).numpy(), ref["jac"], eb["jac"])


def test_csr_host_path():
    key, ncells = "hydrocarbon", 5000
    m = workloads.mechanism(key)
    gc = gpu_mech(key, "csr")
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    Jh, _, _ = gc.jacobian_host(torch.from_numpy(rho), torch.from_numpy(T), torch.from_numpy(Y), chunk=1024)
    Jd, _, _ = gc.jacobian(dev(rho), dev(T), dev(Y))
    assert Jh.shape == (gc.jac_nnz, ncells)
    assert torch.equal(Jh, Jd.cpu())


@pytest.mark.parametrize("key,parts,ncells", [("tiny", 0, 2048), ("tiny", 2, 2048), ("hydrocarbon", 0, 1024)])
def test_csr_implicit_step_equals_dense(key, parts, ncells):
    m = workloads.mechanism(key)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells)
    for prec in (binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR):
        out = []
        for fmt in ("dense", "csr"):
            gm = gpu_mech(key, fmt, parts)
            r, t, y = dev(rho), dev(T), dev(Y)
            it, st = gm.implicit_step(r, t, y, workloads.IMPLICIT_DT, precision=prec)
            torch.cuda.synchronize()
            out.append((t.cpu().numpy(), y.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()))
        (t0, y0, i0, s0), (t1, y1, i1, s1) = out
        assert np.array_equal(s0, s1) and np.array_equal(i0, i1)
        ok = s0 == 0
        assert ok.sum() > 0.25 * ncells
        assert np.array_equal(t0[ok], t1[ok]) and np.array_equal(y0[:, ok], y1[:, ok])
