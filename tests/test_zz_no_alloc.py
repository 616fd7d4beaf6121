"""The allocation-free implicit step against the regular one.

qss_implicit_step_noalloc exists for callers that cannot let the library
allocate device memory (applications that manage all of the GPU's memory
themselves, or loops that must not pay an allocation's synchronisation): its
Newton scratch is a fixed array in the library's device memory.  It runs the
same kernels on the same per-cell arithmetic as qss_implicit_step, so on the
same inputs the two must agree (within the implicit-step gate of the other
tests; in practice bit for bit).  Two calls in a row check that the shared
array's leftover contents from one call do not leak into the next.

This file is collected last on purpose (a failure here should not stop a
first-failure run before every other test has run).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism

pytestmark = pytest.mark.gpu


def _close(a, b, N):
    """Within the implicit-step gate; cells that ended non-finite (inf or NaN)
    must end the same way in both results."""
    atol = np.r_[np.full(N, 1e-20), 1e-10][:, None]
    same = (a == b) | (np.isnan(a) & np.isnan(b))
    with np.errstate(invalid="ignore"):
        return same | (np.abs(a - b) <= 1e-10 * np.abs(b) + 10 * atol)


def _call(fn, gm, rho, T, Y, dt, prec, ncells, ld):
    t = torch.from_numpy(T.copy()).cuda()
    y = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    it = torch.zeros(ld, dtype=torch.int32, device="cuda")
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    rc = fn(gm.h, ncells, ld, ctypes.c_void_p(dt.data_ptr()), 0, ctypes.c_void_p(rho.data_ptr()),
            ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(y.data_ptr()), prec, None,
            ctypes.c_void_p(it.data_ptr()), ctypes.c_void_p(st.data_ptr()), None)
    torch.cuda.synchronize()
    binding.check(rc)
    return t.cpu().numpy(), y.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("prec", [binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR])
def test_noalloc_matches_regular_two_calls(prec):
    L = binding.lib()
    L.qss_implicit_step_noalloc.argtypes = L.qss_implicit_step.argtypes
    m = workloads.mechanism("tiny")
    gm = binding.Mechanism(build_mechanism(m), 0)
    for call, seed in enumerate((21, 22)):      # two calls in a row, different inputs
        ncells = 5000 + 37 * call
        cfg = workloads.STATES["tiny"]
        cfg = type(cfg)(**{**cfg.__dict__, "seed": seed})
        rho, T, Y = mechgen.generate_states(m, cfg, ncells)
        r = torch.from_numpy(rho).cuda()
        dt = torch.full((1,), 1e-6, dtype=torch.float64, device="cuda")
        ref = _call(L.qss_implicit_step, gm, r, T, Y, dt, prec, ncells, ncells)
        got = _call(L.qss_implicit_step_noalloc, gm, r, T, Y, dt, prec, ncells, ncells)
        assert np.array_equal(got[3], ref[3]) and np.array_equal(got[2], ref[2])
        phi_ref = np.vstack([ref[1], ref[0][None]])
        phi_got = np.vstack([got[1], got[0][None]])
        assert _close(phi_got, phi_ref, gm.N).all()


def test_noalloc_chunks_and_arguments():
    """A batch several times larger than what the fixed array holds at once
    (processed in chunks) and an argument error."""
    L = binding.lib()
    L.qss_implicit_step_noalloc.argtypes = L.qss_implicit_step.argtypes
    m = workloads.mechanism("tiny")
    gm = binding.Mechanism(build_mechanism(m), 0)
    # tiny: 10*10 + 3*10 doubles + 5 ints = 1060 bytes per cell: ~63k cells a chunk
    ncells = 400000
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], ncells)
    r = torch.from_numpy(rho).cuda()
    dt = torch.full((1,), 1e-6, dtype=torch.float64, device="cuda")
    ref = _call(L.qss_implicit_step, gm, r, T, Y, dt, binding.QSS_LU_FP64, ncells, ncells)
    got = _call(L.qss_implicit_step_noalloc, gm, r, T, Y, dt, binding.QSS_LU_FP64, ncells, ncells)
    assert np.array_equal(got[3], ref[3])
    assert _close(np.vstack([got[1], got[0][None]]), np.vstack([ref[1], ref[0][None]]), gm.N).all()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    Yz = torch.zeros((gm.N, 8), dtype=torch.float64, device="cuda")
    rc = L.qss_implicit_step_noalloc(gm.h, 9, 8, ctypes.c_void_p(x.data_ptr()), 0, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(Yz.data_ptr()), 0, None,
                                     None, None, None)
    assert rc == -1


def test_noalloc_partitioned_mechanism_in_chunks():
    """The large mechanism's partitioned Jacobian keeps its frontier inside the
    same fixed array (after the Newton counters): about 61 KB per cell, so
    3000 cells run in three chunks of 1088 cells, a per-cell size that does
    not divide the array evenly.  Status, iterations and the new state match
    the regular entry point's."""
    L = binding.lib()
    L.qss_implicit_step_noalloc.argtypes = L.qss_implicit_step.argtypes
    m = workloads.mechanism("large")
    gm = binding.Mechanism(build_mechanism(m, **workloads.build_options("large")), 0)
    ncells = 3000
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["large"], ncells)
    r = torch.from_numpy(rho).cuda()
    dt = torch.full((1,), 1e-9, dtype=torch.float64, device="cuda")
    for prec in (binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR):
        ref = _call(L.qss_implicit_step, gm, r, T, Y, dt, prec, ncells, ncells)
        got = _call(L.qss_implicit_step_noalloc, gm, r, T, Y, dt, prec, ncells, ncells)
        assert (ref[3] == 0).mean() > 0.5
        assert np.array_equal(got[3], ref[3]) and np.array_equal(got[2], ref[2])
        assert _close(np.vstack([got[1], got[0][None]]), np.vstack([ref[1], ref[0][None]]), gm.N).all()
