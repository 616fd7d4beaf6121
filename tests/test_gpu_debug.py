"""QSS_DEBUG artefacts: the kernels check every index they form before the
access and report a violation in a device status word instead of trapping.

* A debug build computes bit for bit what the release build computes (the
  checks only guard accesses) and reports nothing on valid calls, including
  ragged and tiny batches (1..4093 cells, ld > ncells), the partitioned
  Jacobian and both implicit-step forms.
* A check fires: the debug Jacobian kernel launched directly with
  ld < ncells (the library's host checks reject that, so the test loads the
  kernel itself) records code 3 for the cells beyond ld.  Every array is
  sized for ncells rows, so no access could leave its buffer even without
  the check.
"""
import ctypes
import json
import os

import numpy as np
import pytest
import torch

from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism, cubin_file

pytestmark = pytest.mark.gpu

DEBUG = ("QSS_DEBUG=1",)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("parts", [0, 2])
def test_debug_build_matches_release_and_reports_nothing(parts):
    m = workloads.mechanism("tiny")
    rel = binding.Mechanism(build_mechanism(m, jac_parts=parts), 0)
    dbg = binding.Mechanism(build_mechanism(m, defines=DEBUG, jac_parts=parts), 0)
    with pytest.raises(binding.QSSError) as e:
        rel.debug_status()
    assert e.value.code == -8
    assert dbg.debug_status() == 0
    for ncells, ld in ((1, 1), (31, 37), (64, 64), (129, 160), (4093, 4096)):
        rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], ncells, ld=ld)
        r, t, y = dev(rho), dev(T), dev(Y)
        outs = []
        for gm in (rel, dbg):
            J, w, td = gm.jacobian(r, t, y, ncells=ncells)
            w2, td2 = gm.wdot(r, t, y, ncells=ncells)
            torch.cuda.synchronize()
            outs.append([x.cpu().numpy()[..., :ncells] for x in (J, w, td, w2, td2)])
        for a, b in zip(*outs):
            assert np.array_equal(a, b, equal_nan=True)
        assert dbg.debug_status() == 0
        for prec in (binding.QSS_LU_FP64, binding.QSS_LU_FP32_IR):
            res = []
            for gm in (rel, dbg):
                tt, yy = dev(T), dev(Y)
                it, st = gm.implicit_step(r, tt, yy, 1e-7, precision=prec, ncells=ncells)
                torch.cuda.synchronize()
                res.append((tt.cpu().numpy(), yy.cpu().numpy(), it.cpu().numpy()[:ncells], st.cpu().numpy()[:ncells]))
            for a, b in zip(*res):
                assert np.array_equal(a, b, equal_nan=True)
            assert dbg.debug_status() == 0


def _cuda():
    L = ctypes.CDLL("libcuda.so.1")
    for nm, args in (("cuModuleLoad", [ctypes.c_void_p, ctypes.c_char_p]),
                     ("cuModuleGetFunction", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p]),
                     ("cuModuleGetGlobal_v2", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p]),
                     ("cuLaunchKernel", [ctypes.c_void_p] + [ctypes.c_uint] * 6 + [ctypes.c_uint, ctypes.c_void_p,
                                                                                     ctypes.c_void_p, ctypes.c_void_p]),
                     ("cuCtxSynchronize", []), ("cuModuleUnload", [ctypes.c_void_p]),
                     ("cuMemcpyDtoH_v2", [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t])):
        getattr(L, nm).argtypes = args
        getattr(L, nm).restype = ctypes.c_int
    return L


def test_debug_check_reports_cell_beyond_ld():
    m = workloads.mechanism("tiny")
    art = build_mechanism(m, defines=DEBUG)
    gm = binding.Mechanism(art, 0)       # initialises the device's primary context
    torch.cuda.synchronize()
    ncells, ld = 256, 200                # threads 200..255 must stop at the check
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], ncells)
    r, t, y = dev(rho), dev(T), dev(Y)   # Y holds N x 256 >= N x 200 entries
    J = torch.zeros((gm.jac_nnz, ncells), dtype=torch.float64, device="cuda")
    w = torch.zeros((gm.N, ncells), dtype=torch.float64, device="cuda")
    td = torch.zeros(ncells, dtype=torch.float64, device="cuda")
    L = _cuda()
    mod, fn = ctypes.c_void_p(), ctypes.c_void_p()
    assert L.cuModuleLoad(ctypes.byref(mod), cubin_file(art, "jac.cubin").encode()) == 0
    try:
        assert L.cuModuleGetFunction(ctypes.byref(fn), mod, b"qss_jac_kernel") == 0
        word, nbytes = ctypes.c_uint64(), ctypes.c_size_t()
        assert L.cuModuleGetGlobal_v2(ctypes.byref(word), ctypes.byref(nbytes), mod, b"qss_debug_word") == 0
        vals = [ctypes.c_longlong(ncells), ctypes.c_longlong(ld)] + \
            [ctypes.c_void_p(x.data_ptr()) for x in (r, t, y, J, w, td)] + [ctypes.c_void_p(0)] * 4
        args = (ctypes.c_void_p * len(vals))(*[ctypes.cast(ctypes.byref(v), ctypes.c_void_p) for v in vals])
        block = int(json.load(open(os.path.join(art, "meta.json")))["block"])
        assert L.cuLaunchKernel(fn, (ncells + block - 1) // block, 1, 1, block, 1, 1, 0, None, args, None) == 0
        assert L.cuCtxSynchronize() == 0
        code = ctypes.c_int(0)
        assert L.cuMemcpyDtoH_v2(ctypes.byref(code), word.value, 4) == 0
        assert code.value == 3
        # the launch writes entry e of cell c < ld at flat position e * ld + c:
        # that region was computed, everything after it is untouched
        Jf = J.view(-1).cpu().numpy()
        assert np.all(Jf[gm.jac_nnz * ld:] == 0.0) and np.count_nonzero(Jf[:gm.jac_nnz * ld]) > ld
    finally:
        L.cuModuleUnload(mod)
