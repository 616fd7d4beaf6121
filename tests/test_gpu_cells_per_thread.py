"""The FP64 Jacobian kernel with two cells per thread (build option
cells_per_thread = 2, an autotuner candidate) on the GPU: a ragged batch
(odd cell count, so the last thread's second cell lies beyond the batch) with
ld > ncells against the oracle under the parity gate, the padding beyond the
batch untouched, and an implicit step (list mode: the Jacobian kernel reads
the active list two cells per thread) giving the default artefact's statuses
and states within the implicit step's gate.  (The hydrocarbon form passed the
same test when it was timed; the tiny one is kept in the suite because it
compiles in seconds.)"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests.parity import assert_gate

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("key,ncells", [("tiny", 4093)])
def test_two_cells_per_thread(key, ncells):
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    g2 = binding.Mechanism(build_mechanism(m, cells_per_thread=2), 0)
    g1 = binding.Mechanism(build_mechanism(m, **workloads.build_options(key)), 0)
    ld = ncells + 35
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], ncells, ld=ld)
    J = torch.full((g2.jac_nnz, ld), 7.0, dtype=torch.float64, device="cuda")
    w = torch.full((g2.N, ld), 7.0, dtype=torch.float64, device="cuda")
    td = torch.full((ld,), 7.0, dtype=torch.float64, device="cuda")
    g2.jacobian(dev(rho), dev(T), dev(Y), ncells=ncells, jac=J, wdot=w, Tdot=td)
    torch.cuda.synchronize()
    assert bool((J[:, ncells:] == 7.0).all() and (w[:, ncells:] == 7.0).all() and (td[ncells:] == 7.0).all())
    ref = om.eval(rho, T, Y, ncells=ncells)
    eb = om.errbound(rho, T, Y, ncells=ncells)
    assert_gate("jac", J.cpu().numpy()[:, :ncells], ref["jac"][..., :ncells], eb["jac"][..., :ncells])
    assert_gate("wdot", w.cpu().numpy()[:, :ncells], ref["wdot"][..., :ncells], eb["wdot"][..., :ncells])
    assert_gate("Tdot", td.cpu().numpy()[:ncells], ref["Tdot"][..., :ncells], eb["Tdot"][..., :ncells])
    res = []
    for g in (g1, g2):
        t, y = dev(T), dev(Y)
        it, st = g.implicit_step(dev(rho), t, y, 1e-9, precision=binding.QSS_LU_FP64, ncells=ncells)
        torch.cuda.synchronize()
        res.append((t.cpu().numpy()[:ncells], y.cpu().numpy()[:, :ncells], st.cpu().numpy()[:ncells]))
    (T1, Y1, s1), (T2, Y2, s2) = res
    assert np.array_equal(s1, s2)
    ok = s1 == 0
    assert ok.mean() > 0.5
    W = np.array(g1.W)[:, None]
    p1 = np.vstack([rho[None, :ncells] * Y1 / W, T1[None]])[:, ok]
    p2 = np.vstack([rho[None, :ncells] * Y2 / W, T2[None]])[:, ok]
    atol = np.r_[np.full(g1.N, 1e-20), 1e-10][:, None]
    assert np.all(np.abs(p2 - p1) <= 1e-10 * np.abs(p1) + 10 * atol)
