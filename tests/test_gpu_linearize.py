"""Linearized mechanisms on the GPU (Section 2.2, Alg. 1).

The hydrocarbon workload with quadratic QSS couplings added, linearized by
each of the paper's three methods (species, reaction, one-sided), compiled
and evaluated through the C ABI, against the oracle on the same linearized
mechanism: wdot, Tdot and J under the parity gate.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_05974_b300 import binding, mechgen, workloads
from paper_2405_05974_b300.qssc import linearize
from paper_2405_05974_b300.qssc.build import build_mechanism
from tests.parity import assert_gate

pytestmark = pytest.mark.gpu


def coupled_hydrocarbon():
    return mechgen.add_quadratic_couplings(workloads.mechanism("hydrocarbon"), 8, 5)


@pytest.mark.parametrize("method", list(linearize.METHODS))
def test_linearized_mechanism_parity(method):
    m = linearize.linearize(coupled_hydrocarbon(), method)
    gm = binding.Mechanism(build_mechanism(m), 0)
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["hydrocarbon"], 1024)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    J, w, td = gm.jacobian(d(rho), d(T), d(Y))
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert_gate("wdot", w.cpu().numpy(), ref["wdot"], eb["wdot"])
    assert_gate("Tdot", td.cpu().numpy(), ref["Tdot"], eb["Tdot"])
    r = assert_gate("jac", J.cpu().numpy(), ref["jac"], eb["jac"])
    print(method, gm.N, gm.Q, gm.M, r)
