"""Pins of the oracle's substep integrator (backward-Euler substeps with
local error control), CPU only.

* A <=> B with constant temperature: the exact relaxation is exponential;
  the integrated state approaches it, with the global error shrinking like
  the square root of the tolerance (local error control of a first-order
  method: h ~ sqrt(tol)).
* A single accepted substep is exactly one backward-Euler step.
* Every substep conserves mass (rho fixed, sum of Y unchanged).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_05974_b300 import mechgen, workloads
from tests.test_oracle_pins import _ab_mech, state_from_C

T0 = 1300.0


def _ab():
    na = [1.0, 0, 0, 0, 0, 0, 0.0]
    nb = [1.0, 0, 0, 0, 0, 0, -0.4]     # K_c = exp(-0.4); u = 0 so T stays fixed
    m = _ab_mech(2.0e6, 0.0, 0.0, na, nb)
    return m, 2.0e6, 2.0e6 / math.exp(-0.4)


def test_linear_relaxation_closed_form_and_order():
    m, kf, kb = _ab()
    om = oracle.OracleMech(m)
    CA0, CB0 = 1.5, 0.25
    rho, T, Y = state_from_C(m, [CA0, CB0, 1.0], T0)
    D = 1e-6
    Ceq = (CA0 + CB0) * kb / (kf + kb)
    exact = Ceq + (CA0 - Ceq) * math.exp(-(kf + kb) * D)
    errs = []
    for rtol in (1e-3, 1e-4):
        T2, Y2, ns, st = om.integrate(rho, T, Y, D, rtol=rtol, atol_C=1e-12, max_rounds=2000)
        assert st[0] == 0
        CA = om.conc(rho, Y2)[0, 0]
        errs.append(abs(CA - exact) / abs(CA0 - Ceq))
        assert T2[0] == pytest.approx(T0, rel=1e-14)
    assert errs[1] < 5e-3
    assert 2.0 < errs[0] / errs[1] < 5.0, errs      # sqrt(10) per decade


def test_single_substep_is_one_backward_euler_step():
    m = workloads.mechanism("tiny")
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], 16)
    dt = 1e-10
    Ti, Yi, ns, st = om.integrate(rho, T, Y, dt, h0=dt, rtol=1.0, atol_C=1.0, atol_T=1.0)
    Tb, Yb, it, sb = om.be_step(rho, T, Y, dt, max_iter=20)
    one = (st == 0) & (ns == 1) & (sb == 0)
    assert one.mean() > 0.9
    assert np.array_equal(Ti[one], Tb[one]) and np.array_equal(Yi[:, one], Yb[:, one])


@pytest.mark.parametrize("key", ["tiny", "hydrocarbon"])
def test_integration_conserves_mass(key):
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 12)
    T2, Y2, ns, st = om.integrate(rho, T, Y, 1e-7)
    ok = st == 0
    assert ok.any()
    assert np.all(np.abs(Y2[:, ok].sum(0) - Y[:, ok].sum(0)) <= 1e-9)
