"""Pins of the oracle's substep integrator (backward-Euler or variable-step
BDF2 substeps with local error control), CPU only.

* A <=> B with constant temperature: the exact relaxation is exponential;
  the integrated state approaches it, with the global error shrinking like
  tol^(1/2) for backward Euler (local error ~ h^2 held at tol: h ~ tol^(1/2),
  error ~ tol / h) and tol^(2/3) for BDF2 (local error ~ h^3).
* Two substeps of BDF2 (a backward-Euler start, then the two-step formula
  with equal steps) equal the closed-form solves of the linear system.
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


def test_bdf2_relaxation_order_and_steps():
    m, kf, kb = _ab()
    om = oracle.OracleMech(m)
    CA0, CB0 = 1.5, 0.25
    rho, T, Y = state_from_C(m, [CA0, CB0, 1.0], T0)
    D = 1e-6
    Ceq = (CA0 + CB0) * kb / (kf + kb)
    exact = Ceq + (CA0 - Ceq) * math.exp(-(kf + kb) * D)
    errs, steps = [], []
    for rtol in (1e-4, 1e-5, 1e-6):
        T2, Y2, ns, st = om.integrate(rho, T, Y, D, rtol=rtol, atol_C=1e-12, max_rounds=4000, order=2)
        assert st[0] == 0
        errs.append(abs(om.conc(rho, Y2)[0, 0] - exact) / abs(CA0 - Ceq))
        steps.append(ns[0])
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 6.0 and 3.5 < r2 < 6.0, errs     # 10^(2/3) = 4.64 per decade
    _, _, ns_be, _ = om.integrate(rho, T, Y, D, rtol=1e-5, atol_C=1e-12, max_rounds=4000, order=1)
    assert steps[1] * 3 < ns_be[0], (steps, ns_be)


def test_bdf2_two_substeps_closed_form():
    """h0 = D/2 with a loose tolerance: a backward-Euler substep, then one
    BDF2 substep with w = 1, phi2 = (I - 2h/3 A)^-1 (4/3 phi1 - 1/3 phi0)."""
    m, kf, kb = _ab()
    om = oracle.OracleMech(m)
    CA0, CB0 = 1.5, 0.25
    rho, T, Y = state_from_C(m, [CA0, CB0, 1.0], T0)
    D = 1e-6
    h = D / 2
    T2, Y2, ns, st = om.integrate(rho, T, Y, D, h0=h, rtol=1.0, atol_C=1.0, atol_T=1.0, order=2)
    assert st[0] == 0 and ns[0] == 2
    A = np.array([[-kf, kb], [kf, -kb]])
    p0 = np.array([CA0, CB0])
    p1 = np.linalg.solve(np.eye(2) - h * A, p0)
    p2 = np.linalg.solve(np.eye(2) - (2.0 / 3.0) * h * A, 4.0 / 3.0 * p1 - 1.0 / 3.0 * p0)
    assert np.allclose(om.conc(rho, Y2)[:2, 0], p2, rtol=1e-14, atol=0)
    assert T2[0] == pytest.approx(T0, rel=1e-14)
    # with order 1 the same two substeps are two backward-Euler steps
    T1, Y1, ns1, st1 = om.integrate(rho, T, Y, D, h0=h, rtol=1.0, atol_C=1.0, atol_T=1.0, order=1)
    p2be = np.linalg.solve(np.eye(2) - h * A, p1)
    assert ns1[0] == 2 and np.allclose(om.conc(rho, Y1)[:2, 0], p2be, rtol=1e-14, atol=0)


@pytest.mark.parametrize("order", [1, 2])
def test_single_substep_is_one_backward_euler_step(order):
    m = workloads.mechanism("tiny")
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], 16)
    dt = 1e-10
    Ti, Yi, ns, st = om.integrate(rho, T, Y, dt, h0=dt, rtol=1.0, atol_C=1.0, atol_T=1.0, order=order)
    Tb, Yb, it, sb = om.be_step(rho, T, Y, dt, max_iter=20)
    one = (st == 0) & (ns == 1) & (sb == 0)
    assert one.mean() > 0.9
    assert np.array_equal(Ti[one], Tb[one]) and np.array_equal(Yi[:, one], Yb[:, one])


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("key", ["tiny", "hydrocarbon"])
def test_integration_conserves_mass(key, order):
    m = workloads.mechanism(key)
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES[key], 12)
    T2, Y2, ns, st = om.integrate(rho, T, Y, 1e-7, order=order)
    ok = st == 0
    assert ok.any()
    assert np.all(np.abs(Y2[:, ok].sum(0) - Y[:, ok].sum(0)) <= 1e-9)
