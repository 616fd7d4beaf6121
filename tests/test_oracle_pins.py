"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself:
the paper's worked SCC example (Fig. 2), textbook closed forms of special
cases (Arrhenius units, equilibrium constants of single-coefficient NASA
polynomials, Lindemann/Troe limits, the Lu-Law single-QSS expression, Cramer's
rule for a 2-species SCC, a linear backward-Euler step), invariants (mass
conservation of atom-balanced mechanisms with exact QSS), binary128 brute
force, complex-step and finite-difference derivatives.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2405_05974_b300 import mechgen, workloads
from tests import mechs as hm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def state_from_C(mech, C, T):
    C = np.asarray(C, dtype=np.float64)
    if C.ndim == 1:
        C = C[:, None]
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    return mechgen.concentrations_to_state(mech, C, T)


# ---------------------------------------------------------------------------
# Tarjan on the paper's example graph (Section 2.3, Fig. 2)
# ---------------------------------------------------------------------------

def test_tarjan_fig2_partition_and_order():
    g = json.load(open(os.path.join(GOLDEN, "tarjan_fig2.json")))
    names = sorted({v for e in g["edges_as_drawn"] for v in e})
    ix = {nm: i for i, nm in enumerate(names)}
    for direction in (0, 1):
        edges = [(ix[a], ix[b]) if direction == 0 else (ix[b], ix[a]) for a, b in g["edges_as_drawn"]]
        comps = oracle.tarjan(len(names), edges)
        got = sorted(sorted(names[v] for v in c) for c in comps)
        assert got == sorted(sorted(c) for c in g["expected_sccs"])
        # every component appears after the components it needs (u needs v)
        pos = {}
        for ci, c in enumerate(comps):
            for v in c:
                pos[v] = ci
        for u, v in edges:
            assert pos[v] <= pos[u]
        # condensed graph: the only inter-component edge joins S6 and G2
        inter = {(pos[u], pos[v]) for u, v in edges if pos[u] != pos[v]}
        assert len(inter) == 1
        (cu, cv), = inter
        members = {frozenset(names[v] for v in comps[cu]), frozenset(names[v] for v in comps[cv])}
        assert members == {frozenset(["S6"]), frozenset(g["group_names"]["G2"])}


def test_generated_qss_groups_match_plan():
    for key in ("tiny", "hydrocarbon", "large"):
        m = workloads.mechanism(key)
        om = oracle.OracleMech(m)
        got = sorted(sorted(om.names[om.N + q] for q in g) for g in om.qss_groups())
        want = sorted(sorted(g) for g in m["planned_qss_groups"])
        assert got == want, key


# ---------------------------------------------------------------------------
# Rate laws: units, Arrhenius, equilibrium constants, third body, falloff
# ---------------------------------------------------------------------------

ISO = {"C": 1, "H": 2, "O": 1}


def _ab_mech(A, b, Ea, nasa_a, nasa_b, reversible=True):
    sp = [hm.species("A", ISO, nasa=nasa_a), hm.species("B", ISO, nasa=nasa_b),
          hm.species("N2", {"N": 2})]
    return hm.mech("ab", sp, [hm.reaction({"A": 1}, {"B": 1}, A, b, Ea, reversible)])


@pytest.mark.parametrize("b,Ea,T", [(0.0, 0.0, 1000.0), (1.0, 0.0, 1500.0), (-0.7, 25000.0, 1800.0),
                                    (2.0, 12000.0, 900.0)])
def test_unimolecular_arrhenius(b, Ea, T):
    A = 3.0e9
    m = _ab_mech(A, b, Ea, hm.nasa_only(1, 3.0), hm.nasa_only(1, 3.0), reversible=False)
    rho, TT, Y = state_from_C(m, [1.0, 0.0, 1.0], T)
    o = oracle.OracleMech(m).eval(rho, TT, Y)
    kf = A * T ** b * math.exp(-Ea * hm.CAL / (hm.R * T))
    assert o["wdot"][1, 0] == pytest.approx(kf, rel=1e-13)
    assert o["wdot"][0, 0] == pytest.approx(-kf, rel=1e-13)


@pytest.mark.parametrize("k,val", [(1, 3.7), (2, 2e-3), (3, -4e-7), (4, 3e-10), (5, -2e-13),
                                   (6, 2500.0), (7, 1.3)])
def test_equilibrium_constant_single_nasa_coefficient(k, val):
    """A <=> B with only NASA coefficient k differing: K_c = exp(-(g_B - g_A)/RT)
    with g/RT in closed form; the reverse rate is k_f / K_c."""
    T = 1234.5
    base = [2.0, 0, 0, 0, 0, 0, 0]
    na = base
    nb = hm.nasa_only(k, base[k - 1] + val, base)
    m = _ab_mech(1.0e6, 0.0, 0.0, na, nb)
    om = oracle.OracleMech(m)
    rho, TT, Y = state_from_C(m, [0.0, 1.0, 1.0], T)
    o = om.eval(rho, TT, Y)
    dg = hm.g_over_RT_single(k, val, T) if k != 1 else hm.g_over_RT_single(1, val, T)
    Kc = math.exp(-dg)
    assert o["wdot"][1, 0] == pytest.approx(-1.0e6 / Kc, rel=1e-12)


def test_detailed_balance_zero_rate():
    T = 1700.0
    m = _ab_mech(5e8, 0.5, 8000.0, [3.1, 1e-4, -2e-8, 1e-12, 0, -1000.0, 2.0],
                 [4.0, -2e-4, 3e-8, -1e-12, 1e-16, 500.0, -1.0])
    om = oracle.OracleMech(m)
    # K_c from the two single-step rates, then set C_B/C_A = K_c
    r1 = om.eval(*state_from_C(m, [1.0, 0.0, 1.0], T))["wdot"][1, 0]
    r2 = om.eval(*state_from_C(m, [0.0, 1.0, 1.0], T))["wdot"][1, 0]
    Kc = r1 / -r2
    o = om.eval(*state_from_C(m, [1.0, Kc, 1.0], T))
    assert abs(o["wdot"][1, 0]) <= 1e-13 * r1


def test_delta_nu_pressure_factor():
    """A <=> B + C with g/RT = a6/T only: K_c = exp(-sum nu a6/T) (P0/(R T))^1."""
    T = 1500.0
    sp = [hm.species("A", {"C": 1, "H": 4}, nasa=hm.nasa_only(6, 100.0)),
          hm.species("B", {"C": 1, "H": 3}, nasa=hm.nasa_only(6, 300.0)),
          hm.species("C", {"H": 1}, nasa=hm.nasa_only(6, -50.0)),
          hm.species("N2", {"N": 2})]
    m = hm.mech("dn", sp, [hm.reaction({"A": 1}, {"B": 1, "C": 1}, 1.0e5)])
    om = oracle.OracleMech(m)
    o = om.eval(*state_from_C(m, [0.0, 1.0, 1.0, 1.0], T))
    Kc = math.exp(-(300.0 - 50.0 - 100.0) / T) * hm.P0 / (hm.R * T)
    # reverse: q_b = (k_f / K_c) C_B C_C with k_f in s^-1 -> k_b in m^3/mol/s
    assert o["wdot"][0, 0] == pytest.approx(1.0e5 / Kc, rel=1e-12)


def test_bimolecular_units():
    """A = 1e13 cm^3/mol/s is 1e7 m^3/mol/s."""
    sp = [hm.species("A", {"H": 1}), hm.species("B", {"O": 2}), hm.species("C", {"O": 1}),
          hm.species("D", {"H": 1, "O": 1}), hm.species("N2", {"N": 2})]
    m = hm.mech("bi", sp, [hm.reaction({"A": 1, "B": 1}, {"C": 1, "D": 1}, 1.0e13, reversible=False)])
    o = oracle.OracleMech(m).eval(*state_from_C(m, [0.5, 2.0, 0.0, 0.0, 1.0], 1000.0))
    assert o["wdot"][2, 0] == pytest.approx(1.0e7 * 0.5 * 2.0, rel=1e-14)


def test_third_body_efficiencies_and_units():
    """A + B + M -> AB + M: rate = k [M] C_A C_B with A in cm^6/mol^2/s (x1e-12)
    and [M] = sum eff_k C_k over transported species."""
    sp = [hm.species("A", {"H": 1}), hm.species("B", {"O": 1, "H": 1}),
          hm.species("AB", {"H": 2, "O": 1}), hm.species("N2", {"N": 2})]
    eff = {"N2": 0.7, "AB": 2.5}
    rx = [hm.reaction({"A": 1, "B": 1}, {"AB": 1}, 2.0e15, reversible=False,
                      third_body={"efficiencies": eff})]
    m = hm.mech("tb", sp, rx)
    C = [0.3, 0.4, 0.5, 2.0]
    o = oracle.OracleMech(m).eval(*state_from_C(m, C, 1200.0))
    M = 0.3 + 0.4 + 2.5 * 0.5 + 0.7 * 2.0
    assert o["wdot"][2, 0] == pytest.approx(2.0e15 * 1e-12 * M * 0.3 * 0.4, rel=1e-14)


def _troe_mech(A_inf, A0, troe):
    sp = [hm.species("A", {"H": 1}), hm.species("B", {"O": 1, "H": 1}),
          hm.species("AB", {"H": 2, "O": 1}), hm.species("N2", {"N": 2})]
    fo = {"low": {"A": A0, "b": 0.0, "Ea": 0.0}, "troe": troe}
    rx = [hm.reaction({"A": 1, "B": 1}, {"AB": 1}, A_inf, reversible=False,
                      third_body={"efficiencies": {}}, falloff=fo)]
    return hm.mech("troe", sp, rx)


def test_falloff_lindemann():
    """F_cent = 1 (alpha = 0, T*** and T** -> infinity) makes the broadening
    factor exactly 1: k = k_inf Pr / (1 + Pr), Pr = k0 [M] / k_inf."""
    T = 1000.0
    C = [1.0, 1.0, 0.0, 3.0]
    Mconc = sum(C)
    kinf = 1e13 * 1e-6
    lind = [0.0, 1e300, 1.0, 1e300]
    for Pr in (1e-6, 1.0, 1e6):
        A0 = Pr * kinf / (Mconc * 1e-12)   # k0 in cm^6/mol^2/s (x1e-12 to SI)
        m = _troe_mech(1e13, A0, lind)
        o = oracle.OracleMech(m).eval(*state_from_C(m, C, T))
        assert o["wdot"][2, 0] == pytest.approx(kinf * Pr / (1 + Pr), rel=1e-12)


def test_troe_centre_point():
    """Where log10 Pr = -c (so f1 = 0) the broadening factor equals F_cent."""
    T = 1300.0
    alpha, T3, T1, T2 = 0.35, 300.0, 2000.0, 6000.0
    Fc = (1 - alpha) * math.exp(-T / T3) + alpha * math.exp(-T / T1) + math.exp(-T2 / T)
    c = -0.4 - 0.67 * math.log10(Fc)
    Pr = 10 ** (-c)
    C = [1.0, 1.0, 0.0, 2.0]
    Mconc = sum(C)
    A0 = Pr * 1e7 / (Mconc * 1e-12)
    m = _troe_mech(1e13, A0, [alpha, T3, T1, T2])
    o = oracle.OracleMech(m).eval(*state_from_C(m, C, T))
    assert o["wdot"][2, 0] == pytest.approx(1e7 * Pr / (1 + Pr) * Fc, rel=1e-12)


def _troe_log10_F(troe, T, x, lFc):
    """log10 of the oracle's broadening factor at log10 Pr = x - c(F_cent):
    the falloff rate divided by its Lindemann part k_inf Pr/(1 + Pr) C_A C_B."""
    c = -0.4 - 0.67 * lFc
    Pr = 10.0 ** (x - c)
    C = [1.0, 1.0, 0.0, 2.0]
    A0 = Pr * 1e7 / (sum(C) * 1e-12)
    m = _troe_mech(1e13, A0, troe)
    o = oracle.OracleMech(m).eval(*state_from_C(m, C, T))
    return math.log10(o["wdot"][2, 0] / (1e7 * Pr / (1 + Pr)))


# (alpha, T***, T*, T**) and T: each F_cent term alone, and mixtures
_TROE_CASES = [((0.0, 300.0, 2000.0, 1e300), 1300.0),     # (1 - alpha) exp(-T/T***) only
               ((1.0, 300.0, 2000.0, 1e300), 1300.0),     # alpha exp(-T/T*) only
               ((0.0, 1.0, 2000.0, 6000.0), 1300.0),      # exp(-T**/T) only
               ((0.35, 300.0, 2000.0, 6000.0), 1300.0),
               ((0.7, 120.0, 900.0, 4500.0), 950.0)]


def _fcent(troe, T):
    alpha, T3, T1, T2 = troe
    return (1 - alpha) * math.exp(-T / T3) + alpha * math.exp(-T / T1) + math.exp(-T2 / T)


@pytest.mark.parametrize("troe,T", _TROE_CASES)
def test_troe_fcent_terms_at_centre(troe, T):
    """At the centre of the broadening curve (f1 = 0) F equals F_cent.  The
    parameter sets switch on one F_cent term at a time ((1 - alpha)
    exp(-T/T***), alpha exp(-T/T*), exp(-T**/T)), so a wrong sign, a swapped
    T/T* ratio or a dropped term in any of them moves the centre value."""
    lFc = math.log10(_fcent(troe, T))
    assert _troe_log10_F(troe, T, 0.0, lFc) == pytest.approx(lFc, rel=1e-12)


@pytest.mark.parametrize("troe,T", _TROE_CASES[3:])
def test_troe_broadening_off_centre(troe, T):
    """Away from the centre, the Gilbert-Luther-Troe broadening satisfies
    log10 F = log10 F_cent / (1 + f1^2) with 1/f1 = n'/x - 0.14, an exact
    affine relation between 1/f1 and 1/x (x = log10 Pr + c).  Recovering f1
    from the oracle's F at points on both sides of the centre and fitting
    1/f1 against 1/x must give intercept -0.14 and slope
    n' = 0.75 - 1.27 log10 F_cent with zero residual: 0.41 for 0.14, a sign
    slip in n' (0.75 + 1.27 log F_cent), a wrong c (which shifts every x) or a
    missing square fails it.  The fit is also the large-|Pr| limit: as
    1/x -> 0 the intercept is the limit of 1/f1, log10 F -> log10 F_cent /
    (1 + 0.14^-2)."""
    lFc = math.log10(_fcent(troe, T))
    xs = np.array([-12.0, -6.0, -3.0, -1.5, -0.6, 0.4, 1.0, 2.5, 4.0])
    lF = np.array([_troe_log10_F(troe, T, x, lFc) for x in xs])
    f1 = np.sign(xs) * np.sqrt(lFc / lF - 1.0)
    A = np.vstack([1.0 / xs, np.ones_like(xs)]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, 1.0 / f1, rcond=None)
    assert icpt == pytest.approx(-0.14, abs=1e-10)
    assert slope == pytest.approx(0.75 - 1.27 * lFc, rel=1e-10)
    assert np.max(np.abs(A @ np.array([slope, icpt]) - 1.0 / f1)) <= 1e-10


@pytest.mark.parametrize("troe,T", _TROE_CASES[3:])
def test_troe_broadening_vanishes_at_pole(troe, T):
    """Where the denominator n' - 0.14 x of f1 vanishes (x = n'/0.14), f1 is
    infinite and the broadening factor is exactly 1; just past the pole F
    drops below 1 again.  Pins n' and 0.14 jointly at a point far from the
    centre."""
    lFc = math.log10(_fcent(troe, T))
    xp = (0.75 - 1.27 * lFc) / 0.14
    assert abs(_troe_log10_F(troe, T, xp, lFc)) <= 1e-13
    assert _troe_log10_F(troe, T, xp + 2.0, lFc) < -1e-4


# ---------------------------------------------------------------------------
# QSS closed forms
# ---------------------------------------------------------------------------

def test_single_qss_species_closed_form():
    """A -> q -> B: C_q = k1 C_A / k2; omega_B = k2 C_q (Lu-Law singleton)."""
    sp = [hm.species("A", ISO), hm.species("B", ISO), hm.species("N2", {"N": 2}),
          hm.species("q", ISO, qss=True)]
    k1, k2 = 3.0e4, 7.0e8
    m = hm.mech("q1", sp, [hm.reaction({"A": 1}, {"q": 1}, k1, reversible=False),
                           hm.reaction({"q": 1}, {"B": 1}, k2, reversible=False)])
    o = oracle.OracleMech(m).eval(*state_from_C(m, [2.0, 0.5, 1.0], 1000.0), cq=True)
    assert o["cq"][0, 0] == pytest.approx(k1 * 2.0 / k2, rel=1e-14)
    assert o["wdot"][1, 0] == pytest.approx(k1 * 2.0, rel=1e-14)
    assert o["wdot"][0, 0] == pytest.approx(-k1 * 2.0, rel=1e-14)


def test_two_species_scc_cramer():
    """A -> q1 <=> q2 -> B (q1, q2 strongly connected): Cramer's rule."""
    T = 1100.0
    sp = [hm.species("A", ISO, nasa=hm.nasa_only(1, 3.0)), hm.species("B", ISO, nasa=hm.nasa_only(1, 3.0)),
          hm.species("N2", {"N": 2}), hm.species("q1", ISO, qss=True, nasa=hm.nasa_only(6, 400.0)),
          hm.species("q2", ISO, qss=True, nasa=hm.nasa_only(6, -300.0))]
    k1, k2f, k3 = 2.0e3, 5.0e6, 8.0e7
    m = hm.mech("q2", sp, [hm.reaction({"A": 1}, {"q1": 1}, k1, reversible=False),
                           hm.reaction({"q1": 1}, {"q2": 1}, k2f, reversible=True),
                           hm.reaction({"q2": 1}, {"B": 1}, k3, reversible=False)])
    om = oracle.OracleMech(m)
    assert om.qss_groups() == [[0, 1]]
    CA = 1.7
    o = om.eval(*state_from_C(m, [CA, 0.2, 1.0], T), cq=True)
    Kc = math.exp(-(-300.0 - 400.0) / T)
    k2b = k2f / Kc
    # [-k2f  k2b     ] [q1]   [-k1 CA]
    # [ k2f -k2b - k3] [q2] = [   0  ]
    a11, a12, a21, a22 = -k2f, k2b, k2f, -k2b - k3
    b1, b2 = -k1 * CA, 0.0
    det = a11 * a22 - a12 * a21
    q1 = (b1 * a22 - a12 * b2) / det
    q2 = (a11 * b2 - b1 * a21) / det
    assert o["cq"][0, 0] == pytest.approx(q1, rel=1e-13)
    assert o["cq"][1, 0] == pytest.approx(q2, rel=1e-13)
    assert o["wdot"][1, 0] == pytest.approx(k3 * q2, rel=1e-13)


# ---------------------------------------------------------------------------
# invariants and brute force on the generated mechanisms
# ---------------------------------------------------------------------------

def _states(key, n):
    m = workloads.mechanism(key)
    return m, mechgen.generate_states(m, workloads.STATES[key], n)


@pytest.mark.parametrize("key,n", [("tiny", 256), ("hydrocarbon", 128), ("large", 32)])
def test_mass_conservation(key, n):
    """Atom balance plus exact QSS: sum_k W_k omega_k = 0 over transported
    species, and sum_k W_k J_kj = 0 for every column j."""
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    o = om.eval(rho, T, Y)
    W = om.W
    s = (W[:, None] * o["wdot"]).sum(0)
    scale = (W[:, None] * np.abs(o["wdot"])).sum(0)
    assert np.all(np.abs(s) <= 1e-13 * scale)
    nn = om.n
    J = o["jac"].reshape(nn, nn, -1)
    cs = (W[:, None, None] * J[:om.N]).sum(0)
    cscale = (W[:, None, None] * np.abs(J[:om.N])).sum(0)
    # the column sums see the cancellation inside each entry as well
    assert np.all(np.abs(cs) <= 1e-11 * cscale + 1e-300)


@pytest.mark.parametrize("key,n", [("tiny", 256), ("hydrocarbon", 64), ("large", 16)])
def test_qss_residual_and_solvers(key, n):
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    r, mag = om.qss_residual(rho, T, Y)
    assert np.all(np.abs(r) <= 1e-12 * mag)
    a = om.eval(rho, T, Y, jac=False, cq=True, ordered=True)["cq"]
    b = om.eval(rho, T, Y, jac=False, cq=True, ordered=False)["cq"]
    assert np.allclose(a, b, rtol=1e-12, atol=0)
    assert np.all(a >= 0)
    q = om.qss_newton_q128(rho, T, Y, iters=3)
    assert np.allclose(a, q, rtol=1e-12, atol=0)


@pytest.mark.parametrize("key,n", [("tiny", 64), ("hydrocarbon", 16), ("large", 4)])
def test_jacobian_complex_step(key, n):
    """Complex-step derivative of the oracle's own f = (wdot, Tdot) agrees with
    its analytic Jacobian to 1e-12 relative, or within the first-order rounding
    bound where the entry's terms cancel."""
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    J = om.eval(rho, T, Y)["jac"]
    Jcs = om.jac_complex_step(rho, T, Y)
    eb = om.errbound(rho, T, Y)["jac"]
    ok = np.abs(J - Jcs) <= 1e-12 * np.abs(J) + 2.0 * eb + 1e-300
    assert ok.all(), np.argwhere(~ok)[:5]


@pytest.mark.parametrize("key,n", [("tiny", 64), ("hydrocarbon", 16), ("large", 4)])
def test_running_error_bound_holds(key, n):
    """The first-order rounding bound of the FP64 results (running error
    analysis) dominates their distance to the binary128 evaluation."""
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    o = om.eval(rho, T, Y)
    q = om.eval_q128(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    assert np.all(np.abs(o["jac"] - q["jac"]) <= eb["jac"] + 1e-300)
    assert np.all(np.abs(o["wdot"] - q["wdot"]) <= eb["wdot"] + 1e-300)
    assert np.all(np.abs(o["Tdot"] - q["Tdot"]) <= eb["Tdot"] + 1e-300)


# ---------------------------------------------------------------------------
# Simplified Jacobians (Section 3.2.1) and the FD temperature column (3.2.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("key,n", [("tiny", 64), ("hydrocarbon", 16)])
def test_constant_qss_jacobian_is_derivative_at_fixed_cq(key, n):
    """The constant-QSS Jacobian is d f(phi; C_Q) / d phi with C_Q held at its
    solved values: the complex step through the explicit rate expressions with
    C_Q frozen (no QSS solve) must agree with the hand-written partials, every
    row including that of T."""
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    cq = om.eval(rho, T, Y, jac=False, cq=True)["cq"]
    v = om.eval_variant(rho, T, Y, "const_qss")
    Jcs = om.jac_cs_fixed_cq(rho, T, Y, cq)
    ok = np.abs(v["jac"] - Jcs) <= 1e-12 * np.abs(Jcs) + 2.0 * v["jac_err"] + 1e-300
    assert ok.all(), np.argwhere(~ok)[:5]
    # and it is not the exact Jacobian (the dropped term is not zero)
    Jex = om.eval(rho, T, Y)["jac"]
    assert np.abs(v["jac"] - Jex).max() > 1e-6 * np.abs(Jex).max()


@pytest.mark.parametrize("key,n", [("tiny", 64), ("hydrocarbon", 16)])
def test_zero_qss_jacobian_species_rows(key, n):
    """The zero-QSS Jacobian's species rows are d omega(phi; C_Q = 0) / d phi
    (complex step with the QSS concentrations frozen at zero); its source term
    stays the exact one."""
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    v = om.eval_variant(rho, T, Y, "zero_qss")
    Jcs = om.jac_cs_fixed_cq(rho, T, Y, np.zeros((om.Q, T.shape[0])))
    N, nn = om.N, om.n
    a = v["jac"].reshape(nn, nn, -1)[:N]
    b = Jcs.reshape(nn, nn, -1)[:N]
    e = v["jac_err"].reshape(nn, nn, -1)[:N]
    ok = np.abs(a - b) <= 1e-12 * np.abs(b) + 2.0 * e + 1e-300
    assert ok.all(), np.argwhere(~ok)[:5]
    ref = om.eval(rho, T, Y, jac=False)
    assert np.array_equal(v["wdot"], ref["wdot"]) and np.array_equal(v["Tdot"], ref["Tdot"])


def test_variants_coincide_without_qss_species():
    """With no QSS species the second term of Eq. JQSS is absent: all three
    constructions give the same Jacobian, bit for bit."""
    na = [3.5, 1e-4, 0, 0, 0, -1000.0, 2.0]
    nb = [3.2, -2e-4, 0, 0, 0, 500.0, 1.0]
    m = _ab_mech(2.0e8, 0.5, 30000.0, na, nb)
    om = oracle.OracleMech(m)
    rho, T, Y = state_from_C(m, [[1.5, 0.2], [0.25, 0.9], [1.0, 1.0]], [1300.0, 1700.0])
    Js = [om.eval_variant(rho, T, Y, v)["jac"] for v in ("exact", "const_qss", "zero_qss")]
    assert np.array_equal(Js[0], Js[1]) and np.array_equal(Js[0], Js[2])
    assert np.array_equal(Js[0], om.eval(rho, T, Y)["jac"])


@pytest.mark.parametrize("key,n", [("tiny", 64), ("hydrocarbon", 16)])
def test_fd_temperature_column(key, n):
    """Section 3.2.2 reading: the species rows' T column by a central
    difference with h = 2^(e-20) (T in [2^e, 2^(e+1))).  It agrees with the
    complex-step T column to the difference's truncation and rounding error;
    the concentration columns are those of the analytic Jacobian."""
    m, (rho, T, Y) = _states(key, n)
    om = oracle.OracleMech(m)
    v = om.eval_variant(rho, T, Y, "exact", "fd")
    J = om.eval(rho, T, Y)["jac"]
    Jcs = om.jac_complex_step(rho, T, Y)
    N, nn = om.N, om.n
    a, b, c = (x.reshape(nn, nn, -1) for x in (v["jac"], J, Jcs))
    e = v["jac_err"].reshape(nn, nn, -1)
    assert np.array_equal(a[:N, :N], b[:N, :N])
    d = np.abs(a[:, N] - c[:, N])
    ok = d <= 1e-7 * np.abs(c[:, N]) + 4.0 * e[:, N] + 1e-300
    assert ok.all(), (np.argwhere(~ok)[:5], d.max())
    # the step is small: the FD column is far closer than a 1 % step would be
    assert np.median(d / (np.abs(c[:, N]) + 1e-300)) < 1e-8


def test_fd_errbound_values_match_plain_fd():
    """The running-error FD performs the same FP64 operations as the plain
    one (identical values); its bounds are finite and nonnegative.  (The
    running-error type itself is pinned against binary128 in
    test_running_error_bound_holds.)"""
    m, (rho, T, Y) = _states("tiny", 32)
    om = oracle.OracleMech(m)
    J = om.jac_fd(rho, T, Y, dC=1e-4, dT=1e-4)
    Jb, E = om.jac_fd_errbound(rho, T, Y, dC=1e-4, dT=1e-4)
    assert np.array_equal(J, Jb)
    assert np.all(E >= 0) and np.all(np.isfinite(E))


def test_jacobian_central_fd_second_order():
    m, (rho, T, Y) = _states("tiny", 16)
    om = oracle.OracleMech(m)
    J = om.eval(rho, T, Y)["jac"]
    errs = []
    for h in (1e-3, 5e-4):
        Jfd = om.jac_fd(rho, T, Y, dC=h, dT=h * 100, central=True)
        errs.append(np.linalg.norm(Jfd - J) / np.linalg.norm(J))
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, errs


def _paper_C_states(m, n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    N = sum(1 for s in m["species"] if not s["qss"])
    C = rng.uniform(lo, hi, size=(N, n))
    T = rng.uniform(300.0, 1300.0, size=n)
    return mechgen.concentrations_to_state(m, C, T)


def test_fd_first_order_convergence_appendixC():
    """Appendix C protocol: C ~ U[0.1, 1.1] mol/m^3, T ~ U[300, 1300] K,
    one-sided FD in C converges to the analytic Jacobian at first order."""
    m = workloads.mechanism("tiny")
    om = oracle.OracleMech(m)
    rho, T, Y = _paper_C_states(m, 64, 0.1, 1.1, 7)
    J = om.eval(rho, T, Y)["jac"]
    nn = om.n
    Jc = J.reshape(nn, nn, -1)[:, :om.N]
    hs = [1e-2, 1e-3, 1e-4, 1e-5]
    e = []
    for h in hs:
        Jfd = om.jac_fd(rho, T, Y, dC=h, dT=1e-3, central=False).reshape(nn, nn, -1)[:, :om.N]
        num = np.sqrt(((Jfd - Jc) ** 2).sum(axis=(0, 1)))
        den = np.sqrt((Jc ** 2).sum(axis=(0, 1)))
        e.append(np.mean(num / den))
    slope = np.polyfit(np.log10(hs), np.log10(e), 1)[0]
    assert 0.85 < slope < 1.15, (slope, e)


def test_frobenius_error_protocol_section3():
    """Section 3.2.1 protocol: C ~ U[1e-4, 1], T ~ U[300, 1300], central FD
    with perturbation 1e-4: the relative Frobenius error is small."""
    m = workloads.mechanism("tiny")
    om = oracle.OracleMech(m)
    rho, T, Y = _paper_C_states(m, 100, 1e-4, 1.0, 11)
    J = om.eval(rho, T, Y)["jac"]
    Jfd = om.jac_fd(rho, T, Y, dC=1e-4, dT=1e-4, central=True)
    eps = np.mean(np.linalg.norm(J - Jfd, axis=0) / np.linalg.norm(Jfd, axis=0))
    assert eps < 1e-5


# ---------------------------------------------------------------------------
# backward-Euler step
# ---------------------------------------------------------------------------

def test_be_linear_closed_form():
    """A <=> B with u = 0 (h/RT = 1, so Tdot = 0): the backward-Euler step is the
    2x2 linear solve, reached by Newton in one update."""
    T0 = 1300.0
    na = [1.0, 0, 0, 0, 0, 0, 0.0]
    nb = [1.0, 0, 0, 0, 0, 0, -0.4]   # shifts g/RT by +0.4: K_c = exp(-0.4)
    m = _ab_mech(2.0e6, 0.0, 0.0, na, nb)
    sp = m["species"]
    om = oracle.OracleMech(m)
    CA0, CB0, CN = 1.5, 0.25, 1.0
    rho, T, Y = state_from_C(m, [CA0, CB0, CN], T0)
    dt = 3e-7
    T2, Y2, it, st = om.be_step(rho, T, Y, dt)
    kf = 2.0e6
    kb = kf / math.exp(-0.4)
    den = 1 + dt * kf + dt * kb
    CA = ((1 + dt * kb) * CA0 + dt * kb * CB0) / den
    CB = CA0 + CB0 - CA
    C2 = om.conc(rho, Y2)[:, 0]
    assert st[0] == 0 and it[0] <= 2
    assert C2[0] == pytest.approx(CA, rel=1e-13)
    assert C2[1] == pytest.approx(CB, rel=1e-13)
    assert T2[0] == pytest.approx(T0, rel=1e-15)
    del sp


def test_be_mass_and_residual_hydrocarbon():
    m, (rho, T, Y) = _states("hydrocarbon", 32)
    om = oracle.OracleMech(m)
    dt = workloads.IMPLICIT_DT
    T2, Y2, it, st = om.be_step(rho, T, Y, dt)
    ok = st == 0
    assert ok.sum() >= 4
    # mass: sum_k Y_k is conserved (rho fixed, sum_k W_k omega_k = 0)
    assert np.allclose(Y2[:, ok].sum(0), Y[:, ok].sum(0), rtol=1e-11, atol=0)
    # residual G(phi) = phi - phi0 - dt f(phi) at the returned state
    phi0 = np.vstack([om.conc(rho, Y), T[None, :]])
    phi = np.vstack([om.conc(rho, Y2), T2[None, :]])
    f, _ = om.eval_phi(phi, jac=False)
    G = phi - phi0 - dt * f
    scale = np.abs(phi) + np.abs(phi0) + dt * np.abs(f)
    assert np.all(np.abs(G[:, ok]) <= 1e-10 * scale[:, ok].max(axis=0))


# ---------------------------------------------------------------------------
# Temperature equation (constant volume, Section 3.2.2: heat release from the
# production rates)
# ---------------------------------------------------------------------------

def test_tdot_single_coefficient_closed_form():
    """A -> B + C, irreversible, NASA sets with only a1 and a6: h/RT = a1 + a6/T,
    so the molar internal energy is u = R (T (a1 - 1) + a6) and c_v = R (a1 - 1).
    With q = k_f C_A the constant-volume energy equation gives
    Tdot = -q sum_k nu_k (T (a1_k - 1) + a6_k) / sum_k C_k (a1_k - 1).
    The reaction changes the mole count, so h in place of u (an extra R T per
    mole) fails, and c_p in place of c_v in the denominator fails."""
    T = 1234.5
    nasa = {"A": (3.0, 1500.0), "B": (4.2, -2500.0), "C": (2.5, 700.0), "N2": (3.5, 0.0)}
    sp = [hm.species("A", {"C": 1, "H": 4}, nasa=[nasa["A"][0], 0, 0, 0, 0, nasa["A"][1], 0.0]),
          hm.species("B", {"C": 1, "H": 3}, nasa=[nasa["B"][0], 0, 0, 0, 0, nasa["B"][1], 0.0]),
          hm.species("C", {"H": 1}, nasa=[nasa["C"][0], 0, 0, 0, 0, nasa["C"][1], 0.0]),
          hm.species("N2", {"N": 2}, nasa=[nasa["N2"][0], 0, 0, 0, 0, 0.0, 0.0])]
    kf = 3.0e4
    m = hm.mech("tdot", sp, [hm.reaction({"A": 1}, {"B": 1, "C": 1}, kf, reversible=False)])
    C = {"A": 0.8, "B": 0.3, "C": 0.2, "N2": 5.0}
    o = oracle.OracleMech(m).eval(*state_from_C(m, [C[k] for k in ("A", "B", "C", "N2")], T))
    q = kf * C["A"]
    nu = {"A": -1, "B": 1, "C": 1, "N2": 0}
    num = sum(nu[k] * (T * (nasa[k][0] - 1.0) + nasa[k][1]) for k in nu)
    den = sum(C[k] * (nasa[k][0] - 1.0) for k in nu)
    assert o["Tdot"][0] == pytest.approx(-q * num / den, rel=1e-13)


def _internal_energy(mech, om, rho, T, Y):
    """U = sum_k C_k u_k(T) per unit volume, with the molar internal energy
    u = h - R T from the NASA-7 enthalpy h/RT = a1 + a2 T/2 + a3 T^2/3 +
    a4 T^3/4 + a5 T^4/5 + a6/T (single-range sets); also returns
    sum_k |C_k u_k| as a scale."""
    tr = [s for s in mech["species"] if not s["qss"]]
    C = om.conc(rho, Y)
    u = np.zeros_like(C)
    for k, s in enumerate(tr):
        assert s["nasa_lo"] == s["nasa_hi"]
        a = s["nasa_lo"]
        h_RT = a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
        u[k] = hm.R * T * (h_RT - 1.0)
    return (C * u).sum(0), np.abs(C * u).sum(0), C, u


def test_internal_energy_conserved_along_integration():
    """At constant volume the mixture's internal energy sum_k C_k u_k(T) is
    constant: the chemistry only moves energy between chemical and sensible
    forms.  Integrating the tiny workload over 2e-9 s (T moves by up to a few
    hundred K), the oracle's trajectory keeps U to 2e-4 of the sensible energy
    it moved at rtol 1e-7, and the drift falls like the backward-Euler global
    error, tol^(1/2) (ten times over two decades); c_p in place of c_v, or h
    in place of u, in Tdot changes the temperature rise by tens of percent
    and fails it."""
    m = workloads.mechanism("tiny")
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["tiny"], 6)
    U0, S0, _, u0 = _internal_energy(m, om, rho, T, Y)
    drift = []
    for rtol in (1e-5, 1e-7):
        T2, Y2, ns, st = om.integrate(rho, T, Y, 2e-9, rtol=rtol, atol_C=1e-14, atol_T=1e-8,
                                      max_rounds=20000)
        assert np.all(st == 0)
        U1, _, C1, u1 = _internal_energy(m, om, rho, T2, Y2)
        sensible = np.abs((C1 * (u1 - u0)).sum(0))
        assert np.all(np.abs(T2 - T) > 1.0)
        drift.append(np.abs(U1 - U0) / sensible)
    assert np.all(drift[1] <= 2e-4), drift
    assert np.all(drift[0] / drift[1] > 5.0), drift
