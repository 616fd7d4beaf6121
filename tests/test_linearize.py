"""Linearization of quadratic QSS couplings (Section 2.2, Alg. 1), CPU side.

Pins: hand-derived answers of Alg. 1 on small coupling patterns (including
the paper's single-reaction example, where either species may be retyped),
an independent brute force over every subset of QSS species, the closed form
of a reverse-only reaction in the oracle, and the compiler's linearized
models against the oracle.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2405_05974_b300 import mechgen, workloads
from paper_2405_05974_b300.qssc import linearize as L
from paper_2405_05974_b300.qssc import mech as qmech
from paper_2405_05974_b300.qssc import model as qmodel
from tests import mechs as hm


def _chain_mech(pairs, reversible=False):
    """QSS species a..e, transported X, N2; one reaction q1 + q2 -> X per pair."""
    names = sorted({x for p in pairs for x in p})
    sp = [hm.species("X", {"H": 2}), hm.species("N2", {"N": 2})]
    sp += [hm.species(q, {"H": 1}, qss=True) for q in names]
    rx = [hm.reaction({a: 1, b: 1} if a != b else {a: 2}, {"X": 1}, 1e12, reversible=reversible)
          for a, b in pairs]
    # every QSS species gets a linear source and sink
    for q in names:
        rx.append(hm.reaction({"X": 1}, {q: 1, "N2": 1}, 1e10, reversible=False))
        rx.append(hm.reaction({q: 1}, {"N2": 1}, 1e11, reversible=False))
    return hm.mech("chain", sp, rx)


def test_alg1_paper_single_reaction_example():
    """One coupling P7 + P5 <=> P12 (Section 2.2's PXC7H15 + PXC5H11 <=> NC12H26):
    retyping either species removes it."""
    m = _chain_mech([("P5", "P7")], reversible=True)
    assert L.couplings(m) == [(0, "forward")]
    assert sorted(L.species_candidates(m)) == [("P5",), ("P7",)]


def test_alg1_chain_of_couplings():
    """Couplings a-b, b-c, c-d: the smallest covers have two species, and
    exactly {a,c}, {b,c}, {b,d} work (hand enumeration of the 6 pairs)."""
    m = _chain_mech([("a", "b"), ("b", "c"), ("c", "d")])
    assert set(L.involved_species(m)) == {"a", "b", "c", "d"}
    got = {frozenset(s) for s in L.species_candidates(m)}
    assert got == {frozenset("ac"), frozenset("bc"), frozenset("bd")}


def test_alg1_self_coupling_and_reverse_direction():
    """2 e -> X forces e; X <=> a + b (reverse coupled) needs a or b."""
    m = _chain_mech([("e", "e")])
    m["reactions"].append(hm.reaction({"X": 1}, {"a": 1, "b": 1}, 1e12, reversible=True))
    sp = m["species"]
    sp += [hm.species("a", {"H": 1}, qss=True), hm.species("b", {"H": 1}, qss=True)]
    for q in ("a", "b"):
        m["reactions"].append(hm.reaction({q: 1}, {"N2": 1}, 1e11, reversible=False))
    assert any(d == "reverse" for _, d in L.couplings(m))
    got = {frozenset(s) for s in L.species_candidates(m)}
    assert got == {frozenset({"e", "a"}), frozenset({"e", "b"})}


def _brute_force_covers(m):
    qss = [s["name"] for s in m["species"] if s["qss"]]

    def coupled(qset):
        for r in m["reactions"]:
            for side, on in ((r["reactants"], r.get("forward", True)), (r["products"], r["reversible"])):
                if on and sum(nu for s, nu in side.items() if s in qset) >= 2:
                    return True
        return False

    for k in range(0, len(qss) + 1):
        found = [set(c) for c in itertools.combinations(qss, k) if not coupled(set(qss) - set(c))]
        if found:
            return found


@pytest.mark.parametrize("key,n,seed", [("tiny", 6, 3), ("hydrocarbon", 8, 5), ("hydrocarbon", 5, 9)])
def test_alg1_matches_brute_force(key, n, seed):
    m = mechgen.add_quadratic_couplings(workloads.mechanism(key), n, seed)
    got = sorted(sorted(c) for c in L.species_candidates(m))
    want = sorted(sorted(c) for c in _brute_force_covers(m))
    assert got == want


@pytest.mark.parametrize("method", list(L.METHODS))
def test_linearized_mechanisms_compile(method):
    m = mechgen.add_quadratic_couplings(workloads.mechanism("hydrocarbon"), 8, 5)
    with pytest.raises(qmech.MechanismError):
        qmech.parse(m)
    lm = L.linearize(m, method)
    assert L.couplings(lm) == []
    ir = qmech.parse(lm)
    qmodel.build_model(ir)
    if method == "reaction":
        assert len(lm["reactions"]) == len(m["reactions"]) - len({j for j, _ in L.couplings(m)})
    if method == "one-sided":
        assert any(r.get("forward", True) is False for r in lm["reactions"])


def test_reverse_only_reaction_closed_form():
    """A <=> B with the forward direction removed: omega_A = +k_b C_B,
    k_b = k_f / K_c, K_c = exp(-(g_B - g_A)/RT) (no mole change)."""
    T0 = 1400.0
    na = [1.0, 0, 0, 0, 0, 0, 0.0]
    nb = [1.0, 0, 0, 0, 0, 0, -0.7]    # g_B/RT - g_A/RT = +0.7
    sp = [hm.species("A", {"H": 2}, nasa=na), hm.species("B", {"H": 2}, nasa=nb),
          hm.species("N2", {"N": 2})]
    r = hm.reaction({"A": 1}, {"B": 1}, 3.0e6)
    r["forward"] = False
    m = hm.mech("rev_only", sp, [r])
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.concentrations_to_state(m, np.array([[1.2], [0.4], [1.0]]), np.array([T0]))
    w = om.eval(rho, T, Y)["wdot"][:, 0]
    kb = 3.0e6 / math.exp(-0.7)
    assert w[0] == pytest.approx(kb * 0.4, rel=1e-13)
    assert w[1] == pytest.approx(-kb * 0.4, rel=1e-13)
    J = om.eval(rho, T, Y)["jac"].reshape(4, 4, 1)[:, :, 0]
    assert J[0, 0] == 0.0 and J[0, 1] == pytest.approx(kb, rel=1e-13)


@pytest.mark.parametrize("method", list(L.METHODS))
def test_linearized_model_matches_oracle(method):
    """The compiler's linearized model (DAG interpreter) against the oracle on
    the same linearized mechanism: wdot, Tdot and J."""
    m = L.linearize(mechgen.add_quadratic_couplings(workloads.mechanism("hydrocarbon"), 8, 5), method)
    ir = qmech.parse(m)
    mod = qmodel.build_model(ir)
    om = oracle.OracleMech(m)
    rho, T, Y = mechgen.generate_states(m, workloads.STATES["hydrocarbon"], 2)
    ref = om.eval(rho, T, Y)
    eb = om.errbound(rho, T, Y)
    C = om.conc(rho, Y)
    n = ir.N + 1
    for c in range(2):
        env = {mod.C[k]: float(C[k, c]) for k in range(ir.N)}
        env[mod.T] = float(T[c])
        outs = mod.wdot + [mod.Tdot] + [mod.jac[i][j] for i in range(n) for j in range(n)]
        got = np.array(mod.g.evaluate(outs, env, fns=mod.bind))
        want = np.r_[ref["wdot"][:, c], ref["Tdot"][c], ref["jac"][:, c]]
        bound = np.r_[eb["wdot"][:, c], eb["Tdot"][c], eb["jac"][:, c]]
        tol = 1e-9 * np.abs(want) + 1e-20 + 64 * bound
        bad = np.abs(got - want) > tol
        assert not bad.any(), np.argwhere(bad)[:5]
