"""Linearization of quadratic QSS couplings (Section 2.2, Alg. 1).

A reaction direction has a *quadratic coupling* when its reactant side holds
two or more QSS species counted with multiplicity (q1 + q2 -> ..., 2 q ->
...): its rate is then a product of QSS concentrations and the QSS relations
omega_Q(C, C_Q) = 0 stop being linear in C_Q.  The forward direction reads
the reaction's reactants, the reverse direction (reversible reactions only)
its products.  A QSS species is *involved* in a coupling when it is one of
the reactants of a coupled direction.

Three ways to remove the couplings, each returning a new mechanism
dictionary that the compiler accepts:

* species linearization (Alg. 1): turn a smallest set of involved QSS
  species into transported species.  The candidates are searched by subset
  size, smallest first, among the involved species; every smallest set that
  removes all couplings is returned, and the first (in the order of the
  involved species) is applied unless the caller picks another;
* reaction linearization: drop every reaction with a coupled direction
  (both directions go, so detailed balance is kept);
* one-sided reaction linearization: drop only the coupled direction(s): a
  coupled reverse direction makes the reaction irreversible; a coupled
  forward direction keeps the reaction as reverse-only (``"forward": false``,
  rate of progress -k_b prod C'' with k_b = k_f / K_c); both coupled drops the
  reaction.
"""
from __future__ import annotations

import copy
import itertools
from typing import Dict, List, Set, Tuple


def _qss_names(mech: dict) -> Set[str]:
    return {s["name"] for s in mech["species"] if s["qss"]}


def _order(side: Dict[str, int], qss: Set[str]) -> int:
    return sum(int(nu) for s, nu in side.items() if s in qss)


def couplings(mech: dict, qss: Set[str] = None) -> List[Tuple[int, str]]:
    """(reaction index, "forward" | "reverse") of every coupled direction."""
    qss = _qss_names(mech) if qss is None else qss
    out = []
    for j, r in enumerate(mech["reactions"]):
        if r.get("forward", True) and _order(r["reactants"], qss) >= 2:
            out.append((j, "forward"))
        if r["reversible"] and _order(r["products"], qss) >= 2:
            out.append((j, "reverse"))
    return out


def involved_species(mech: dict) -> List[str]:
    """QSS species that are reactants of a coupled direction (the set A of
    Alg. 1), in species order."""
    qss = _qss_names(mech)
    inv = set()
    for j, d in couplings(mech, qss):
        r = mech["reactions"][j]
        side = r["reactants"] if d == "forward" else r["products"]
        inv.update(s for s in side if s in qss)
    return [s["name"] for s in mech["species"] if s["name"] in inv]


def species_candidates(mech: dict) -> List[Tuple[str, ...]]:
    """Alg. 1: the smallest sets of involved QSS species whose transfer to
    the transported set removes every coupling ([()] if there is none)."""
    A = involved_species(mech)
    qss = _qss_names(mech)
    if not couplings(mech, qss):
        return [()]
    for i in range(1, len(A) + 1):
        B = [sub for sub in itertools.combinations(A, i) if not couplings(mech, qss - set(sub))]
        if B:
            return B
    return []


def _retype(mech: dict, names) -> dict:
    out = copy.deepcopy(mech)
    names = set(names)
    for s in out["species"]:
        if s["name"] in names:
            s["qss"] = False
    # the compiler and the oracle order species as transported, then QSS
    out["species"] = [s for s in out["species"] if not s["qss"]] + [s for s in out["species"] if s["qss"]]
    return out


def species_linearization(mech: dict, choice: int = 0) -> dict:
    B = species_candidates(mech)
    if not B:
        raise ValueError("no set of QSS species removes the couplings")
    out = _retype(mech, B[choice])
    out["name"] = f"{mech.get('name', 'mech')}_linS"
    out["linearization"] = {"method": "species", "retyped": list(B[choice]),
                            "candidates": [list(b) for b in B]}
    return out


def reaction_linearization(mech: dict) -> dict:
    drop = {j for j, _ in couplings(mech)}
    out = copy.deepcopy(mech)
    out["reactions"] = [r for j, r in enumerate(out["reactions"]) if j not in drop]
    out["name"] = f"{mech.get('name', 'mech')}_linR"
    out["linearization"] = {"method": "reaction", "dropped": sorted(drop)}
    return out


def one_sided_linearization(mech: dict) -> dict:
    cpl = couplings(mech)
    fwd = {j for j, d in cpl if d == "forward"}
    rev = {j for j, d in cpl if d == "reverse"}
    out = copy.deepcopy(mech)
    keep = []
    for j, r in enumerate(out["reactions"]):
        f_on = r.get("forward", True) and j not in fwd
        r_on = r["reversible"] and j not in rev
        if not f_on and not r_on:
            continue
        r["reversible"] = r_on
        if not f_on:
            r["forward"] = False
        keep.append(r)
    out["reactions"] = keep
    out["name"] = f"{mech.get('name', 'mech')}_linO"
    out["linearization"] = {"method": "one-sided", "forward_dropped": sorted(fwd),
                            "reverse_dropped": sorted(rev)}
    return out


METHODS = {"species": species_linearization, "reaction": reaction_linearization,
           "one-sided": one_sided_linearization}


def linearize(mech: dict, method: str) -> dict:
    return METHODS[method](mech)
