"""Mechanism intermediate representation for the compiler.

Reads the mechanism dictionary (see ``mechgen``), orders species as
transported (0..N-1) then QSS (N..N+Q-1), converts rate parameters to SI
(CHEMKIN cm-mol-s -> m-mol-s by (1e-6)^(order-1); cal/mol -> J/mol), and
checks the linearity condition of the QSS relations (Section 2.2): the
reactant side of every active reaction direction holds at most one QSS
species, with coefficient one (``qssc.linearize`` removes the couplings that
break it).  A reaction may be reverse-only (``"forward": false``).
"""
from __future__ import annotations

import hashlib
import json
import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

R_GAS = 8.31446261815324
CAL = 4.184
P_STD = 101325.0


@dataclass
class Rxn:
    lhs: List[Tuple[int, int]]
    rhs: List[Tuple[int, int]]
    reversible: bool
    kind: int                    # 0 elementary, 1 third body, 2 Troe falloff
    lnA: float                   # ln of the SI pre-exponential factor (k_inf for falloff)
    b: float
    EaR: float                   # Ea / R in K
    eff: Dict[int, float] = field(default_factory=dict)   # non-unit collision efficiencies
    lnA0: float = 0.0
    b0: float = 0.0
    Ea0R: float = 0.0
    troe: Tuple[float, float, float, float] = (0.0, 1.0, 1.0, 1.0)
    qss_l: int = -1
    qss_r: int = -1
    forward: bool = True         # False: reverse-only (one-sided linearization)


@dataclass
class MechIR:
    name: str
    names: List[str]
    N: int
    Q: int
    W: List[float]
    nasa_lo: List[List[float]]
    nasa_hi: List[List[float]]
    Tmid: List[float]
    rxns: List[Rxn]
    digest: str


class MechanismError(ValueError):
    pass


def parse(mech: dict) -> MechIR:
    sp = mech["species"]
    order = [s for s in sp if not s["qss"]] + [s for s in sp if s["qss"]]
    names = [s["name"] for s in order]
    ix = {nm: i for i, nm in enumerate(names)}
    N = sum(1 for s in sp if not s["qss"])
    Q = len(sp) - N
    if N < 1:
        raise MechanismError("mechanism has no transported species")
    rxns = []
    for j, r in enumerate(mech["reactions"]):
        try:
            lhs = [(ix[s], int(nu)) for s, nu in r["reactants"].items()]
            rhs = [(ix[s], int(nu)) for s, nu in r["products"].items()]
        except KeyError as e:
            raise MechanismError(f"reaction {j}: unknown species {e}") from None
        if any(nu <= 0 for _, nu in lhs + rhs):
            raise MechanismError(f"reaction {j}: stoichiometric coefficients must be positive")
        forward = bool(r.get("forward", True))
        reversible = bool(r["reversible"])
        if not forward and not reversible:
            raise MechanismError(f"reaction {j}: both directions removed")
        ql = [(s, nu) for s, nu in lhs if s >= N]
        qr = [(s, nu) for s, nu in rhs if s >= N]
        # only the reactant side of an active direction enters a rate
        for side, lab, active in ((ql, "left", forward), (qr, "right", reversible)):
            if active and (len(side) > 1 or (side and side[0][1] != 1)):
                raise MechanismError(
                    f"reaction {j}: quadratic QSS coupling on the {lab} side "
                    "(linearization of the QSS relations is required first: qssc.linearize)")
        kind = 2 if r.get("falloff") else (1 if r.get("third_body") else 0)
        order_ = sum(nu for _, nu in lhs)
        ord_inf = order_ + (1 if kind == 1 else 0)
        if r["A"] <= 0:
            raise MechanismError(f"reaction {j}: A must be positive")
        lnA = math.log(r["A"]) + (ord_inf - 1) * math.log(1e-6)
        eff = {}
        if kind:
            for s, e in (r.get("third_body") or {}).get("efficiencies", {}).items():
                if s not in ix:
                    raise MechanismError(f"reaction {j}: unknown collider {s}")
                if ix[s] < N and float(e) != 1.0:
                    eff[ix[s]] = float(e)
        rx = Rxn(lhs=lhs, rhs=rhs, reversible=reversible, kind=kind, lnA=lnA,
                 b=float(r["b"]), EaR=float(r["Ea"]) * CAL / R_GAS, eff=eff,
                 qss_l=(ql[0][0] - N) if (ql and forward) else -1,
                 qss_r=(qr[0][0] - N) if (qr and reversible) else -1, forward=forward)
        if kind == 2:
            lo = r["falloff"]["low"]
            if lo["A"] <= 0:
                raise MechanismError(f"reaction {j}: low-pressure A must be positive")
            rx.lnA0 = math.log(lo["A"]) + order_ * math.log(1e-6)
            rx.b0 = float(lo["b"])
            rx.Ea0R = float(lo["Ea"]) * CAL / R_GAS
            rx.troe = tuple(float(x) for x in r["falloff"]["troe"])
        rxns.append(rx)
    digest = hashlib.sha256(json.dumps(mech, sort_keys=True).encode()).hexdigest()[:16]
    return MechIR(name=mech.get("name", "mech"), names=names, N=N, Q=Q,
                  W=[float(s["W"]) for s in order[:N]],
                  nasa_lo=[list(map(float, s["nasa_lo"])) for s in order],
                  nasa_hi=[list(map(float, s["nasa_hi"])) for s in order],
                  Tmid=[float(s.get("Tmid", 1000.0)) for s in order], rxns=rxns, digest=digest)
