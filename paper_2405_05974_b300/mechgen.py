"""Seeded synthetic QSS mechanisms and thermochemical states (inputs only).

This module is the single source of inputs for both the CUDA path and the
CPU oracle.  It draws random numbers and lays out a mechanism description; it
evaluates none of the method's arithmetic (no rates, no thermodynamic
functions, no QSS algebra, no graph analysis).  Structural properties that the
method relies on -- linear QSS coupling (Section 2.1/2.2: at most one QSS
species per reaction side, coefficient one), the strongly-connected-component
layout of the QSS dependency digraph (Section 2.3, Fig. 2) and bounded
equilibrium constants -- are obtained by construction, and are verified by
tests with the compiler's and the oracle's own analyses.

Mechanism dictionary schema (``mech``)::

    {"name": str, "seed": int,
     "units": {"A": "cm-mol-s", "Ea": "cal/mol"},
     "elements": ["C", "H", "O", "N"],
     "species": [{"name", "W" (kg/mol), "composition": {el: n}, "qss": bool,
                  "nasa_lo": [a1..a7], "nasa_hi": [a1..a7], "Tmid": K}],
     "reactions": [{"reactants": {sp: nu}, "products": {sp: nu},
                    "reversible": bool, "A": float, "b": float, "Ea": float,
                    "third_body": None | {"efficiencies": {sp: eff}},
                    "falloff": None | {"low": {"A","b","Ea"},
                                        "troe": [alpha, T3, T1, T2]},
                    "duplicate": bool}]}

Transported species are listed first, QSS species after them.  ``A`` is in
CHEMKIN cm-mol-s units for the reaction's order (the low-pressure limit of a
falloff reaction has one more order), ``Ea`` in cal/mol.  Third-body and
falloff reactions both carry an ``efficiencies`` table (default 1 for every
transported species; QSS species never act as colliders).

State arrays are SoA: ``rho[ncells]`` (kg/m^3), ``T[ncells]`` (K),
``Y[N][ncells]`` (mass fractions of the N transported species).
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

ATOMIC_WEIGHT = {"C": 12.011e-3, "H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}
ELEMENTS = ("C", "H", "O", "N")
R_GAS = 8.31446261815324  # J/(mol K), used only to turn (P, T, Y) into rho
P_ATM = 101325.0
T_REF_RATE = 1000.0     # K, reference temperature of the drawn pre-exponential factors
T_REF_THERMO = 1500.0   # K, temperature at which the a1 term of g/RT vanishes

# Small species always present as transported species.  Tuples are (C, H, O, N).
CORE_SPECIES = [
    ("N2", (0, 0, 0, 2)), ("O2", (0, 0, 2, 0)), ("H2", (0, 2, 0, 0)),
    ("H2O", (0, 2, 1, 0)), ("H", (0, 1, 0, 0)), ("O", (0, 0, 1, 0)),
    ("OH", (0, 1, 1, 0)), ("CO", (1, 0, 1, 0)), ("CO2", (1, 0, 2, 0)),
    ("HO2", (0, 1, 2, 0)), ("H2O2", (0, 2, 2, 0)), ("CH4", (1, 4, 0, 0)),
    ("CH3", (1, 3, 0, 0)), ("CH2O", (1, 2, 1, 0)), ("C2H4", (2, 4, 0, 0)),
    ("C2H6", (2, 6, 0, 0)),
]
# Composition steps used to grow related species (so that atom-balanced
# transfer reactions between them exist).
STEPS = [(0, 1, 0, 0), (0, 2, 0, 0), (0, 0, 1, 0), (0, 1, 1, 0), (1, 2, 0, 0),
         (1, 3, 0, 0), (1, 0, 1, 0), (0, 1, 2, 0)]


@dataclass
class MechConfig:
    """Sizes and distributions of one synthetic mechanism."""
    name: str
    n_transported: int
    n_qss: int
    n_reactions: int
    n_third_body: int
    n_troe: int
    qss_groups: List[int]            # sizes of the QSS strongly connected groups
    seed: int
    all_reversible: bool = False
    dup_fraction: float = 0.0        # fraction of reactions that are DUPLICATE copies
    qss_reaction_fraction: float = 0.55
    max_carbon: int = 4


@dataclass
class StateConfig:
    """Distribution of the thermochemical states of one workload."""
    T_range: Tuple[float, float]
    P_range_atm: Tuple[float, float]
    P_log_uniform: bool
    dirichlet_alpha: float
    near_pure_fraction: float = 0.0
    seed: int = 0


# ---------------------------------------------------------------------------
# species
# ---------------------------------------------------------------------------

def _comp_add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _comp_sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def _comp_name(c):
    s = ""
    for el, n in zip(ELEMENTS, c):
        if n:
            s += el + (str(n) if n > 1 else "")
    return s or "X"


def _weight(c):
    return sum(n * ATOMIC_WEIGHT[el] for el, n in zip(ELEMENTS, c))


def _valid(c, max_carbon):
    C, H, O, N = c
    if min(c) < 0 or N != 0 or sum(c) == 0:
        return False
    if C > max_carbon or O > 3:
        return False
    if H > 2 * C + 2 + (1 if O else 0) + O:
        return False
    return True


def _grow_species(rng, start, count, taken, max_carbon):
    """Random walk over compositions from ``start`` by the STEPS moves."""
    out = []
    frontier = list(start)
    tries = 0
    while len(out) < count and tries < 100000:
        tries += 1
        base = frontier[rng.integers(len(frontier))]
        step = STEPS[rng.integers(len(STEPS))]
        sign = 1 if rng.random() < 0.7 else -1
        c = _comp_add(base, tuple(sign * s for s in step))
        if not _valid(c, max_carbon) or c in taken:
            continue
        taken.add(c)
        out.append(c)
        frontier.append(c)
    if len(out) < count:
        raise RuntimeError("could not grow enough distinct species compositions")
    return out


def _nasa(rng, comp):
    """NASA-7 coefficients: a1 ~ U(2.5, 6); a2..a5 small and scaled per power;
    a6, a7 = element-additive part + bounded perturbation, and a7 also carries
    -a1 (ln T_c - 1) with T_c = 1500 K, so that the a1 term of g/RT is small
    over the workloads' temperature range.  The element-additive parts cancel in
    any atom-balanced reaction, which keeps every equilibrium constant bounded
    (|ln K_c| of order 10) without evaluating one."""
    h_el = {"C": -1500.0, "H": -2500.0, "O": -4000.0, "N": 0.0}
    s_el = {"C": 1.0, "H": 0.6, "O": 1.5, "N": 1.0}
    a1 = rng.uniform(2.5, 6.0)
    a = [a1,
         rng.uniform(-1e-3, 1e-3),
         rng.uniform(-1e-6, 1e-6),
         rng.uniform(-1e-9, 1e-9),
         rng.uniform(-1e-12, 1e-12)]
    a6 = sum(n * h_el[el] for el, n in zip(ELEMENTS, comp)) + rng.uniform(-500.0, 500.0)
    a7 = (sum(n * s_el[el] for el, n in zip(ELEMENTS, comp)) - a1 * (math.log(T_REF_THERMO) - 1.0)
          + rng.uniform(-1.0, 1.0))
    return [float(x) for x in a] + [float(a6), float(a7)]


# ---------------------------------------------------------------------------
# reactions
# ---------------------------------------------------------------------------

def _arrhenius(rng):
    """(A_ref, b, Ea): A_ref ~ log-U(1e6, 1e14) is the bimolecular-equivalent
    rate coefficient (cm^3/mol/s) at T_REF_RATE and P_ATM; b ~ U(-1, 2);
    Ea ~ U(0, 40) kcal/mol, stored in cal/mol.  ``_chemkin_A`` turns A_ref into
    the CHEMKIN pre-exponential factor of the reaction's order."""
    a_ref = 10.0 ** rng.uniform(6.0, 14.0)
    b = rng.uniform(-1.0, 2.0)
    ea = rng.uniform(0.0, 40000.0)
    return (float(a_ref), float(b), float(ea))


def _chemkin_A(a_ref, b, order):
    """CHEMKIN A (cm-mol-s, reaction order ``order``) such that A T^b C_ref^(order-2)
    equals a_ref at T = T_REF_RATE, C_ref = P_ATM/(R T_REF_RATE) in mol/cm^3."""
    c_ref = P_ATM / (R_GAS * T_REF_RATE) * 1e-6
    return float(a_ref * c_ref ** (2 - order) / T_REF_RATE ** b)


class _Builder:
    def __init__(self, cfg: MechConfig, rng):
        self.cfg = cfg
        self.rng = rng
        self.comps: List[tuple] = []
        self.names: List[str] = []
        self.is_qss: List[bool] = []
        self.reactions: List[dict] = []
        self.keys = set()

    # index helpers -------------------------------------------------------
    def non_qss(self):
        return [i for i, q in enumerate(self.is_qss) if not q and self.names[i] != "N2"]

    def build_pair_index(self, pool):
        idx: Dict[tuple, List[tuple]] = {}
        for a_pos, a in enumerate(pool):
            idx.setdefault(self.comps[a], []).append((a,))
            for b in pool[a_pos:]:
                idx.setdefault(_comp_add(self.comps[a], self.comps[b]), []).append((a, b))
        return idx

    def key(self, lhs, rhs):
        l = tuple(sorted(lhs))
        r = tuple(sorted(rhs))
        return (l, r) if l <= r else (r, l)

    def add(self, lhs, rhs, reversible, kind="plain", allow_dup=False):
        k = self.key(lhs, rhs)
        if k in self.keys and not allow_dup:
            return False
        if sorted(lhs) == sorted(rhs):
            return False
        self.keys.add(k)
        A, b, Ea = _arrhenius(self.rng)
        rxn = {"lhs": list(lhs), "rhs": list(rhs), "reversible": bool(reversible),
               "A": A, "b": b, "Ea": Ea, "kind": kind, "duplicate": False}
        self.reactions.append(rxn)
        return True


def _qss_count(b: _Builder, side):
    return sum(1 for s in side if b.is_qss[s])


def _find_link(b: _Builder, qa, qb, pair_idx_nonqss):
    """Balanced reactions with QSS ``qa`` on the left and QSS ``qb`` on the
    right, every other participant transported:
    qa + X -> qb + Y,  qa + X -> qb,  qa -> qb + Y."""
    opts = []
    by_comp = {b.comps[i]: i for i in b.non_qss()}
    for x in b.non_qss():
        tot = _comp_add(b.comps[qa], b.comps[x])
        rest = _comp_sub(tot, b.comps[qb])
        if all(v == 0 for v in rest):
            opts.append(([qa, x], [qb]))
        elif rest in by_comp:
            opts.append(([qa, x], [qb, by_comp[rest]]))
    rest = _comp_sub(b.comps[qa], b.comps[qb])
    if rest in by_comp:
        opts.append(([qa], [qb, by_comp[rest]]))
    return opts


def _find_with_one_qss(b: _Builder, q, pair_idx_nonqss, side="rhs"):
    """Balanced reactions with ``q`` on one side and only transported species
    elsewhere: (X [+ X']) -> q [+ Y]."""
    opts = []
    nq = b.non_qss()
    for y in [None] + nq:
        tot = b.comps[q] if y is None else _comp_add(b.comps[q], b.comps[y])
        for pair in pair_idx_nonqss.get(tot, []):
            lhs = list(pair)
            rhs = [q] + ([y] if y is not None else [])
            if len(lhs) + len(rhs) < 3 and len(lhs) == 1 and y is None:
                continue
            opts.append((lhs, rhs))
    return opts


def generate_mechanism(cfg: MechConfig) -> dict:
    """Build one seeded synthetic QSS mechanism."""
    for attempt in range(200):
        rng = np.random.default_rng([cfg.seed, attempt])
        try:
            return _generate(cfg, rng)
        except RuntimeError:
            continue
    raise RuntimeError(f"mechanism generation failed for {cfg.name}")


def _generate(cfg: MechConfig, rng) -> dict:
    b = _Builder(cfg, rng)
    N, Q = cfg.n_transported, cfg.n_qss
    taken = set()
    core = CORE_SPECIES[:min(len(CORE_SPECIES), max(N - 1, 7))]
    for nm, c in core:
        b.comps.append(c)
        b.names.append(nm)
        b.is_qss.append(False)
        taken.add(c)
    extra_t = N - len(core)
    starts = [c for _, c in core if c[3] == 0]
    for c in _grow_species(rng, starts, max(extra_t, 0), taken, cfg.max_carbon):
        b.comps.append(c)
        b.names.append(_comp_name(c))
        b.is_qss.append(False)
    b.comps = b.comps[:N]
    b.names = b.names[:N]
    b.is_qss = b.is_qss[:N]
    # QSS species grow from transported compositions (radical-like relatives)
    qcomps = _grow_species(rng, [c for c in b.comps if c[3] == 0], Q, taken, cfg.max_carbon)
    for c in qcomps:
        b.comps.append(c)
        b.names.append(_comp_name(c) + "_q")
        b.is_qss.append(True)
    n_sp = N + Q
    qss_ids = list(range(N, n_sp))

    pool = b.non_qss()
    pidx = b.build_pair_index(pool)

    # --- feasibility of QSS -> QSS links -----------------------------------
    link = {}
    for qa in qss_ids:
        for qb in qss_ids:
            if qa != qb:
                o = _find_link(b, qa, qb, pidx)
                if o:
                    link[(qa, qb)] = o
    # --- assign QSS species to planned groups ----------------------------
    groups = _assign_groups(rng, cfg.qss_groups, qss_ids, link)
    group_of = {}
    for gi, g in enumerate(groups):
        for s in g:
            group_of[s] = gi

    # --- structural reactions --------------------------------------------
    # (1) chains inside each group: reversible links make the group strongly
    #     connected (a reversible QSS-QSS reaction gives edges both ways).
    for g in groups:
        for a, c in zip(g[:-1], g[1:]):
            opts = link.get((a, c)) or [(r, l) for (l, r) in link.get((c, a), [])]
            lhs, rhs = opts[rng.integers(len(opts))]
            if not b.add(lhs, rhs, True, "plain"):
                raise RuntimeError("duplicate structural link")
    # (2) acyclic edges between groups (irreversible, earlier group -> later)
    n_cross = 0
    if not cfg.all_reversible and len(groups) > 1:
        want = max(1, len(groups) - 1)
        pairs = [(x, y) for (x, y) in link if group_of[x] < group_of[y]]
        rng.shuffle(pairs)
        for (x, y) in pairs[: 3 * want]:
            if n_cross >= want:
                break
            opts = link[(x, y)]
            lhs, rhs = opts[rng.integers(len(opts))]
            if b.add(lhs, rhs, False, "plain"):
                n_cross += 1
    # (3) every QSS species: production from transported species and a
    #     consumption channel to transported species only (reversible, so the
    #     same reaction serves both; this keeps -A strictly diagonally dominant)
    for q in qss_ids:
        opts = _find_with_one_qss(b, q, pidx)
        if not opts:
            raise RuntimeError("QSS species without transported-only channel")
        rng.shuffle(opts)
        added = 0
        for lhs, rhs in opts:
            if b.add(lhs, rhs, True, "plain"):
                added += 1
                if added >= 2:
                    break
        if added == 0:
            raise RuntimeError("no channel")

    # --- third-body and falloff reactions (recombination form) -------------
    recomb = []
    for c_id in range(n_sp):
        if b.names[c_id] == "N2":
            continue
        for pair in pidx.get(b.comps[c_id], []):
            if len(pair) == 2:
                recomb.append((list(pair), [c_id]))
    # pairs may include one QSS species on the product side only
    rng.shuffle(recomb)
    need = cfg.n_third_body + cfg.n_troe
    picked = []
    for lhs, rhs in recomb:
        if len(picked) >= need:
            break
        if _qss_count(b, lhs) > 1 or _qss_count(b, rhs) > 1:
            continue
        k = b.key(lhs, rhs)
        if k in b.keys:
            continue
        b.keys.add(k)
        picked.append((lhs, rhs))
    if len(picked) < need:
        raise RuntimeError("not enough recombination reactions")
    for i, (lhs, rhs) in enumerate(picked):
        A, bb, Ea = _arrhenius(rng)
        kind = "troe" if i < cfg.n_troe else "tb"
        b.reactions.append({"lhs": lhs, "rhs": rhs, "reversible": True, "A": A, "b": bb,
                            "Ea": Ea, "kind": kind, "duplicate": False})

    # --- fill with elementary reactions ------------------------------------
    n_dup_pairs = int(round(cfg.dup_fraction * cfg.n_reactions / 2.0))
    target_plain = cfg.n_reactions - n_dup_pairs - len(b.reactions)
    if target_plain < 0:
        raise RuntimeError("too many structural reactions")
    qss_opts = []
    for q in qss_ids:
        qss_opts += _find_with_one_qss(b, q, pidx)
    plain_opts = []
    for tot, pairs in pidx.items():
        if len(pairs) >= 2:
            for i in range(len(pairs)):
                for j in range(i + 1, len(pairs)):
                    if len(pairs[i]) + len(pairs[j]) >= 3:
                        plain_opts.append((list(pairs[i]), list(pairs[j])))
    added = 0
    guard = 0
    while added < target_plain and guard < 200000:
        guard += 1
        use_q = rng.random() < cfg.qss_reaction_fraction and qss_opts
        src = qss_opts if use_q else plain_opts
        if not src:
            src = qss_opts or plain_opts
        lhs, rhs = src[rng.integers(len(src))]
        if rng.random() < 0.5:
            lhs, rhs = rhs, lhs
        rev = True if cfg.all_reversible else (rng.random() < 0.85)
        if b.add(lhs, rhs, rev, "plain"):
            added += 1
    if added < target_plain:
        raise RuntimeError("not enough elementary reactions")
    # --- duplicate pairs: same stoichiometry, independent rate parameters ----
    plain_ids = [i for i, r in enumerate(b.reactions) if r["kind"] == "plain"]
    rng.shuffle(plain_ids)
    for i in plain_ids[:n_dup_pairs]:
        r = b.reactions[i]
        r["duplicate"] = True
        A, bb, Ea = _arrhenius(rng)
        b.reactions.append({"lhs": list(r["lhs"]), "rhs": list(r["rhs"]),
                            "reversible": r["reversible"], "A": A, "b": bb, "Ea": Ea,
                            "kind": "plain", "duplicate": True})
    if len(b.reactions) != cfg.n_reactions:
        raise RuntimeError("reaction count mismatch")

    # --- shuffle reaction order, assemble the dictionary --------------------
    order = rng.permutation(len(b.reactions))
    species = []
    for i in range(n_sp):
        nasa = _nasa(rng, b.comps[i])
        species.append({"name": b.names[i], "W": _weight(b.comps[i]),
                        "composition": {el: int(n) for el, n in zip(ELEMENTS, b.comps[i]) if n},
                        "qss": bool(b.is_qss[i]), "nasa_lo": nasa, "nasa_hi": list(nasa),
                        "Tmid": 1000.0})
    transported = [b.names[i] for i in range(N)]
    reactions = []
    for oi in order:
        r = b.reactions[int(oi)]
        reac, prod = {}, {}
        for s in r["lhs"]:
            reac[b.names[s]] = reac.get(b.names[s], 0) + 1
        for s in r["rhs"]:
            prod[b.names[s]] = prod.get(b.names[s], 0) + 1
        order = len(r["lhs"]) + (1 if r["kind"] == "tb" else 0)
        d = {"reactants": reac, "products": prod, "reversible": r["reversible"],
             "A": _chemkin_A(r["A"], r["b"], order), "b": r["b"], "Ea": r["Ea"], "third_body": None,
             "falloff": None, "duplicate": r["duplicate"]}
        if r["kind"] in ("tb", "troe"):
            k = int(rng.integers(3, 7))
            chosen = rng.choice(len(transported), size=min(k, len(transported)), replace=False)
            eff = {transported[int(c)]: float(rng.uniform(0.5, 3.0)) for c in sorted(chosen)}
            d["third_body"] = {"efficiencies": eff}
        if r["kind"] == "troe":
            # low-pressure limit: A0 = A_inf 10^U(2,6) in CHEMKIN units (one more
            # order), both referred to T_REF_RATE
            b0 = float(rng.uniform(-2.0, 0.0))
            a0_at_ref = d["A"] * T_REF_RATE ** d["b"] * 10.0 ** rng.uniform(2.0, 6.0)
            d["falloff"] = {
                "low": {"A": float(a0_at_ref / T_REF_RATE ** b0), "b": b0,
                        "Ea": float(rng.uniform(0.0, 0.8) * d["Ea"])},
                "troe": [float(rng.uniform(0.1, 0.9)), float(rng.uniform(50.0, 500.0)),
                         float(rng.uniform(500.0, 3000.0)), float(rng.uniform(3000.0, 8000.0))]}
        reactions.append(d)
    mech = {"name": cfg.name, "seed": cfg.seed,
            "units": {"A": "cm-mol-s", "Ea": "cal/mol"},
            "elements": list(ELEMENTS), "species": species, "reactions": reactions,
            "planned_qss_groups": [[b.names[s] for s in g] for g in groups]}
    return mech


def _assign_groups(rng, sizes, qss_ids, link):
    """Partition QSS species into chains of the requested sizes such that
    consecutive members have a balanced linking reaction (either direction)."""
    sizes = sorted(sizes, reverse=True)
    assert sum(sizes) == len(qss_ids)

    def linked(a, c):
        return (a, c) in link or (c, a) in link

    for _ in range(500):
        free = list(qss_ids)
        rng.shuffle(free)
        groups = []
        ok = True
        for sz in sizes:
            if sz == 1:
                groups.append([free.pop()])
                continue
            chain = None
            for start in list(free):
                path = [start]
                avail = [x for x in free if x != start]
                while len(path) < sz:
                    nxt = [x for x in avail if linked(path[-1], x)]
                    if not nxt:
                        break
                    x = nxt[rng.integers(len(nxt))]
                    path.append(x)
                    avail.remove(x)
                if len(path) == sz:
                    chain = path
                    break
            if chain is None:
                ok = False
                break
            for x in chain:
                free.remove(x)
            groups.append(chain)
        if ok:
            order = rng.permutation(len(groups))
            return [groups[int(i)] for i in order]
    raise RuntimeError("could not place QSS groups")


# ---------------------------------------------------------------------------
# states
# ---------------------------------------------------------------------------

def add_quadratic_couplings(mech: dict, n_couplings: int, seed: int) -> dict:
    """A copy of ``mech`` with ``n_couplings`` extra reactions whose rates are
    products of QSS concentrations (Section 2.2's quadratic couplings), as a
    synthetic stand-in for QSS mechanisms that need linearization.

    Kinds, in turn: q_a + q_b <=> X + Y (forward coupled), X + Y <=> q_a + q_b
    (reverse coupled), 2 q_a -> X (irreversible, forward coupled), and
    q_a + q_b <=> q_c + q_d (both directions coupled).  Reversible reactions
    are atom balanced (products found among species of the same total
    composition); where no balanced partner exists the reaction is made
    irreversible, which needs no equilibrium constant.  Rate parameters are
    drawn like the others' (bimolecular)."""
    import copy
    rng = np.random.default_rng(seed)
    out = copy.deepcopy(mech)
    sp = out["species"]
    comp = {x["name"]: tuple(x["composition"].get(e, 0) for e in ELEMENTS) for x in sp}
    qss = [x["name"] for x in sp if x["qss"]]
    tr = [x["name"] for x in sp if not x["qss"]]
    pairs_tr = {}
    for i, a in enumerate(tr):
        for b_ in tr[i:]:
            pairs_tr.setdefault(tuple(u + v for u, v in zip(comp[a], comp[b_])), []).append((a, b_))
    pairs_q = {}
    for i, a in enumerate(qss):
        for b_ in qss[i + 1:]:
            pairs_q.setdefault(tuple(u + v for u, v in zip(comp[a], comp[b_])), []).append((a, b_))

    def side(names):
        d = {}
        for x in names:
            d[x] = d.get(x, 0) + 1
        return d

    added = 0
    tries = 0
    while added < n_couplings and tries < 1000 * max(n_couplings, 1):
        tries += 1
        kind = added % 4
        qa, qb = (str(x) for x in rng.choice(qss, size=2, replace=False))
        key = tuple(u + v for u, v in zip(comp[qa], comp[qb]))
        if kind == 2:
            lhs, rhs, rev = [qa, qa], [str(rng.choice(tr))], False
        elif kind == 3:
            cand = [p for p in pairs_q.get(key, []) if set(p) != {qa, qb}]
            if not cand:
                continue
            lhs, rhs, rev = [qa, qb], list(cand[int(rng.integers(len(cand)))]), True
        else:
            cand = pairs_tr.get(key, [])
            if cand:
                prod, rev = list(cand[int(rng.integers(len(cand)))]), True
            else:
                prod, rev = [str(x) for x in rng.choice(tr, size=2, replace=False)], False
            lhs, rhs = ([qa, qb], prod) if (kind == 0 or not rev) else (prod, [qa, qb])
        a_ref, b, ea = _arrhenius(rng)
        out["reactions"].append({"reactants": side(lhs), "products": side(rhs), "reversible": rev,
                                 "A": _chemkin_A(a_ref, b, 2), "b": b, "Ea": ea, "third_body": None,
                                 "falloff": None, "duplicate": False})
        added += 1
    out["name"] = f"{mech.get('name', 'mech')}_quad{added}"
    return out


def transported_species(mech):
    return [s for s in mech["species"] if not s["qss"]]


def generate_states(mech: dict, scfg: StateConfig, ncells: int, ld: Optional[int] = None):
    """Seeded (rho, T, Y) in SoA layout with leading dimension ``ld``.

    Padding columns (c >= ncells) hold a benign copy of cell 0 so that a
    kernel reading them by mistake still sees finite numbers."""
    rng = np.random.default_rng(scfg.seed)
    sp = transported_species(mech)
    N = len(sp)
    W = np.array([s["W"] for s in sp])
    if ld is None:
        ld = ncells
    T = rng.uniform(scfg.T_range[0], scfg.T_range[1], size=ncells)
    if scfg.P_log_uniform:
        P = np.exp(rng.uniform(math.log(scfg.P_range_atm[0]), math.log(scfg.P_range_atm[1]),
                               size=ncells)) * P_ATM
    else:
        P = rng.uniform(scfg.P_range_atm[0], scfg.P_range_atm[1], size=ncells) * P_ATM
    Y = rng.dirichlet(np.full(N, scfg.dirichlet_alpha), size=ncells)  # [ncells][N]
    if scfg.near_pure_fraction > 0:
        names = [s["name"] for s in sp]
        fuel = int(np.argmax(W * np.array([s["composition"].get("C", 0) for s in sp])))
        air = np.zeros(N)
        air[names.index("O2")] = 0.233
        air[names.index("N2")] = 0.767
        fuel_v = np.zeros(N)
        fuel_v[fuel] = 1.0
        pure_mask = rng.random(ncells) < scfg.near_pure_fraction
        which = rng.random(ncells) < 0.5
        noise = rng.dirichlet(np.full(N, scfg.dirichlet_alpha), size=ncells)
        for c in np.nonzero(pure_mask)[0]:
            base = fuel_v if which[c] else air
            Y[c] = (1.0 - 1e-6) * base + 1e-6 * noise[c]
    Wmix = 1.0 / (Y / W[None, :]).sum(axis=1)
    rho = P * Wmix / (R_GAS * T)
    rho_o = np.empty(ld)
    T_o = np.empty(ld)
    Y_o = np.empty((N, ld))
    rho_o[:ncells] = rho
    T_o[:ncells] = T
    Y_o[:, :ncells] = Y.T
    if ld > ncells and ncells > 0:
        rho_o[ncells:] = rho[0]
        T_o[ncells:] = T[0]
        Y_o[:, ncells:] = Y[0][:, None]
    return rho_o, T_o, Y_o


def concentrations_to_state(mech, C, T):
    """(C [N][n] mol/m^3, T) -> (rho, T, Y) so that rho*Y_k/W_k = C_k.
    Used for the paper's concentration-space sampling protocols."""
    sp = transported_species(mech)
    W = np.array([s["W"] for s in sp])[:, None]
    mass = C * W
    rho = mass.sum(axis=0)
    Y = mass / rho[None, :]
    return rho, np.asarray(T, dtype=np.float64).copy(), Y


def save_mech(mech: dict, path: str):
    with open(path, "w") as f:
        json.dump(mech, f, indent=1, sort_keys=True)


def load_mech(path: str) -> dict:
    with open(path) as f:
        return json.load(f)
