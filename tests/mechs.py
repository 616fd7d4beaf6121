"""Hand-built mechanisms with closed-form answers (test inputs only)."""
import math

R = 8.31446261815324
CAL = 4.184
P0 = 101325.0


def species(name, comp, qss=False, nasa=None, W=None):
    nasa = list(nasa) if nasa is not None else [2.5, 0, 0, 0, 0, 0.0, 0.0]
    if W is None:
        aw = {"C": 12.011e-3, "H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}
        W = sum(aw[e] * n for e, n in comp.items())
    return {"name": name, "W": W, "composition": comp, "qss": qss, "nasa_lo": nasa,
            "nasa_hi": list(nasa), "Tmid": 1000.0}


def reaction(reac, prod, A, b=0.0, Ea=0.0, reversible=True, third_body=None, falloff=None):
    return {"reactants": reac, "products": prod, "reversible": reversible, "A": A, "b": b, "Ea": Ea,
            "third_body": third_body, "falloff": falloff, "duplicate": False}


def mech(name, sp, rx):
    tr = [s for s in sp if not s["qss"]]
    qs = [s for s in sp if s["qss"]]
    return {"name": name, "seed": -1, "units": {"A": "cm-mol-s", "Ea": "cal/mol"},
            "elements": ["C", "H", "O", "N"], "species": tr + qs, "reactions": rx}


def nasa_only(k, value, base=None):
    """NASA-7 set with coefficient k (1-based) = value, others zero (or base)."""
    a = list(base) if base is not None else [0.0] * 7
    a[k - 1] = value
    return a


def g_over_RT_single(k, a, T):
    """Closed form of g/RT = h/RT - s/R when only NASA coefficient k is nonzero."""
    lnT = math.log(T)
    return {1: a * (1.0 - lnT), 2: -a * T / 2.0, 3: -a * T ** 2 / 6.0, 4: -a * T ** 3 / 12.0,
            5: -a * T ** 4 / 20.0, 6: a / T, 7: -a}[k]
