"""CPU emulation of the device exponential, logarithm and reciprocal (qss_device.cuh):
the same operations in the same order on binary64 values, each fma rounded
once (exact rationals), with the table and constants read from the generated
qss_exp_table.inc.  Pins the algorithms and their constants without a GPU:
results within one ulp of the exact values."""
import math
import os
import random
import re
import struct
from decimal import Decimal, getcontext
from fractions import Fraction

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2405_05974_b300", "csrc")


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def ulps(y, exact):
    return abs(y - exact) / math.ulp(abs(exact))


def small_int_to_double(n):
    """qss_small_int_to_double: the float of n (exact for |n| < 2^24) widened
    to binary64 by integer operations on its fields."""
    fb = struct.unpack("<I", struct.pack("<f", float(n)))[0]
    hi = (fb & 0x80000000) | (((fb & 0x7fffffff) >> 3) + 0x38000000)
    hi = hi if fb else 0
    lo = (fb << 29) & 0xffffffff
    return struct.unpack("<d", struct.pack("<Q", (hi << 32) | lo))[0]


def test_small_int_to_double_exact():
    rng = random.Random(11)
    ns = list(range(-70000, 70000)) + [rng.randrange(-(1 << 24) + 1, 1 << 24) for _ in range(20000)]
    ns += [(1 << k) + d for k in range(24) for d in (-1, 0, 1)] + [-(1 << 24) + 1, (1 << 24) - 1]
    for n in ns:
        y = small_int_to_double(n)
        assert y == float(n) and math.copysign(1.0, y) == (-1.0 if n < 0 else 1.0), n


def _exp_table():
    src = open(os.path.join(CSRC, "qss_exp_table.inc")).read()
    const = dict(re.findall(r"#define (QSS_EXP_\w+) (\S+)", src))
    body = src[src.index("{") + 1:src.rindex("}")]
    tab = [float(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    return int(const["QSS_EXP_L"]), float(const["QSS_EXP_INV_STEP"]), float(const["QSS_EXP_STEP_HI"]), \
        float(const["QSS_EXP_STEP_LO"]), tab


def exp_emulated(x, L, inv, hi, lo, tab):
    shifter = 6755399441055744.0
    t = fma(x, inv, shifter)
    n = struct.unpack("<q", struct.pack("<d", t))[0] & 0xffffffff
    n = n - (1 << 32) if n >= 1 << 31 else n
    nd = small_int_to_double(n)
    assert nd == t - shifter
    r = fma(-nd, hi, x)
    r = fma(-nd, lo, r)
    p = fma(r, 1.0 / 6.0, 0.5)
    p = fma(p, r, 1.0)
    q = p * r
    tj = tab[n & (L - 1)]
    return math.ldexp(fma(tj, q, tj), n >> int(math.log2(L)))


def test_exp_table_constants():
    getcontext().prec = 60
    L, inv, hi, lo, tab = _exp_table()
    assert L == len(tab) and L & (L - 1) == 0
    ln2 = Decimal(2).ln()
    for j in range(0, L, 97):
        assert tab[j] == float((Decimal(j) * ln2 / L).exp())
    # n * hi exact for |n| < 2^21 (the fast path's |x| < 708)
    m, _ = math.frexp(hi)
    assert (Fraction(m) * 2 ** 31).denominator == 1
    assert abs(Decimal(hi) + Decimal(lo) - ln2 / L) < Decimal(2) ** -90


def test_exp_within_one_ulp():
    getcontext().prec = 50
    L, inv, hi, lo, tab = _exp_table()
    rng = random.Random(5)
    xs = [rng.uniform(-707.0, 707.0) for _ in range(800)] + [rng.uniform(-1.0, 1.0) for _ in range(800)]
    xs += [(k + 0.5) * math.log(2) / L for k in range(-2000, 2000, 9)] + [0.0, 1e-300, -1e-300]
    for x in xs:
        assert ulps(exp_emulated(x, L, inv, hi, lo, tab), float(Decimal(x).exp())) <= 1.0, x


def rcp_emulated(x, seed_ulps=0):
    """qss_rcp's fast path; the rcp.approx.f32 seed is taken as the correctly
    rounded float reciprocal moved by seed_ulps float ulps (the instruction's
    documented error is at most one ulp)."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    hx = b >> 32
    eb = (hx >> 20) & 0x7ff
    assert 1 <= eb <= 0x7fc
    f = struct.unpack("<f", struct.pack("<I", 0x3f800000 | ((hx & 0xfffff) << 3)))[0]
    r = struct.unpack("<f", struct.pack("<f", 1.0 / f))[0]
    rb = struct.unpack("<I", struct.pack("<f", r))[0] + seed_ulps
    yhi = (hx & 0x80000000) | ((rb >> 3) + ((1919 - eb) << 20)) & 0xffffffff
    y0 = struct.unpack("<d", struct.pack("<Q", (yhi << 32) | ((rb << 29) & 0xffffffff)))[0]
    e = fma(-x, y0, 1.0)
    return fma(y0, fma(e, e, e), y0)


@pytest.mark.parametrize("seed_ulps", [-1, 0, 1])
def test_rcp_within_one_ulp(seed_ulps):
    rng = random.Random(6 + seed_ulps)
    xs = [math.ldexp(rng.uniform(1.0, 2.0), rng.randint(-1021, 1020)) * rng.choice((1, -1)) for _ in range(3000)]
    xs += [1.0, 3.0, math.nextafter(2.0, 0.0), math.nextafter(1.0, 2.0), 2.0 ** 1021, 2.0 ** -1022]
    exact_hits = 0
    for x in xs:
        y = rcp_emulated(x, seed_ulps)
        exact = float(Fraction(1) / Fraction(x))
        assert ulps(y, exact) <= 1.0, x
        exact_hits += y == exact
    assert exact_hits >= 0.99 * len(xs)


def _log_table():
    src = open(os.path.join(CSRC, "qss_log_table.inc")).read()
    base = int(re.search(r"#define QSS_LOG_BASE_BITS (0x[0-9a-f]+)LL", src).group(1), 16)
    ln2hi = float(re.search(r"#define QSS_LOG_LN2_HI (\S+)", src).group(1))
    ln2lo = float(re.search(r"#define QSS_LOG_LN2_LO (\S+)", src).group(1))
    rows = re.findall(r"\{([^{}]+)\}", src[src.index("qss_log_tab"):])
    tab = [tuple(float(v) for v in row.split(",")) for row in rows]
    return base, ln2hi, ln2lo, tab


def log_emulated(x, base, ln2hi, ln2lo, tab):
    xb = struct.unpack("<q", struct.pack("<d", x))[0]
    off = xb - base
    m = off >> 52
    y = struct.unpack("<d", struct.pack("<q", xb - (m << 52)))[0]
    j = (off >> 44) & 255
    c, lhi, llo = tab[j]
    r = fma(y, c, -1.0)
    r2 = r * r
    q = fma(r, 1.0 / 7.0, -1.0 / 6.0)
    q = fma(q, r, 1.0 / 5.0)
    q = fma(q, r, -0.25)
    q = fma(q, r, 1.0 / 3.0)
    q = fma(q, r, -0.5)
    p = fma(r2, q, r)
    md = small_int_to_double(m)
    assert md == float(m)
    head = fma(md, ln2hi, lhi)
    tail = fma(md, ln2lo, llo) + p
    return head + tail


def test_log_within_one_ulp():
    getcontext().prec = 50
    base, ln2hi, ln2lo, tab = _log_table()
    assert len(tab) == 256
    rng = random.Random(7)
    xs = [math.exp(rng.uniform(-700.0, 700.0)) for _ in range(800)] + [rng.uniform(200.0, 5000.0) for _ in range(800)]
    xs += [1.0 + rng.uniform(-1e-3, 1e-3) for _ in range(400)] + [1.0, 2.0, 0.5, math.sqrt(0.5), math.nextafter(1.0, 0.0)]
    for x in xs:
        exact = float(Decimal(x).ln())
        y = log_emulated(x, base, ln2hi, ln2lo, tab)
        if exact == 0.0:
            assert y == 0.0
        else:
            assert ulps(y, exact) <= 1.0, x
