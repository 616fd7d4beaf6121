"""Write qss_log_table.inc: constants of the table-driven natural logarithm.

Reduction in the spirit of Tang's table-driven logarithm (P. T. P. Tang,
"Table-driven implementation of the logarithm function in IEEE
floating-point arithmetic", ACM TOMS 16(4), 1990), with a reciprocal table
instead of a division:

    x = 2^m y,  y in [b, 2b),  b = sqrt(1/2) rounded down to a 2^-8 step of
    the binary64 significand;  y falls in one of 256 cells of equal width in
    the bit pattern, cell j starting at bits(b) + j 2^44;
    c_j ~ 1 / (centre of cell j) with at most 9 significant bits, so that
    r = y c_j - 1 is exact in binary64 (|r| < 2^-8);
    log x = m ln2 + (-log c_j) + log1p(r).

The two cells touching 1.0 use c_j = 1 (then -log c_j = 0 and r = y - 1
exactly), so that log x keeps full relative accuracy next to x = 1.  ln2 and
-log c_j are split into a head with 42 significant bits past the binary
point (m ln2_hi + L_hi is then exact for |m| < 2^10) and a binary64 tail.
Values are computed in 60-digit decimal arithmetic and rounded once.

    python paper_2405_05974_b300/csrc/gen_log_table.py
"""
import math
import os
import struct
from decimal import Decimal, getcontext

getcontext().prec = 60
NCELL = 256
SHIFT = 44                     # cell width in the bit pattern: 2^44 (8 significand bits)
HEAD_STEP = Decimal(2) ** -42  # heads are multiples of 2^-42


def bits(v: float) -> int:
    return struct.unpack("<q", struct.pack("<d", v))[0]


def from_bits(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def head(v: Decimal) -> float:
    return float((v / HEAD_STEP).to_integral_value() * HEAD_STEP)


def nine_bits(v: float) -> float:
    m, e = math.frexp(v)
    return math.ldexp(round(m * 512) / 512, e)


def main():
    base = bits(math.sqrt(0.5)) & ~((1 << SHIFT) - 1)
    one = bits(1.0)
    assert (one - base) % (1 << SHIFT) == 0
    j_one = (one - base) >> SHIFT
    c, Lhi, Llo = [], [], []
    for j in range(NCELL):
        lo = from_bits(base + (j << SHIFT))
        hi = from_bits(base + ((j + 1) << SHIFT))
        if j in (j_one - 1, j_one):
            cj = 1.0
        else:
            cj = nine_bits(2.0 / (lo + hi))
        L = -Decimal(cj).ln()
        h = head(L)
        c.append(cj)
        Lhi.append(h)
        Llo.append(float(L - Decimal(h)))
    ln2 = Decimal(2).ln()
    ln2_hi = head(ln2)
    ln2_lo = float(ln2 - Decimal(ln2_hi))
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "qss_log_table.inc"), "w") as f:
        f.write("// Generated by gen_log_table.py: reciprocal table of the table-driven log.\n")
        f.write(f"#define QSS_LOG_BASE_BITS 0x{base:016x}LL\n")
        f.write(f"#define QSS_LOG_LN2_HI {ln2_hi!r}\n")
        f.write(f"#define QSS_LOG_LN2_LO {ln2_lo!r}\n")
        f.write("// per cell j: c_j, then -log(c_j) as head + tail\n")
        f.write("__device__ const double qss_log_tab[256][3] = {\n")
        for j in range(NCELL):
            f.write(f"  {{{c[j]!r}, {Lhi[j]!r}, {Llo[j]!r}}},\n")
        f.write("};\n")


if __name__ == "__main__":
    main()
