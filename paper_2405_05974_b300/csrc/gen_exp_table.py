"""Write qss_exp_table.inc: constants of the table-driven exponential.

Tang's method (P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989) with a
256-entry table: x = (256 k + j) ln2/256 + r, exp(x) = 2^k 2^(j/256) exp(r).
Values are computed here in 60-digit decimal arithmetic and rounded once to
binary64.

    python paper_2405_05974_b300/csrc/gen_exp_table.py
"""
import math
import os
from decimal import Decimal, getcontext

getcontext().prec = 60
L = 256
LN2 = Decimal(2).ln()


def to_double(d: Decimal) -> float:
    return float(d)  # correctly rounded conversion


def hi_part(v: Decimal, bits: int) -> float:
    """v rounded to a binary64 with at most `bits` significant bits."""
    m, e = math.frexp(to_double(v))
    scale = 2.0 ** bits
    return math.ldexp(round(m * scale) / scale, e)


def main():
    tab = [to_double((Decimal(j) * LN2 / L).exp()) for j in range(L)]
    step = LN2 / L
    hi = hi_part(step, 32)
    lo = to_double(step - Decimal(hi))
    inv = to_double(L / LN2)
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "qss_exp_table.inc"), "w") as f:
        f.write("// Generated by gen_exp_table.py: 2^(j/256), j = 0..255, and the split of ln2/256.\n")
        f.write(f"#define QSS_EXP_INV_STEP {inv!r}\n")
        f.write(f"#define QSS_EXP_STEP_HI {hi!r}\n")
        f.write(f"#define QSS_EXP_STEP_LO {lo!r}\n")
        f.write("__device__ const double qss_exp2_tab[256] = {\n")
        for i in range(0, L, 4):
            f.write("  " + ", ".join(repr(v) for v in tab[i:i + 4]) + ",\n")
        f.write("};\n")


if __name__ == "__main__":
    main()
