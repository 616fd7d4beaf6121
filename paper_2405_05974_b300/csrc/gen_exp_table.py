"""Write qss_exp_table.inc: constants of the table-driven exponential.

Tang's method (P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989) with a
2048-entry table (16 KB, L1-resident): x = (2048 k + j) ln2/2048 + r,
exp(x) = 2^k 2^(j/2048) exp(r), |r| <= ln2/4096, so that a cubic in r suffices.
Values are computed here in 60-digit decimal arithmetic and rounded once to
binary64.

    python paper_2405_05974_b300/csrc/gen_exp_table.py
"""
import math
import os
from decimal import Decimal, getcontext

getcontext().prec = 60
L = 2048
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
    # |n| < 2^21 on the fast path (|x| < 708), so n * hi is exact with 30 bits
    hi = hi_part(step, 30)
    lo = to_double(step - Decimal(hi))
    inv = to_double(L / LN2)
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "qss_exp_table.inc"), "w") as f:
        f.write(f"// Generated by gen_exp_table.py: 2^(j/{L}), j = 0..{L - 1}, and the split of ln2/{L}.\n")
        f.write(f"#define QSS_EXP_L {L}\n")
        f.write(f"#define QSS_EXP_INV_STEP {inv!r}\n")
        f.write(f"#define QSS_EXP_STEP_HI {hi!r}\n")
        f.write(f"#define QSS_EXP_STEP_LO {lo!r}\n")
        f.write(f"__device__ const double qss_exp2_tab[{L}] = {{\n")
        for i in range(0, L, 4):
            f.write("  " + ", ".join(repr(v) for v in tab[i:i + 4]) + ",\n")
        f.write("};\n")


if __name__ == "__main__":
    main()
