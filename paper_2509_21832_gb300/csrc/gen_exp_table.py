"""Write mm_exp_table.inc: the constants of the table-driven exponential used in the micro
kernels (P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
floating-point arithmetic", ACM TOMS 15(2), 1989): exp(x) = 2^m 2^(j/64) exp(r) with
x = (64 m + j) ln2/64 + r, |r| <= ln2/128.

The 64 table entries 2^(j/64) and the two-part split of ln2/64 are computed with Python's
decimal module at 60 significant digits and rounded to the nearest double.
"""
import decimal
import math
import os

D = decimal.Decimal
decimal.getcontext().prec = 60


def dexp(x: D) -> D:
    # Taylor series, enough terms for 60 digits at |x| <= 1
    s, t, k = D(1), D(1), 1
    while True:
        t = t * x / k
        if abs(t) < D(10) ** -70:
            return s
        s += t
        k += 1


def dln2() -> D:
    # ln 2 = sum_{k>=1} 1 / (k 2^k)
    s, k = D(0), 1
    while True:
        t = D(1) / (k * D(2) ** k)
        if t < D(10) ** -70:
            return s
        s += t
        k += 1


def hexd(x: D) -> str:
    return float(x).hex()


def main():
    ln2 = dln2()
    step = ln2 / 64
    # high part with 32 significant bits so that n * L1 is exact for |n| < 2^21
    hi = float(step)
    mant, ex = math.frexp(hi)
    hi = math.ldexp(math.floor(mant * 2 ** 32) / 2 ** 32, ex)
    lo = float(step - D(hi))
    inv = float(D(64) / ln2)
    lines = ["// Generated by gen_exp_table.py: constants of the table-driven exponential.",
             "// kExpInvL = 64/ln2, kExpL1 + kExpL2 = ln2/64 (kExpL1 has 32 significant bits),",
             "// kExpTab[j] = 2^(j/64) rounded to nearest.",
             "constexpr double kExpInvL = %s;" % inv.hex(),
             "constexpr double kExpL1 = %s;" % hi.hex(),
             "constexpr double kExpL2 = %s;" % lo.hex(),
             "static __device__ const double kExpTab[64] = {"]
    for j in range(64):
        lines.append("    %s," % hexd(dexp(D(j) * ln2 / 64)))
    lines.append("};")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mm_exp_table.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
