"""The polynomial of the KFVS half fluxes' erf (paper_2509_21832_gb300/csrc/mm_erf_poly.inc):
the committed coefficients are the generator's, and x P(x^2) evaluated in double by Horner's
rule agrees with the C library's erf on |x| < 1.5 (CPU)."""
import math
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2509_21832_gb300", "csrc")


def committed():
    txt = open(os.path.join(CSRC, "mm_erf_poly.inc")).read()
    vals = [float.fromhex(v) for v in re.findall(r"(-?0x[0-9a-fp.+-]+)", txt)]
    return vals[::-1]  # Horner runs from the highest power down: s^0 .. s^14 after reversal


def test_committed_coefficients_are_the_generators():
    sys.path.insert(0, CSRC)
    try:
        import gen_erf_poly as gen
    finally:
        sys.path.pop(0)
    assert committed() == [float(c) for c in gen.coefficients()]


def test_polynomial_matches_library_erf():
    c = committed()
    assert len(c) == 15 and abs(c[0] - 2.0 / math.sqrt(math.pi)) < 1e-16
    worst = 0.0
    for i in range(-3000, 3001):
        x = 1.4999 * i / 3000
        if x == 0.0:
            continue
        s = x * x
        p = c[-1]
        for v in reversed(c[:-1]):
            p = p * s + v
        worst = max(worst, abs(x * p - math.erf(x)) / abs(math.erf(x)))
    assert worst < 6e-16, worst
