"""Writes ss_same_centre.txt: (ss|ss) of four unit-normalised s primitives of
exponent alpha on one centre, from the closed form 2 sqrt(alpha/pi) (the
textbook primitive formula 2 pi^{5/2} / (p q sqrt(p+q)) F_0(0) with
p = q = 2 alpha, times the normalisation (2 alpha/pi)^{3/4} to the fourth),
evaluated in exact arithmetic by sympy and rounded to 17 significant digits.
Uses neither the oracle nor the library."""
import os

import sympy as sp

ALPHAS = ["0.1", "1.0", "2.5", "100.0", "5000.0"]

HEADER = """# (ss|ss) for four unit-normalised s primitives of exponent alpha on one centre.
# Closed form: with p = q = 2 alpha and N = (2 alpha/pi)^{3/4}, the textbook
# primitive formula 2 pi^{5/2} / (p q sqrt(p+q)) F_0(0) times N^4 reduces to
# 2 sqrt(alpha/pi).  Values below are that expression at 17 significant digits.
# alpha      (ss|ss)
"""


def main():
    lines = [HEADER]
    for a in ALPHAS:
        v = sp.N(2 * sp.sqrt(sp.Rational(a) / sp.pi), 17)
        lines.append(f"{a:<10} {sp.sstr(v, full_prec=True)}\n")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ss_same_centre.txt")
    with open(path, "w") as f:
        f.write("".join(lines))


if __name__ == "__main__":
    main()
