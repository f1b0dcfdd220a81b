"""Writes tests/golden/grad_water_tz.txt: the oracle's full gradient of
E = sum_r [cJ J(P_r, Q_r) + cK K(P_r, Q_r)] (Eq. jkderiv) for the 65-AO
f-shell water (workloads.grad_water_tz: two non-symmetric terms, cJ = 1,
cK = -1/2), from the oracle's explicit four-centre McMurchie-Davidson
derivative integrals (up to g), unscreened.  Calls only oracle/ and the
seeded input generator; about two minutes.
Run: python tests/golden/make_grad_water_tz.py"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2607_05622_gb300 import workloads as W  # noqa: E402


def main():
    O.build()
    wl = W.grad_water_tz()
    t0 = time.time()
    g = O.grad(wl.mol, wl.P, wl.Q, wl.cJ, wl.cK)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grad_water_tz.txt")
    with open(out, "w") as f:
        f.write("# oracle gradient [atom][x y z], 65-AO f-shell water (workloads.grad_water_tz), "
                "cJ=%r cK=%r, %d terms, unscreened (Eq. jkderiv); written by "
                "tests/golden/make_grad_water_tz.py in %.0f s on %d threads\n"
                % (wl.cJ, wl.cK, wl.P.shape[0], time.time() - t0, O.num_threads()))
        for row in g:
            f.write(" ".join(repr(float(v)) for v in row) + "\n")
    print(out)


if __name__ == "__main__":
    main()
