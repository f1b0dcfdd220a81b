"""Writes tests/golden/grad_chain200_atom19.txt: the oracle's gradient row of
atom 19 (a hydrogen at the chain's end) for the 200-AO chain with its 16
separable symmetric terms (cJ = 1, cK = 0), i.e. d/dR_19 sum_r J(P_r, Q_r) of
Eq. jkderiv from the oracle's explicit four-centre McMurchie-Davidson
derivative integrals, unscreened.  Calls only oracle/ and the seeded input
generator; about six minutes on 8 cores (the row needs every ordered shell
quartet with a shell on the atom).  Run: python tests/golden/make_grad_chain200.py"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2607_05622_gb300 import workloads as W  # noqa: E402

ATOM = 19


def main():
    O.build()
    wl = W.config4()
    t0 = time.time()
    g = O.grad(wl.mol, wl.P, wl.Q, wl.cJ, wl.cK, atom_filter=ATOM)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"grad_chain200_atom{ATOM}.txt")
    with open(out, "w") as f:
        f.write("# oracle gradient row, 200-AO chain (workloads.config4), atom %d, "
                "cJ=%r cK=%r, %d terms, unscreened (Eq. jkderiv); written by "
                "tests/golden/make_grad_chain200.py in %.0f s on %d threads\n"
                % (ATOM, wl.cJ, wl.cK, wl.P.shape[0], time.time() - t0, O.num_threads()))
        f.write(" ".join(repr(float(v)) for v in g[ATOM]) + "\n")
    print(out)


if __name__ == "__main__":
    main()
