"""Writes the stored expected values under tests/golden/ from the oracle only.

cubic10_exact_moments.txt: exact Chebyshev moments mu_n = Tr T_n(H~)/N of the
paper's evaluation lattice (Sec. IV-A: 10x10x10 cubic, periodic, zero diagonal,
-1 off-diagonals), rescaled with the Gershgorin bounds +-6 padded by eps = 0.01
(a = 12/1.99, b = 0), n = 0 .. 511 (the paper's Fig. 6 compares N = 256 and 512).

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def main():
    H = O.lattice_hamiltonian((10, 10, 10), onsite=np.zeros(1000))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    mu = O.exact_moments(H, a, b, 512)
    with open(os.path.join(HERE, "cubic10_exact_moments.txt"), "w") as f:
        f.write("# exact KPM moments, 10x10x10 periodic cubic lattice of Sec. IV-A (t=1, eps=0)\n")
        f.write(f"# a = {float(a)!r}  b = {float(b)!r}  (Gershgorin +-6, padding eps=0.01)\n")
        f.write("# written by tests/golden/make_golden.py from oracle.exact_moments\n")
        for n, m in enumerate(mu):
            f.write(f"{n} {float(m)!r}\n")


if __name__ == "__main__":
    main()
