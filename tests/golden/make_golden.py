"""Writes the oracle regression fixture oracle_ka108.txt.

Calls only the CPU oracle (and the seeded input generator for the inputs).
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0912_3824_gb300 import synth  # noqa: E402


def main():
    p = synth.ka_params()
    s = synth.perturb(synth.make_system(108, 1.2, 1.0, 61, p), 0.1, 61 + 1000)
    f, e, w7 = oracle.forces_brute(p, s.box, s.species, s.pos)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_ka108.txt")
    with open(out, "w") as fh:
        fh.write("# KA mixture, 108 particles, density 1.2, fcc + uniform perturbation 0.1,\n")
        fh.write("# seeds 61 / 1061; oracle brute-force forces (tests/golden/make_golden.py)\n")
        fh.write("# w7: " + " ".join(repr(float(x)) for x in w7) + "\n")
        fh.write("# columns: species x y z fx fy fz e\n")
        for i in range(s.n):
            row = [s.pos[i, 0], s.pos[i, 1], s.pos[i, 2], f[i, 0], f[i, 1], f[i, 2], e[i]]
            fh.write(f"{int(s.species[i])} " + " ".join(repr(float(x)) for x in row) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
