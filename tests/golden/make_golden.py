"""Write the stored expected values under tests/golden/ from the CPU oracle.

differentiation_true_roots.txt: refined roots C* (bisection to 1e-13 inside
the first sign-changing bracket of Algorithm 1) of the differentiation
workload's seeded true model (12 layers over a half-space) at its 150
log-spaced wavelengths 1..150 m, grid 50..1200 m/s step 0.25. The observed
curve of that workload is these values plus seeded N(0, 2^2) noise.

Run: python tests/golden/make_golden.py   (calls only oracle/)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2003_02256_gb300 import workloads as W  # noqa: E402


def main():
    _, g, true = W.differentiation_batch(n_models=1)
    h, a, b, r, lam = true.model(0)
    _, idx, st = oracle.dispersion(true.as_dict(), g.c0, g.dc, g.n_c)
    assert (st == 0).all()
    roots = [oracle.root(h, a, b, r, l, g.c0, g.dc, g.n_c, int(i)) for l, i in zip(lam, idx)]
    with open(os.path.join(HERE, "differentiation_true_roots.txt"), "w") as f:
        f.write("# refined roots C* (m/s) of the differentiation workload's true model,\n")
        f.write("# written by tests/golden/make_golden.py from the CPU oracle\n")
        f.write("# columns: wavelength_m  grid_index  root_m_per_s\n")
        for l, i, c in zip(lam, idx, roots):
            f.write(f"{l:.17g} {int(i)} {c:.17g}\n")


if __name__ == "__main__":
    main()
