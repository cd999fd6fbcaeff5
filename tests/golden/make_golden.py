"""Write the stored oracle values of tests/golden/ (calls only oracle/ and the
seeded input builders; never the CUDA path).

    python tests/golden/make_golden.py

c1_gamma.txt: Gamma_nk (1/s) of the tiny simple-cubic model (2 bands, 1 atom,
27 R) on its 6^3 k grid, summed over the full 6^3 q grid (Eqs. scatter_rate,
BTE_W), T = 300 K, mu = 0.5 eV (mid-gap), Gaussian smearing 5 meV, FP64.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import synthetic as S          # noqa: E402
from oracle import eph as O    # noqa: E402

GRID = (6, 6, 6)
T, MU, SIGMA = 300.0, 0.5, 0.005


def c1_gamma():
    m = S.model_c1()
    return O.scattering_rates_grid(m, GRID, GRID, np.arange(int(np.prod(GRID))), T, MU, SIGMA)


def main():
    g = c1_gamma()
    path = os.path.join(HERE, "c1_gamma.txt")
    header = ("Gamma_nk (1/s), tiny simple-cubic model, 6^3 k x 6^3 q, T = 300 K, mu = 0.5 eV, "
              "sigma = 5 meV; rows = k-grid index, columns = band; written by make_golden.py "
              "from the FP64 oracle")
    np.savetxt(path, g, fmt="%.17e", header=header)
    print(path, g.shape)


if __name__ == "__main__":
    main()
