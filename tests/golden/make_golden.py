"""Writes the stored reference values under tests/golden/ (calls only oracle/).

fci_energies.txt: lowest FCI energies (Eh) of the seeded synthetic integrals,
from ``oracle.hamiltonian.fci_energies`` (determinant FCI, exact to rounding).
Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic_inputs as si  # noqa: E402
from oracle.hamiltonian import eri_from_cholesky, fci_energies  # noqa: E402

CASES = [  # name, K, N, twoS, n_chol, ell, h_min, nroots
    ("k6_n6", 6, 6, 0, 24, 3.0, -4.0, 2),
    ("k8_n8", 8, 8, 0, 32, 3.0, -4.0, 4),
]

if __name__ == "__main__":
    lines = ["# name K N twoS n_chol ell h_min : FCI energies (Eh), seed 0 integrals"]
    for name, K, N, twoS, nc, ell, hmin, nr in CASES:
        h, L = si.make_integrals(K, nc, ell=ell, h_min=hmin, seed=0)
        e = fci_energies(h, eri_from_cholesky(L), N, twoS, nr)
        lines.append(f"{name} {K} {N} {twoS} {nc} {ell} {hmin} : " + " ".join(f"{x:.15f}" for x in e))
    with open(os.path.join(HERE, "fci_energies.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))
