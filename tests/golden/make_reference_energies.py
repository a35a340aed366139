"""Writes reference_energies.txt: exact ground-state energies of small workloads,
computed by the CPU oracle only (dense LAPACK / sparse ARPACK on the oracle's H).
Run from the repository root: python tests/golden/make_reference_energies.py"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2605_04483_gb300 import inputs  # noqa: E402

CASES = [
    ("config1_hubbard_chain8_obc_U4", inputs.config1()),
    ("abinitio_N10_3a3b_seed11", inputs.ab_initio(10, 3, 3, seed=11)),
    ("abinitio_N12_3a3b_seed2", inputs.ab_initio(12, 3, 3, seed=2)),
    ("hubbard_chain10_obc_U4_5a5b", inputs.hubbard((10,), 5, 5, U=4.0, periodic=False)),
    ("abinitio_N10_4a4b_seed7", inputs.ab_initio(10, 4, 4, seed=7)),
    ("abinitio_N12_4a4b_seed2", inputs.ab_initio(12, 4, 4, seed=2)),
]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reference_energies.txt")
    tmp = out + ".tmp"
    with open(tmp, "w") as f:
        f.write("# Exact ground-state energies (Hartree) from the CPU oracle's H; written by\n"
                "# make_reference_energies.py.  name N n_alpha n_beta fci_dim E0\n")
        for name, w in CASES:
            E = oracle.ground_energy(w.N, w.n_alpha, w.n_beta, w.h, w.g, dense_limit=5000)
            f.write(f"{name} {w.N} {w.n_alpha} {w.n_beta} {w.fci_dim} {E:.15f}\n")
            print(name, w.fci_dim, repr(E))
    os.replace(tmp, out)
