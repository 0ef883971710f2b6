"""Writes fci_energies.txt: FCI ground-state energies of the synthetic ab initio systems that the
GPU sweep tests compare against where the oracle's FCI takes minutes.  Calls only oracle/ (and
the input generators of synthetic/).  Run from the repository root:

    python tests/golden/make_fci_energies.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402
from oracle import fci  # noqa: E402

SYSTEMS = [(10, 10, 0, 0)]   # (L orbitals, N electrons, 2Sz, integral seed)

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fci_energies.txt")
    with open(out, "w") as f:
        f.write("# L N twosz seed E_FCI (Eh); synthetic.integrals(L, seed), oracle.fci.ground_state\n")
        for L, N, tsz, seed in SYSTEMS:
            h, eri = synthetic.integrals(L, seed=seed)
            e = fci.ground_state(h, eri, N, tsz)[0]
            f.write(f"{L} {N} {tsz} {seed} {e!r}\n")
            print(L, N, tsz, seed, e)
