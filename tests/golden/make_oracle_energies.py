"""Writes oracle_energies.txt: the oracle's DF-RHF energy of seeded water clusters (integrals, Coulomb-metric
fitting of eqs. 1-3, SCF to |dE| < 1e-10 Eh and max|FDS - SDF| < 1e-7). Calls only oracle/ and the shared
input generator; takes a few minutes per 8-water cluster on a CPU.

Usage: python tests/golden/make_oracle_energies.py water8 [water2 ...]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dfrhf  # noqa: E402
from paper_1707_03771_gb300 import clusters  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_energies.txt")


def main(names):
    dfrhf.build()
    rows = []
    for name in names:
        s = clusters.workload(name)
        t0 = time.perf_counter()
        r = dfrhf.scf(s)
        assert r.converged, name
        rows.append(f"{name} {float(r.energy)!r} {r.iterations} {time.perf_counter() - t0:.1f}")
        print(rows[-1], flush=True)
    with open(OUT, "w") as fh:
        fh.write("# Oracle DF-RHF energies (Eh) of seeded water clusters, written by make_oracle_energies.py.\n")
        fh.write("# workload energy iterations oracle_seconds\n")
        fh.write("\n".join(rows) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["water2", "water8"])
