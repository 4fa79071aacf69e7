"""Writes periodic_8_exact_eigenvalues.txt: the exact Bloch spectrum of the periodic (8,1,1)
lattice (lhf_workloads.periodic_8), i.e. the eigenvalues of eq. (4.7) at each of its 8 k-points
(Prop. 6.1 eq. (6.7)) for blocks assembled in long double by the oracle's own source
(oracle.extended) and pencils solved in 50-digit arithmetic.  No Bloch function of this lattice
is removed and no overlap direction falls below the canonical cut, so these are the eigenvalues
of the whole pencil.  Calls only oracle/ (and the seeded input generator).  Run from the
repository root:  python tests/golden/make_exact_eigenvalues.py"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lhf_workloads as W  # noqa: E402
from oracle import extended as X  # noqa: E402


def main():
    cfg = W.periodic_8()
    Hl, Sl = X.core_blocks(cfg)
    Hr, Hi = X.block_dft(Hl)
    Sr, Si = X.block_dft(Sl)
    m = Hl.shape[-1]
    Hr, Hi, Sr, Si = (a.reshape(-1, m, m) for a in (Hr, Hi, Sr, Si))
    lines = ["# exact Bloch eigenvalues (Ha) of lhf_workloads.periodic_8(): k-point, then m0 ascending values",
             "# blocks in long double (oracle.extended), pencils in 50-digit arithmetic; written by",
             "# tests/golden/make_exact_eigenvalues.py"]
    for k in range(len(Hr)):
        ev = X.pencil_eigen(X.to_mp_matrix(Hr[k], Hi[k]), X.to_mp_matrix(Sr[k], Si[k]))
        lines.append(f"{k} " + " ".join(f"{float(v):.17e}" for v in ev))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "periodic_8_exact_eigenvalues.txt")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
