"""Writes the stored expected values under tests/golden/ by calling only the
oracle (never the CUDA library).  Run from the repository root:

    python tests/golden/make_golden.py

oracle_uniform_24x17.txt: low(A^T A) and low(|A|^T |A|) of the seeded
U[-1,1) matrix inputs.uniform(24, 17, seed=2110) as exact hex floats, so a
machine of another architecture can check that the oracle reproduces the same
bits (it is compiled without FMA contraction for exactly this reason).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2110_13042_gb300 import inputs  # noqa: E402


def main():
    A = inputs.uniform(24, 17, seed=2110)
    C = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    with open(os.path.join(HERE, "oracle_uniform_24x17.txt"), "w") as f:
        f.write("# low(A^T A) and low(|A|^T|A|) for A = inputs.uniform(24, 17, seed=2110)\n")
        f.write("# written by tests/golden/make_golden.py (oracle only); columns: j k C_jk D_jk\n")
        for j in range(17):
            for k in range(j + 1):
                f.write(f"{j} {k} {float(C[j, k]).hex()} {float(D[j, k]).hex()}\n")


if __name__ == "__main__":
    main()
