"""Writes tests/golden/fp8_strassen_adversarial.txt: inputs on which the FP8
mode's Strassen error comes close to its stated normwise bound
(oracle.fp8.fp8_strassen_bound).  Calls only the oracle.  Run from the
repository root:

    python tests/golden/make_fp8_adversarial.py

The file stores INPUTS, not expected values: the test recomputes the error and
the bound from the oracle.  Search: for Strassen depth d, A is 2^d rows x
2^(d+1) columns, one row per contraction region and one column per column
region of each Strassen operand, and the block C[2^d:, :2^d] = A[:, 2^d:]^T
A[:, :2^d] is computed with d Strassen levels.  Each entry is drawn from
values just below or just above an E4M3 rounding tie (so every operand
rounds by almost half a step, in a known direction) and improved one entry at
a time while the ratio error / bound grows (coordinate ascent from a few
seeded random starts).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import fp8  # noqa: E402

OUT = os.path.join(HERE, "fp8_strassen_adversarial.txt")

# (1 + (2k+1)/16) / 2 -/+ 2^-20: scaled by 2^8 these sit just below / above
# the tie between two neighbouring E4M3 values of [128, 256).
_TIES = [(1 + f / 16) / 2 + s * 2.0 ** -20 for f in (1, 3, 5, 7) for s in (-1, 1)]
CANDIDATES = np.array(_TIES + [-t for t in _TIES])


def ratio(A, d):
    q = 2 ** d
    C, _ = fp8.fp8_ata_lower_blocks(A, [(q, q, 0, q, d)])
    ref = oracle.ata_lower(A)
    e = fp8.column_exponents(A)
    sc = np.ldexp(1.0, e)[:, None] * np.ldexp(1.0, e)[None, :]
    err = np.max(np.abs(np.tril(C) - ref)[q:, :q] / sc[q:, :q])
    return err / fp8.fp8_strassen_bound(A, d)


def search(d, starts, seed):
    rng = np.random.default_rng(seed)
    shape = (2 ** d, 2 ** (d + 1))
    best, best_v = -1.0, None
    for _ in range(starts):
        v = rng.choice(CANDIDATES, size=shape[0] * shape[1])
        cur = ratio(v.reshape(shape), d)
        improved = True
        while improved:
            improved = False
            for i in rng.permutation(v.size):
                for t in CANDIDATES:
                    if t == v[i]:
                        continue
                    w = v.copy()
                    w[i] = t
                    r = ratio(w.reshape(shape), d)
                    if r > cur + 1e-12:
                        v, cur, improved = w, r, True
        if cur > best:
            best, best_v = cur, v
    return best, best_v.reshape(shape)


def main():
    with open(OUT, "w") as f:
        f.write("# Adversarial inputs for oracle.fp8.fp8_strassen_bound, written by\n")
        f.write("# tests/golden/make_fp8_adversarial.py (oracle only).  One block per depth:\n")
        f.write("# 'depth d rows cols ratio' then the rows of A as exact hex floats.\n")
        for d, starts in ((1, 6), (2, 6)):
            r, A = search(d, starts, seed=2110 + d)
            f.write(f"depth {d} {A.shape[0]} {A.shape[1]} {r:.6f}\n")
            for row in A:
                f.write(" ".join(float(x).hex() for x in row) + "\n")
            print(f"depth {d}: ratio {r:.4f}")


if __name__ == "__main__":
    main()
