"""Pins for the FP8 mode's Strassen reference (oracle.fp8.fp8_strassen_atb,
fp8_ata_lower_blocks) and for its normwise bound (fp8_strassen_bound).

* Strassen's algorithm is an identity, so on inputs whose every operand sum
  E4M3 holds exactly ({-1, 0, 1} entries: sums of up to 2^d of them scaled by
  2^(8 - t) are small multiples of powers of two) the reference must equal the
  plain definition bit for bit, at every depth and on ragged sizes (zero
  padding).  A wrong product, result sum, sign or block index breaks this;
  the planted mistakes below show it.
* A hand-worked depth-1 example, where one operand sum rounds and the result
  differs from the depth-0 product, pins the one-rounding-per-operand-sum rule
  and the 2^(8 - t) operand scale.
* The bound holds on random inputs of several distributions, depths and
  ragged shapes, and it is tight within a stated factor: on the adversarial
  inputs of tests/golden/fp8_strassen_adversarial.txt (written by
  make_fp8_adversarial.py from the oracle only) the attained error reaches at
  least 0.4 of the bound at depth 1 and 0.2 at depth 2.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def ternary(m, n, seed):
    return np.random.default_rng(seed).integers(-1, 2, size=(m, n)).astype(np.float64)


def scaled_error(A, blocks):
    C, _ = fp8.fp8_ata_lower_blocks(A, blocks)
    ref = oracle.ata_lower(A)
    e = fp8.column_exponents(A)
    sc = np.ldexp(1.0, e)[:, None] * np.ldexp(1.0, e)[None, :]
    return np.max(np.abs(np.tril(C) - ref) / sc)


@pytest.mark.parametrize("m,n,block", [
    (37, 40, (20, 20, 0, 20)),
    (64, 64, (32, 32, 0, 32)),
    (33, 77, (40, 37, 3, 37)),
    (19, 23, (11, 12, 0, 11)),
    (5, 9, (4, 5, 0, 4)),
])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_exact_on_ternary_inputs(m, n, block, depth):
    A = ternary(m, n, seed=m * n + depth)
    r0, p, c0, q = block
    C, _ = fp8.fp8_ata_lower_blocks(A, [(r0, p, c0, q, depth)])
    assert np.array_equal(np.tril(C), oracle.ata_lower(A))


def test_depth_zero_blocks_are_the_plain_fp8_product():
    A = inputs.uniform(50, 30, seed=5)
    C0, D0 = fp8.fp8_ata_lower(A)
    C, D = fp8.fp8_ata_lower_blocks(A, [(15, 15, 0, 15, 0)])
    assert np.array_equal(C, C0) and np.array_equal(D, D0)


def test_hand_worked_depth_one():
    """X = A[:, 2:4], Y = A[:, 0:2] (every column exponent 0), one row per
    contraction half.  Y's operands are exact; X11 = 17/32 gives
    X11 + X22 = 33/32, scaled by 2^(8-1) = 132, which rounds to 128 (-> 1.0),
    and X11 alone 136 = 1.0625 * 128, a tie that goes to the even 128
    (-> 0.5); X12 - X11 = 7/32 -> 28 is exact.  So M1 = 1.0 * 1.0,
    M2 = 1.25 * 0.5, M3 = M4 = M7 = 0, M5 = 1.0 * 0.5, M6 = 0.21875 * 1.0:
    C11 = M1 + M4 - M5 + M7 = 0.5, C12 = M3 + M5 = 0.5, C21 = M2 + M4 = 0.625,
    C22 = M1 - M2 + M3 + M6 = 0.59375 (the depth-0 product gives 0.625)."""
    A = np.array([[0.5, 0.5, 0.53125, 0.75], [0.5, 0.5, 0.5, 0.5]])
    C, _ = fp8.fp8_ata_lower_blocks(A, [(2, 2, 0, 2, 1)])
    assert C[2, 0] == 0.5 and C[2, 1] == 0.5 and C[3, 0] == 0.625 and C[3, 1] == 0.59375
    C0, _ = fp8.fp8_ata_lower(A)
    assert C0[3, 1] == 0.625


def test_magnitude_sum_dominates_the_product():
    A = inputs.uniform(60, 44, seed=9)
    e = fp8.column_exponents(A)
    Ah = A * np.ldexp(1.0, -e)[None, :]
    for d in (1, 2):
        M, D = fp8.fp8_strassen_atb(Ah[:, 22:], Ah[:, :22], d)
        assert np.all(D >= np.abs(M))


@pytest.mark.parametrize("mistake", ["sign_m6", "result_c21", "operand_block"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    M, Cs = list(fp8._M), dict(fp8._C)
    if mistake == "sign_m6":          # (X12 + X11) instead of (X12 - X11)
        M[5] = (((1, 0, 1), (1, 0, 0)), M[5][1])
    elif mistake == "result_c21":     # C21 = M2 - M4
        Cs[(1, 0)] = ((1, 1), (-1, 3))
    else:                             # M4 = X21^T (Y21 - Y11)
        M[3] = (((1, 1, 0),), M[3][1])
    monkeypatch.setattr(fp8, "_M", tuple(M))
    monkeypatch.setattr(fp8, "_C", Cs)
    A = ternary(16, 16, seed=3)
    C, _ = fp8.fp8_ata_lower_blocks(A, [(8, 8, 0, 8, 1)])
    assert not np.array_equal(np.tril(C), oracle.ata_lower(A))


@pytest.mark.parametrize("maker", ["uniform", "column_scaled_normal", "positive"])
@pytest.mark.parametrize("m,n,block,depth", [
    (256, 256, (128, 128, 0, 128), 1),
    (301, 190, (97, 93, 0, 97), 1),
    (256, 256, (128, 128, 0, 128), 2),
    (203, 150, (70, 80, 5, 65), 2),
    (160, 128, (64, 64, 0, 64), 3),
])
def test_bound_holds(maker, m, n, block, depth):
    if maker == "positive":
        A = np.abs(inputs.uniform(m, n, seed=m + n))
    else:
        A = getattr(inputs, maker)(m, n, seed=m + n)
    A = A.astype(np.float32).astype(np.float64)
    r0, p, c0, q = block
    assert scaled_error(A, [(r0, p, c0, q, depth)]) <= fp8.fp8_strassen_bound(A, depth)


def adversarial():
    out, lines = {}, open(os.path.join(HERE, "golden", "fp8_strassen_adversarial.txt")).read().splitlines()
    lines = [ln for ln in lines if ln and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        _, d, rows, cols, _ = lines[i].split()
        d, rows = int(d), int(rows)
        A = np.array([[float.fromhex(x) for x in lines[i + 1 + r].split()] for r in range(rows)])
        assert A.shape == (rows, int(cols))
        out[d] = A
        i += 1 + rows
    return out


@pytest.mark.parametrize("depth,factor", [(1, 0.4), (2, 0.2)])
def test_bound_is_tight_within_stated_factor(depth, factor):
    A = adversarial()[depth]
    q = 2 ** depth
    r = scaled_error(A, [(q, q, 0, q, depth)]) / fp8.fp8_strassen_bound(A, depth)
    assert factor <= r <= 1.0, r
