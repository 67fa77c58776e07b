"""Pins for the CPU oracle: each check ties it to something other than itself
(exact rational arithmetic, closed forms, special matrices, a library routine,
the paper's multiplication count), chosen so that a dropped term, a wrong sign
or a transposed/wrong operand anywhere in it fails at least one of them."""
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gamma(k):
    return k * U / (1 - k * U)


def exact_lower(A):
    """low(A^T A) in exact rational arithmetic (Fractions of the doubles)."""
    m, n = A.shape
    F = [[Fraction(float(A[i, j])) for j in range(n)] for i in range(m)]
    out = {}
    for j in range(n):
        for k in range(j + 1):
            out[j, k] = sum((F[i][j] * F[i][k] for i in range(m)), Fraction(0))
    return out


# --------------------------------------------------------------------------
# The plain definition (Section 3.1, Eq. "Cij")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(1, 1), (1, 5), (5, 1), (2, 3), (7, 4), (12, 12), (9, 11)])
def test_definition_integer_inputs_exact(m, n):
    A = inputs.integer_valued(m, n, seed=11 + m * 31 + n)
    C = oracle.ata_lower(A)
    ex = exact_lower(A)
    for (j, k), v in ex.items():
        assert C[j, k] == float(v)
    # strict upper triangle untouched
    assert np.all(np.triu(C, 1) == 0)


@pytest.mark.parametrize("m,n", [(1, 1), (3, 2), (8, 5), (12, 7), (11, 12)])
def test_definition_real_inputs_within_summation_bound(m, n):
    A = inputs.uniform(m, n, seed=5 + m + 97 * n)
    C = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    ex = exact_lower(A)
    for (j, k), v in ex.items():
        err = abs(Fraction(C[j, k]) - v)
        assert err <= Fraction(gamma(m)) * Fraction(D[j, k])


def test_definition_vs_library_matmul():
    A = inputs.uniform(50, 37, seed=3)
    C = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    ref = np.tril(A.T @ A)
    assert np.all(np.abs(C - ref) <= 2 * gamma(50) * D + 1e-300)


def test_full_product_exactly_symmetric():
    A = inputs.uniform(33, 21, seed=7)
    F = oracle.ata_full(A)
    assert np.array_equal(F, F.T)
    assert np.array_equal(np.tril(F), oracle.ata_lower(A))


@pytest.mark.parametrize("m,n", [(1, 1), (4, 3), (17, 9), (64, 64)])
def test_all_ones_gives_m_times_J(m, n):
    A = np.ones((m, n))
    C = oracle.ata_lower(A)
    assert np.array_equal(C, np.tril(np.full((n, n), float(m))))
    D = oracle.abs_ata_lower(A)
    assert np.array_equal(D, C)


@pytest.mark.parametrize("m,n", [(4, 4), (16, 11), (64, 64), (256, 40)])
def test_hadamard_columns_give_identity(m, n):
    A = inputs.hadamard(m, n)
    C = oracle.ata_lower(A)
    assert np.array_equal(C, np.eye(n))


def test_psd_quadratic_form_matches_norm():
    A = inputs.uniform(40, 25, seed=19)
    Cl = oracle.ata_lower(A)
    C = Cl + np.tril(Cl, -1).T
    D = oracle.abs_ata_lower(A)
    Dfull = D + np.tril(D, -1).T
    for s in range(5):
        x = inputs.uniform(25, 1, seed=100 + s)[:, 0]
        q = x @ C @ x
        ax = A @ x
        r = ax @ ax
        bound = 4 * gamma(40 + 25) * (np.abs(x) @ Dfull @ np.abs(x))
        assert abs(q - r) <= bound
        assert q >= -bound


def test_denominator_dominates_and_equals_for_nonnegative():
    A = inputs.uniform(30, 10, seed=23)
    C = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    assert np.all(D >= np.abs(C) * (1 - 30 * U))
    P = np.abs(A)
    assert np.array_equal(oracle.abs_ata_lower(P), oracle.ata_lower(P))


def test_sampled_entries_equal_full_oracle_bitwise():
    A = inputs.uniform(70, 30, seed=29)
    C = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    rows = np.array([0, 5, 29, 29, 17, 3])
    cols = np.array([0, 2, 0, 29, 17, 1])
    v, d = oracle.ata_entries(A, rows, cols)
    assert np.array_equal(v, C[rows, cols])
    assert np.array_equal(d, D[rows, cols])
    cj = np.ascontiguousarray(A[:, rows].T)
    ck = np.ascontiguousarray(A[:, cols].T)
    v2, d2 = oracle.dot_pairs(cj, ck)
    assert np.array_equal(v2, v) and np.array_equal(d2, d)


def test_thread_count_does_not_change_values():
    A = inputs.uniform(64, 48, seed=31)
    oracle.set_threads(1)
    C1 = oracle.ata_lower(A)
    oracle.set_threads(0)
    C2 = oracle.ata_lower(A)
    oracle.set_threads(1)
    assert np.array_equal(C1, C2)


def test_inputs_are_counter_based():
    full = inputs.uniform(20, 13, seed=8)
    cols = [12, 0, 5]
    part = inputs.uniform(20, 13, seed=8, cols=cols)
    assert np.array_equal(part, full[:, cols])
    assert full.min() >= -1 and full.max() < 1


# --------------------------------------------------------------------------
# The AtA recursion (Algorithm 1) with Strassen
# --------------------------------------------------------------------------

CASES = [(1, 0), (1, 6), (2, 1), (3, 2), (5, 3), (8, 1)]


@pytest.mark.parametrize("cutoff,depth", CASES)
def test_recursion_bit_exact_on_integer_inputs(cutoff, depth):
    """Exact arithmetic: Strassen and the 2x2 split are identities, and with
    small integers every intermediate is an exactly representable integer."""
    sizes = [(m, n) for m in range(1, 25) for n in range(1, 25) if (m * 7 + n * 3) % 4 == 0]
    sizes += [(40, 40), (39, 40), (40, 33), (1, 40), (40, 1), (37, 29)]
    for (m, n) in sizes:
        A = inputs.integer_valued(m, n, seed=1000 + 41 * m + n)
        ref = oracle.ata_lower(A)
        C, _ = oracle.ata_recursive(A, cutoff, depth)
        assert np.array_equal(np.tril(C), ref), (m, n, cutoff, depth)
        assert np.all(np.triu(C, 1) == 0), "C12 must never be written"


@pytest.mark.parametrize("m,n", [(64, 64), (100, 37), (37, 100), (129, 65)])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_recursion_real_inputs_within_strassen_bound(m, n, depth):
    A = inputs.uniform(m, n, seed=2 * m + 3 * n + depth)
    ref = oracle.ata_lower(A)
    C, _ = oracle.ata_recursive(A, 8, depth)
    # Strassen is normwise stable: |err| <= c(depth) * u * max|A|^2 * m.  A
    # growth allowance of 12^depth * 64 (Higham's bound shape) is far below any
    # mistake, which shows up as O(1) errors.
    tol = 64 * 12.0 ** depth * m * U
    assert np.max(np.abs(np.tril(C) - ref)) <= tol


def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "ata_mult_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, c = line.split()
                rows.append((int(n), int(c)))
    return rows


@pytest.mark.parametrize("n,count", _golden_counts())
def test_multiplication_count_matches_paper(n, count):
    A = inputs.uniform(n, n, seed=n)
    _, cnt = oracle.ata_recursive(A, cutoff=1, depth=64)
    assert cnt["mults"] == count


@pytest.mark.parametrize("L,d,c", [(1, 0, 4), (2, 1, 3), (3, 2, 4), (2, 3, 8)])
def test_recursion_structure_counts(L, d, c):
    """Square n = c 2^L with c >= 2^d (no Strassen level capped): 4^L leaves; 2 (4^L - 1)/3 Strassen calls, each with
    7^d classical leaves and (7^d - 1)/6 splits of 18 block additions."""
    n = c * 2 ** L
    A = inputs.uniform(n, n, seed=L * 10 + d)
    _, cnt = oracle.ata_recursive(A, cutoff=c, depth=d)
    calls = 2 * (4 ** L - 1) // 3
    assert cnt["syrk_leaves"] == 4 ** L
    assert cnt["ata_calls"] == (4 ** (L + 1) - 1) // 3
    assert cnt["gemm_leaves"] == calls * 7 ** d
    assert cnt["strassen_levels"] == calls * (7 ** d - 1) // 6
    assert cnt["block_adds"] == 18 * cnt["strassen_levels"]


@pytest.mark.parametrize("r,p,q", [(1, 1, 1), (2, 2, 2), (3, 5, 4), (16, 9, 13), (31, 30, 17)])
@pytest.mark.parametrize("depth", [0, 1, 2, 5])
def test_strassen_atb_exact_on_integers(r, p, q, depth):
    A = inputs.integer_valued(r, p, seed=r * 100 + p)
    B = inputs.integer_valued(r, q, seed=r * 100 + q + 7)
    C, _ = oracle.strassen_atb(A, B, depth)
    assert np.array_equal(C, A.T @ B)


def test_strassen_count_is_seven_to_the_k():
    for k in range(5):
        n = 2 ** k
        A = inputs.uniform(n, n, seed=k)
        _, cnt = oracle.strassen_atb(A, A, depth=64)
        assert cnt["mults"] == 7 ** k


# --------------------------------------------------------------------------
# The pins above catch planted mistakes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mutation", [1, 2, 3])
def test_planted_mistakes_are_caught(mutation):
    A = inputs.integer_valued(13, 11, seed=77)
    ref = oracle.ata_lower(A)
    oracle.set_mutation(mutation)
    try:
        C, _ = oracle.ata_recursive(A, cutoff=2, depth=2)
    finally:
        oracle.set_mutation(0)
    assert not np.array_equal(np.tril(C), ref)
    C, _ = oracle.ata_recursive(A, cutoff=2, depth=2)
    assert np.array_equal(np.tril(C), ref)


def test_oracle_reproduces_stored_bits_across_machines():
    """The stored values were written by tests/golden/make_golden.py on another
    machine; without FMA contraction the oracle must reproduce every bit."""
    A = inputs.uniform(24, 17, seed=2110)
    C = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    with open(os.path.join(GOLDEN, "oracle_uniform_24x17.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            j, k, c, d = line.split()
            assert C[int(j), int(k)] == float.fromhex(c)
            assert D[int(j), int(k)] == float.fromhex(d)
