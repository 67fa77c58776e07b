"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (componentwise, relative to D = |A|^T |A|, zero where D == 0):
  F64 and F64_EMU  <= 1e-13   (native FP64 and 6-digit emulation, depth <= 3)
  F32              <= 5e-5
  F32_BF16         rigorous input-rounding bound (one 8-bit digit per column)
and bit-exact results wherever the arithmetic is exact (small integers,
Hadamard columns), bit-identical repeated runs, and an untouched strict upper
triangle."""
import math

import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16 = 0, 1, 2, 4
TOL = {F64: 1e-13, F64_EMU: 1e-13, F32: 5e-5}


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def h(ata):
    hd = ata.Handle()
    yield hd
    hd.close()


def is_f32(mode):
    return mode in (F32, F32_BF16)


def run(h, A, mode, cutoff=0, depth=0, slices=0, sentinel=float("nan"), strassen_min=2):
    # strassen_min=2: apply the requested Strassen depth even to small blocks
    h.set_config(cutoff, depth, slices, strassen_min)
    dt = torch.float32 if is_f32(mode) else torch.float64
    n = A.shape[1]
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(dt).cuda()
    Cd = torch.full((n, n), sentinel, dtype=dt, device="cuda")
    h.lower(Ad, Cd, mode)
    rc = h.sync()
    assert rc == 0, f"ata_sync -> {rc}"
    return Cd.cpu().numpy().astype(np.float64)


def rel_err(C, ref, D):
    n = ref.shape[0]
    low = np.tril_indices(n)
    e = np.abs(C[low] - ref[low])
    d = D[low]
    zero = d == 0
    assert np.all(e[zero] == 0), "nonzero result where |A|^T|A| is zero"
    if np.all(zero):
        return 0.0
    return float(np.max(e[~zero] / d[~zero]))


def upper_untouched(C):
    n = C.shape[0]
    return bool(np.all(np.isnan(C[np.triu_indices(n, 1)])))


def reference(A):
    A64 = np.asarray(A, np.float64)
    return oracle.ata_lower(A64), oracle.abs_ata_lower(A64)


# ----------------------------------------------------------------- cases --

def test_config1_fp64_emulation_and_native(h):
    """256 x 192 FP64 U[-1,1], recursion cutoff 64, Strassen depth 1."""
    A = inputs.uniform(256, 192, seed=1)
    ref, D = reference(A)
    for mode in (F64_EMU, F64):
        C = run(h, A, mode, cutoff=64, depth=1)
        assert upper_untouched(C)
        assert rel_err(C, ref, D) <= TOL[mode], mode


SHAPES = [(256, 192), (300, 257), (37, 129), (1000, 385), (4099, 130), (129, 1), (1, 77), (513, 640)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("depth", [0, 1, 2, 3])
def test_emulation_matches_oracle(h, m, n, depth):
    A = inputs.uniform(m, n, seed=m * 7 + n)
    ref, D = reference(A)
    cutoff = max(1, n // 4)
    C = run(h, A, F64_EMU, cutoff=cutoff, depth=depth)
    assert upper_untouched(C)
    assert rel_err(C, ref, D) <= 1e-13


@pytest.mark.parametrize("m,n", [(256, 192), (300, 257), (1000, 385), (64, 1)])
@pytest.mark.parametrize("depth", [0, 1, 2])
def test_native_f64_matches_oracle(h, m, n, depth):
    A = inputs.uniform(m, n, seed=m + 3 * n)
    ref, D = reference(A)
    C = run(h, A, F64, cutoff=max(1, n // 4), depth=depth)
    assert upper_untouched(C)
    assert rel_err(C, ref, D) <= 1e-13


@pytest.mark.parametrize("m,n", [(256, 192), (1000, 385), (4099, 130)])
@pytest.mark.parametrize("depth", [0, 1, 2])
def test_f32_matches_oracle(h, m, n, depth):
    A = inputs.uniform(m, n, seed=m + n).astype(np.float32)
    ref, D = reference(A)
    C = run(h, A, F32, cutoff=max(1, n // 4), depth=depth)
    assert upper_untouched(C)
    assert rel_err(C, ref, D) <= 5e-5


def bf16_bound(A):
    """|C - C_ref| <= 2^-8 (2^e_j S_k + 2^e_k S_j) + m 2^-16 2^(e_j + e_k), with
    S_j = sum_i |a_ij| and 2^e_j > max_i |a_ij| the column scale: one digit
    rounded to 7 fraction bits of the column scale (error <= 2^-8 2^e_j)."""
    A = np.asarray(A, np.float64)
    m = A.shape[0]
    mx = np.max(np.abs(A), axis=0)
    _, e = np.frexp(mx)
    sc = np.where(mx > 0, np.ldexp(1.0, e), 0.0)
    S = np.sum(np.abs(A), axis=0)
    return 2.0 ** -8 * (sc[:, None] * S[None, :] + S[:, None] * sc[None, :]) + \
        m * 2.0 ** -16 * sc[:, None] * sc[None, :]


@pytest.mark.parametrize("depth", [0, 1])
def test_bf16_within_rounding_bound(h, depth):
    A = inputs.uniform(777, 300, seed=5).astype(np.float32)
    ref, _ = reference(A)
    C = run(h, A, F32_BF16, cutoff=75, depth=depth)
    B = bf16_bound(A)
    low = np.tril_indices(300)
    assert np.all(np.abs(C[low] - ref[low]) <= B[low] * (1 + 1e-6) + 1e-30)
    assert upper_untouched(C)


@pytest.mark.parametrize("mode", [F64_EMU, F64, F32, F32_BF16])
@pytest.mark.parametrize("depth", [0, 1, 3])
def test_integer_inputs_bit_exact(h, mode, depth):
    """Small integers: every mode's arithmetic is exact, Strassen included."""
    A = inputs.integer_valued(531, 277, seed=9)
    ref, _ = reference(A)
    C = run(h, A, mode, cutoff=70, depth=depth)
    low = np.tril_indices(277)
    assert np.array_equal(C[low], ref[low])


@pytest.mark.parametrize("mode", [F64_EMU, F64, F32, F32_BF16])
def test_hadamard_gives_identity(h, mode):
    A = inputs.hadamard(256, 200)
    C = run(h, A, mode, cutoff=50, depth=1)
    low = np.tril_indices(200)
    assert np.array_equal(C[low], np.eye(200)[low])


def test_all_ones_gives_m(h):
    A = np.ones((333, 150))
    for mode in (F64_EMU, F64, F32):
        C = run(h, A, mode, cutoff=40, depth=1)
        low = np.tril_indices(150)
        assert np.all(C[low] == 333.0)


@pytest.mark.parametrize("mode", [F64_EMU, F64, F32])
def test_repeated_runs_bit_identical(h, mode):
    A = inputs.uniform(700, 333, seed=12)
    C1 = run(h, A, mode, cutoff=80, depth=2)
    C2 = run(h, A, mode, cutoff=80, depth=2)
    low = np.tril_indices(333)
    assert np.array_equal(C1[low], C2[low])


def test_column_scaled_inputs(h):
    """N(0,1) entries with per-column scales 10^U(-3,3): the power-of-two
    column equilibration keeps the componentwise error at the FP64 level."""
    A = inputs.column_scaled_normal(2000, 300, seed=4)
    ref, D = reference(A)
    C = run(h, A, F64_EMU, depth=0)
    assert rel_err(C, ref, D) <= 1e-13
    C = run(h, A, F64, depth=0)
    assert rel_err(C, ref, D) <= 1e-13


def test_degenerate_sizes(h, ata):
    # m == 0: low(C) is zero; n == 0: nothing happens.
    n = 50
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    A = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    assert h.lower_ptr(0, n, A.data_ptr(), n, C.data_ptr(), n, F64_EMU) == 0
    assert h.sync() == 0
    Cn = C.cpu().numpy()
    assert np.all(Cn[np.tril_indices(n)] == 0) and upper_untouched(Cn)
    assert h.lower_ptr(5, 0, A.data_ptr(), 1, C.data_ptr(), 1, F64_EMU) == 0
    # zero column: C row/column exactly zero
    Az = inputs.uniform(100, 20, seed=3)
    Az[:, 7] = 0
    ref, D = reference(Az)
    Cz = run(h, Az, F64_EMU)
    assert rel_err(Cz, ref, D) <= 1e-13


def test_error_codes(h, ata):
    n = 16
    A = torch.zeros((8, n), dtype=torch.float64, device="cuda")
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    assert h.lower_ptr(8, n, A.data_ptr(), n - 1, C.data_ptr(), n, F64_EMU) == 1   # lda < n
    assert h.lower_ptr(8, n, A.data_ptr(), n, C.data_ptr(), n - 1, F64_EMU) == 1   # ldc < n
    assert h.lower_ptr(-1, n, A.data_ptr(), n, C.data_ptr(), n, F64_EMU) == 1
    assert h.lower_ptr(8, n, A.data_ptr(), n, C.data_ptr(), n, 3) == 2             # dtype
    assert h.lower_ptr(8, n, A.data_ptr(), n, A.data_ptr(), n, F64_EMU) == 1       # overlap
    assert h.lower_ptr(8, n, 0, n, C.data_ptr(), n, F64_EMU) == 1                  # null A


def test_nonfinite_input_reported(h):
    A = inputs.uniform(64, 32, seed=2)
    A[3, 5] = np.inf
    h.set_config(0, 0, 0, 0)
    Ad = torch.from_numpy(A).cuda()
    Cd = torch.zeros((32, 32), dtype=torch.float64, device="cuda")
    assert h.lower_ptr(64, 32, Ad.data_ptr(), 32, Cd.data_ptr(), 32, F64_EMU) == 0
    assert h.sync() == 1          # ATA_ERR_INVALID from the device status word
    assert h.sync() == 0          # cleared


# ------------------------------------------- the measured configuration --

def sampled_pairs(n, count, seed):
    """Lower-triangle (j, k) samples including diagonal, quadrant-boundary and
    last-row entries."""
    rng = np.random.default_rng(seed)
    j = rng.integers(0, n, count)
    k = (rng.random(count) * (j + 1)).astype(np.int64)
    fixed = [(0, 0), (n - 1, n - 1), (n - 1, 0), (n // 2, n // 2 - 1), (n // 2, 0),
             (n - 1, n // 2), (n // 4, n // 4 - 1), (3 * n // 4, n // 2 - 1)]
    j = np.concatenate([j, [a for a, _ in fixed]])
    k = np.concatenate([k, [b for _, b in fixed]])
    return j, k


@pytest.mark.parametrize("mode,depth", [(F64_EMU, 0), (F64_EMU, 1), (F64_EMU, 2), (F64_EMU, 3),
                                        (F32, 1)])
def test_8192_square_sampled(h, mode, depth):
    """A 8192 x 8192 U[-1,1] (the benchmarked configuration), checked on
    sampled entries computed one by one by the oracle."""
    m = n = 8192
    A = inputs.uniform(m, n, seed=2110)
    if is_f32(mode):
        A = A.astype(np.float32)
    C = run(h, A, mode, cutoff=2048, depth=depth, sentinel=0.0, strassen_min=1024)
    j, k = sampled_pairs(n, 3000, seed=depth)
    A64 = np.asarray(A, np.float64)
    vals, dens = oracle.dot_pairs(np.ascontiguousarray(A64[:, j].T), np.ascontiguousarray(A64[:, k].T))
    err = np.max(np.abs(C[j, k] - vals) / dens)
    assert err <= TOL[mode], err
    assert np.all(np.triu(C, 1) == 0)


@pytest.mark.parametrize("slices", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("depth", [0, 1])
def test_every_digit_count(h, slices, depth):
    """F64_EMU with S digits (F = 8 + 9 (S - 1) fraction bits per column): the
    error stays within 8 units of the digit representation, 2^(3 - F) of
    (|A|^T|A|)_jk (floored at 1e-14: the int64 sum and its final rounding), and
    small integers are exact for every S."""
    A = inputs.uniform(700, 333, seed=40 + slices)
    ref, D = reference(A)
    C = run(h, A, F64_EMU, cutoff=80, depth=depth, slices=slices)
    tol = max(2.0 ** (3 - (8 + 9 * (slices - 1))), 1e-14)
    assert rel_err(C, ref, D) <= tol
    assert upper_untouched(C)
    Ai = inputs.integer_valued(531, 277, seed=9)
    Ci = run(h, Ai, F64_EMU, cutoff=70, depth=depth, slices=slices)
    low = np.tril_indices(277)
    assert np.array_equal(Ci[low], reference(Ai)[0][low])


@pytest.mark.parametrize("mode", [F64_EMU, F32, F32_BF16])
@pytest.mark.parametrize("m,n", [(512, 700), (1024, 385), (2048, 1301)])
def test_planes_of_a_from_the_fused_sums(h, mode, m, n):
    """Depth 1 with the top block's row split on a K step (m / 2 a multiple
    of 16): the fused operand-sum prep also writes the digit planes of A and
    A's own prep pass is skipped.  Exact on small integers (F32_BF16: within
    its bound), oracle tolerance on random data, the strict upper triangle
    untouched; twice in a row, and after a call of another shape on the same
    handle (the planes' zero padding is restored when a plan is loaded)."""
    Ai = inputs.integer_valued(m, n, seed=m + n, lo=-4, hi=4).astype(np.float32 if is_f32(mode) else np.float64)
    refi, _ = reference(Ai)
    low = np.tril_indices(n)
    for _ in range(2):
        C = run(h, Ai, mode, cutoff=max(1, n // 2), depth=1)
        assert np.array_equal(C[low], refi[low])
        assert upper_untouched(C)
        run(h, inputs.uniform(300, 200, seed=1).astype(Ai.dtype), mode, cutoff=0, depth=0)  # another plan
    Ar = inputs.uniform(m, n, seed=m * 3 + n).astype(Ai.dtype)
    ref, D = reference(Ar)
    C = run(h, Ar, mode, cutoff=max(1, n // 2), depth=1)
    if mode == F32_BF16:
        assert np.all(np.abs(C[low] - ref[low]) <= bf16_bound(Ar)[low] * (1 + 1e-6) + 1e-30)
    else:
        assert rel_err(C, ref, D) <= (1e-13 if mode == F64_EMU else 5e-5)
    assert upper_untouched(C)


def test_one_digit_wide_tile_at_its_contraction_limit(h):
    """One BF16 digit on 128 x 192 tiles keeps 32-bit sums for contractions
    of up to 16384 rows: with every digit at its largest (|x| = 256, from
    entries just below the column's power of two) the sum reaches 2^30 and
    must not wrap.  The result is then exactly m (each entry rounds to 1)."""
    m, n = 16384, 200
    A = np.full((m, n), 0.999, dtype=np.float32)
    A[::2, 1::2] = -0.999  # mixed signs in some columns
    C = run(h, A, F32_BF16, cutoff=0, depth=0)
    ref = oracle.ata_lower(np.where(A > 0, 1.0, -1.0))  # the digit-rounded matrix, exactly
    low = np.tril_indices(n)
    assert np.array_equal(C[low], ref[low])
    assert upper_untouched(C)
