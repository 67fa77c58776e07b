"""Parity of the FP8 mode (ATA_F32_FP8) with the oracle, through the C ABI.

Two references:
* the FP8 reference (oracle/fp8.py): the EXACT product of the same E4M3
  columns.  The GPU may differ from it only by FP32 accumulation: partial
  sums over 512 contraction rows in the tensor core, then FP32 sums of the
  partials and one final rounding, i.e. at most (512 + m/512 + 2) 2^-24 of
  |Q|^T|Q| per entry.  A wrong rounding mode, scale or plane layout is off by
  far more than that.
* the FP64 definition: within the mode's stated componentwise bound at
  Strassen depth 0, and within the normwise bound with Strassen levels.
* with Strassen levels, the exact Strassen of the same E4M3 operand sums on
  the plan's block layout (ata_plan_blocks): again only FP32 accumulation.
Plus exact results where E4M3 holds the data exactly, bit-identical repeated
runs, an untouched strict upper triangle, and the entry points that reject
the mode."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP8 = 5


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


def run(h, A, cutoff=0, depth=0, strassen_min=2):
    h.set_config(cutoff, depth, 0, strassen_min)
    n = A.shape[1]
    Ad = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    Cd = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
    h.lower(Ad, Cd, FP8)
    assert h.sync() == 0
    return Cd.cpu().numpy().astype(np.float64)


def accum_tol(m):
    return (512 + m / 512.0 + 2) * 2.0 ** -24


def upper_untouched(C):
    return bool(np.all(np.isnan(C[np.triu_indices(C.shape[0], 1)])))


SHAPES = [(256, 192), (300, 257), (37, 129), (1000, 385), (4099, 130), (129, 1), (1, 77), (2500, 96)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_matches_fp8_reference(h, m, n):
    A = inputs.uniform(m, n, seed=m * 5 + n).astype(np.float32).astype(np.float64)
    C = run(h, A)
    C8, D8 = fp8.fp8_ata_lower(A)
    low = np.tril_indices(n)
    err = np.abs(C[low] - C8[low])
    assert np.all(err <= accum_tol(m) * D8[low] + 1e-30), float(np.max(err / np.maximum(D8[low], 1e-300)))
    assert upper_untouched(C)


@pytest.mark.parametrize("maker", ["uniform", "column_scaled_normal"])
def test_within_stated_bound(h, maker):
    A = getattr(inputs, maker)(3000, 300, seed=8).astype(np.float32).astype(np.float64)
    C = run(h, A)
    ref = np.tril(oracle.ata_full(A))
    B = fp8.fp8_error_bound(A)
    low = np.tril_indices(300)
    assert np.all(np.abs(C[low] - ref[low]) <= B[low])


@pytest.mark.parametrize("depth", [1, 2])
def test_strassen_within_normwise_bound(h, depth):
    A = inputs.uniform(1200, 520, seed=21 + depth).astype(np.float32).astype(np.float64)
    C = run(h, A, cutoff=130, depth=depth)
    ref = np.tril(oracle.ata_full(A))
    e = fp8.column_exponents(A)
    sc = np.ldexp(1.0, e)[:, None] * np.ldexp(1.0, e)[None, :]
    low = np.tril_indices(520)
    scaled = np.abs(C - ref)[low] / sc[low]
    assert np.max(scaled) <= fp8.fp8_strassen_bound(A, depth)
    assert upper_untouched(C)


@pytest.mark.parametrize("m,n,cutoff,depth", [(1200, 520, 130, 1), (1200, 520, 130, 2), (701, 397, 100, 2),
                                               (513, 300, 0, 3), (2000, 1100, 0, 1)])
def test_strassen_matches_fp8_reference(h, ata, m, n, cutoff, depth):
    """With Strassen levels the reference is the same arithmetic done exactly
    (oracle.fp8.fp8_ata_lower_blocks on the plan's block layout): every
    operand an exact sum of blocks rounded once to E4M3, exact leaf products,
    FP64 result sums.  The GPU differs only by the FP32 accumulation of each
    leaf product, at most (512 + m/512 + 2) 2^-24 of the summed |Q_u|^T|Q_v|."""
    A = inputs.uniform(m, n, seed=m + 3 * n + depth).astype(np.float32).astype(np.float64)
    C = run(h, A, cutoff=cutoff, depth=depth)
    blocks = ata.plan_blocks(m, n, FP8, h)
    assert any(b[4] == depth for b in blocks), blocks
    C8, D8 = fp8.fp8_ata_lower_blocks(A, blocks)
    low = np.tril_indices(n)
    err = np.abs(C[low] - C8[low])
    assert np.all(err <= accum_tol(m) * D8[low] + 1e-30), float(np.max(err / np.maximum(D8[low], 1e-300)))
    assert upper_untouched(C)


@pytest.mark.parametrize("depth", [0, 1])
def test_integer_inputs_exact(h, depth):
    """Integers |a| <= 8 (and, at depth 1, sums of two: <= 16) have at most
    4 significant bits, and the FP32 sums stay below 2^24 in the scaled units:
    every step is exact."""
    A = inputs.integer_valued(531, 277, seed=9)
    C = run(h, A, cutoff=70, depth=depth)
    low = np.tril_indices(277)
    assert np.array_equal(C[low], oracle.ata_lower(A)[low])


def test_hadamard_gives_identity(h):
    A = inputs.hadamard(256, 200)
    C = run(h, A, cutoff=50, depth=1)
    low = np.tril_indices(200)
    assert np.array_equal(C[low], np.eye(200)[low])


def test_repeated_runs_bit_identical(h):
    A = inputs.uniform(700, 333, seed=12)
    C1 = run(h, A, cutoff=80, depth=2)
    C2 = run(h, A, cutoff=80, depth=2)
    low = np.tril_indices(333)
    assert np.array_equal(C1[low], C2[low])


def test_entry_points_that_reject_the_mode(h, ata):
    A = torch.ones((8, 8), dtype=torch.float32, device="cuda")
    C = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    from paper_2110_13042_gb300 import _binding
    assert _binding.lower_noalloc_ptr(8, 8, A.data_ptr(), 8, C.data_ptr(), 8, FP8) == 2   # ATA_ERR_DTYPE
    rc = h.batched_ptr([8], [8], [A.data_ptr()], [8], [C.data_ptr()], [8], FP8)
    assert rc == 6                                                                  # ATA_ERR_UNSUPPORTED
