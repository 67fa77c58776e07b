"""Winograd's variant of the seven products, and Strassen recursed down to a
size cutoff (a depth budget of ATA_MAX_STRASSEN_DEPTH, stopped only by
strassen_min, as the paper's FastStrassen recurses to its base case), against
the oracle through the C ABI.

Both are identities in exact arithmetic, so on integer-valued inputs (whose
operand sums and products the split-digit and native FP64 modes hold
exactly) the result must equal the plain definition bit for bit; on random
data it must stay within the mode's tolerance (F64, F64_EMU 1e-13, F32 5e-5
of (|A|^T|A|)_jk)."""
import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, FP8 = 0, 1, 2, 5
TOL = {F64: 1e-13, F64_EMU: 1e-13, F32: 5e-5}
WINOGRAD = 1
MAX_DEPTH = 8


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def run(ata, A64, mode, **cfg):
    dt = torch.float64 if mode in (F64, F64_EMU) else torch.float32
    A = torch.from_numpy(A64).to(dt).cuda()
    n = A.shape[1]
    C = torch.full((n, n), float("nan"), dtype=dt, device="cuda")
    h = ata.Handle(**cfg)
    h.lower(A, C, mode)
    assert h.sync() == 0
    info = ata.plan_info(A.shape[0], n, mode, h)
    h.close()
    out = C.double().cpu().numpy()
    assert np.all(np.isnan(out[np.triu_indices(n, 1)]))
    return out, info


@pytest.mark.parametrize("mode", [F64, F64_EMU, F32])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_winograd_integer_inputs_exact(ata, mode, depth):
    m, n = 531, 700
    A = inputs.integer_valued(m, n, seed=depth + 3 * mode, lo=-4, hi=4)
    C, info = run(ata, A, mode, cutoff=170, depth=depth, strassen_min=2, variant=WINOGRAD)
    assert info["depth"] == depth and info["products"] > 0
    low = np.tril_indices(n)
    assert np.array_equal(C[low], oracle.ata_lower(A)[low])


@pytest.mark.parametrize("mode", [F64, F64_EMU, F32])
@pytest.mark.parametrize("depth", [1, 2])
@pytest.mark.parametrize("m,n", [(1000, 1100), (513, 777)])
def test_winograd_random_within_tolerance(ata, mode, depth, m, n):
    A = inputs.uniform(m, n, seed=m + depth)
    C, _ = run(ata, A, mode, cutoff=0, depth=depth, strassen_min=64, variant=WINOGRAD)
    ref, D = oracle.ata_lower(A), oracle.abs_ata_lower(A)
    low = np.tril_indices(n)
    assert float(np.max(np.abs(C[low] - ref[low]) / D[low])) <= TOL[mode]


@pytest.mark.parametrize("mode", [F64_EMU, F32])
def test_winograd_depth_three_keeps_the_tolerance(ata, mode):
    """Winograd's flattened operands sum up to 4^d blocks, so at depth 3 a
    product is up to 12 fraction bits coarser; with the digit count on auto
    the plan adds a digit and the result stays within the mode's target."""
    m, n = 1024, 1024
    A = inputs.uniform(m, n, seed=77)
    C, info = run(ata, A, mode, cutoff=0, depth=3, strassen_min=64, variant=WINOGRAD)
    assert info["depth"] == 3 and info["slices"] == (7 if mode == F64_EMU else 4)
    ref, D = oracle.ata_lower(A), oracle.abs_ata_lower(A)
    low = np.tril_indices(n)
    assert float(np.max(np.abs(C[low] - ref[low]) / D[low])) <= TOL[mode]


@pytest.mark.parametrize("variant", [0, WINOGRAD])
@pytest.mark.parametrize("mode", [F64_EMU, F32, F64])
def test_recursion_to_size_cutoff(ata, variant, mode):
    """Depth budget 8 with strassen_min 64 on 1111 columns: every block is
    split down to below 64 columns (several levels), exact on integers and
    within tolerance on random data."""
    m, n = 600, 1111
    Ai = inputs.integer_valued(m, n, seed=5, lo=-3, hi=3)
    C, info = run(ata, Ai, mode, cutoff=300, depth=MAX_DEPTH, strassen_min=64, variant=variant)
    assert info["depth"] == MAX_DEPTH and info["products"] > 7 ** 2
    low = np.tril_indices(n)
    assert np.array_equal(C[low], oracle.ata_lower(Ai)[low])
    Ar = inputs.uniform(m, n, seed=6)
    C, _ = run(ata, Ar, mode, cutoff=300, depth=MAX_DEPTH, strassen_min=64, variant=variant)
    ref, D = oracle.ata_lower(Ar), oracle.abs_ata_lower(Ar)
    assert float(np.max(np.abs(C[low] - ref[low]) / D[low])) <= TOL[mode]


def test_fp8_mode_keeps_strassen(ata):
    """The FP8 mode's stated bounds are Strassen's: asking for Winograd gives
    the same bits as Strassen."""
    A = inputs.uniform(700, 520, seed=4)
    C1, _ = run(ata, A, FP8, cutoff=130, depth=2, strassen_min=2, variant=0)
    C2, _ = run(ata, A, FP8, cutoff=130, depth=2, strassen_min=2, variant=WINOGRAD)
    low = np.tril_indices(520)
    assert np.array_equal(C1[low], C2[low])


def test_variant_and_depth_validation(ata):
    with pytest.raises(ata.AtaError):
        ata.Handle(variant=2)
    with pytest.raises(ata.AtaError):
        ata.Handle(depth=MAX_DEPTH + 1)
