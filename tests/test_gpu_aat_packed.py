"""The A A^T product (ATA_TRANS) and the packed lower-triangular output
(ATA_PACKED) of ata_syrk_ex / ata_lower_aat, through the C ABI.

* A A^T is the A^T A of the transposed matrix (Section 3 introduction), so
  ata_lower_aat on A must give the very bits of ata_lower on an explicit copy
  of A^T, in every mode and at every Strassen depth (same plan, same
  arithmetic; only the reads of A differ), and match the oracle's
  low(A A^T) within the mode's tolerance.
* A packed lower triangle holds exactly the values of the row-major lower
  triangle (entry (j, k) at j (j + 1) / 2 + k), for both products, with the
  alpha / beta forms, and the zero-product cases.
"""
import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16, FP8 = 0, 1, 2, 4, 5
TRANS, PACKED = 1, 2
TOL = {F64: 1e-13, F64_EMU: 1e-13, F32: 5e-5}


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def tdtype(mode):
    return torch.float64 if mode in (F64, F64_EMU) else torch.float32


def packed_of(C):
    n = C.shape[0]
    j, k = np.tril_indices(n)
    return C[j, k]


@pytest.mark.parametrize("mode", [F64, F64_EMU, F32, F32_BF16, FP8])
@pytest.mark.parametrize("m,n,cutoff,depth", [(385, 1000, 0, 0), (300, 641, 100, 1), (520, 1200, 130, 2),
                                              (77, 1, 0, 0), (1, 77, 0, 0), (129, 256, 64, 1)])
def test_aat_is_ata_of_the_transpose(ata, mode, m, n, cutoff, depth):
    A64 = inputs.uniform(m, n, seed=m * 7 + n)
    A = torch.from_numpy(A64).to(tdtype(mode)).cuda()
    At = A.t().contiguous()
    h = ata.Handle(cutoff=cutoff, depth=depth, strassen_min=2)
    C1 = torch.full((m, m), float("nan"), dtype=A.dtype, device="cuda")
    C2 = torch.full((m, m), float("nan"), dtype=A.dtype, device="cuda")
    h.lower_aat(A, C1, mode)
    h.lower(At, C2, mode)
    assert h.sync() == 0
    low = np.tril_indices(m)
    c1, c2 = C1.double().cpu().numpy(), C2.double().cpu().numpy()
    assert np.array_equal(c1[low], c2[low])
    assert np.all(np.isnan(c1[np.triu_indices(m, 1)]))
    X = A.double().cpu().numpy().T            # the operand of A A^T, as the library sees it
    if mode in TOL:
        ref, D = oracle.ata_lower(X), oracle.abs_ata_lower(X)
        assert np.all(np.abs(c1[low] - ref[low]) <= TOL[mode] * D[low])
    elif mode == FP8:
        blocks = ata.plan_blocks(n, m, FP8, h)
        C8, D8 = fp8.fp8_ata_lower_blocks(X, blocks)
        assert np.all(np.abs(c1[low] - C8[low]) <= (512 + n / 512 + 2) * 2.0 ** -24 * D8[low] + 1e-30)
    h.close()


@pytest.mark.parametrize("mode", [F64, F64_EMU, F32])
def test_aat_with_padded_leading_dimension(ata, mode):
    m, n, lda = 333, 517, 600
    buf = torch.from_numpy(inputs.uniform(m, lda, seed=3)).to(tdtype(mode)).cuda()
    A = buf[:, :n]
    h = ata.Handle(cutoff=128, depth=1, strassen_min=2)
    C = torch.full((m, m), float("nan"), dtype=A.dtype, device="cuda")
    h.lower_aat(A, C, mode)
    assert h.sync() == 0
    X = A.double().cpu().numpy().T
    low = np.tril_indices(m)
    ref, D = oracle.ata_lower(X), oracle.abs_ata_lower(X)
    assert np.all(np.abs(C.double().cpu().numpy()[low] - ref[low]) <= TOL[mode] * D[low])
    h.close()


@pytest.mark.parametrize("mode", [F64, F64_EMU, F32, F32_BF16, FP8])
@pytest.mark.parametrize("flags", [0, TRANS])
@pytest.mark.parametrize("m,n,cutoff,depth", [(500, 300, 0, 0), (700, 520, 130, 1), (400, 777, 128, 2)])
def test_packed_holds_the_lower_triangle(ata, mode, flags, m, n, cutoff, depth):
    A = torch.from_numpy(inputs.uniform(m, n, seed=m + n + flags)).to(tdtype(mode)).cuda()
    nn = m if flags & TRANS else n
    h = ata.Handle(cutoff=cutoff, depth=depth, strassen_min=2)
    C = torch.full((nn, nn), float("nan"), dtype=A.dtype, device="cuda")
    P = torch.full((nn * (nn + 1) // 2 + 5,), float("nan"), dtype=A.dtype, device="cuda")
    h.syrk_ex(A, C, mode, flags=flags)
    h.syrk_ex(A, P[:-5], mode, flags=flags | PACKED)
    assert h.sync() == 0
    p = P.double().cpu().numpy()
    assert np.array_equal(p[:-5], packed_of(C.double().cpu().numpy()))
    assert np.all(np.isnan(p[-5:]))          # nothing written past the triangle
    h.close()


@pytest.mark.parametrize("mode", [F64_EMU, F32])
def test_packed_alpha_beta_and_zero_products(ata, mode):
    m, n = 300, 257
    A = torch.from_numpy(inputs.uniform(m, n, seed=11)).to(tdtype(mode)).cuda()
    h = ata.Handle(cutoff=96, depth=1, strassen_min=2)
    # two row blocks accumulated (beta = 1) equal the stacked product
    P = torch.zeros((n * (n + 1) // 2,), dtype=A.dtype, device="cuda")
    h.syrk_ex(A[:140], P, mode, flags=PACKED, alpha=1.0, beta=0.0)
    h.syrk_ex(A[140:], P, mode, flags=PACKED, alpha=1.0, beta=1.0)
    C = torch.zeros((n, n), dtype=A.dtype, device="cuda")
    h.syrk_ex(A, C, mode, alpha=0.5)
    assert h.sync() == 0
    X = A.double().cpu().numpy()
    ref, D = oracle.ata_lower(X), oracle.abs_ata_lower(X)
    tol = 2 * TOL[mode] * packed_of(D)
    assert np.all(np.abs(P.double().cpu().numpy() - packed_of(ref)) <= tol)
    assert np.all(np.abs(packed_of(C.double().cpu().numpy()) - 0.5 * packed_of(ref)) <= tol)
    # alpha = 0 scales by beta; m = 0 zeroes (packed)
    Q = P.clone()
    h.syrk_ex(A, Q, mode, flags=PACKED, alpha=0.0, beta=2.0)
    Z = torch.full_like(P, 7.0)
    rc = h.syrk_ex_ptr(PACKED, 0, n, 1.0, A.data_ptr(), n, 0.0, Z.data_ptr(), 0, mode)
    assert rc == 0 and h.sync() == 0
    assert torch.equal(Q, 2 * P)
    assert bool((Z == 0).all())
    h.close()


def test_flag_and_argument_errors(ata):
    A = torch.ones((8, 6), dtype=torch.float64, device="cuda")
    C = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    h = ata.Handle()
    assert h.syrk_ex_ptr(4, 8, 6, 1.0, A.data_ptr(), 6, 0.0, C.data_ptr(), 8, F64_EMU) == 1   # unknown flag
    assert h.syrk_ex_ptr(TRANS, 8, 6, 1.0, A.data_ptr(), 5, 0.0, C.data_ptr(), 8, F64_EMU) == 1  # lda < n
    assert h.syrk_ex_ptr(TRANS, 8, 6, 1.0, A.data_ptr(), 6, 0.0, C.data_ptr(), 7, F64_EMU) == 1  # ldc < m
    # packed C overlapping A is rejected; ldc is not checked when packed
    assert h.syrk_ex_ptr(PACKED, 8, 6, 1.0, A.data_ptr(), 6, 0.0, A.data_ptr() + 8, 0, F64_EMU) == 1
    assert h.syrk_ex_ptr(PACKED, 8, 6, 1.0, A.data_ptr(), 6, 0.0, C.data_ptr(), 0, F64_EMU) == 0
    assert h.sync() == 0
    h.close()
