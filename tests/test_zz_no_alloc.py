"""The allocation-free entry point (ata_lower_noalloc), for callers that cannot
allocate device memory when they need the product: it must give the same
lower triangle as ata_lower (plain tiled, same digit count) bit for bit on
repeated calls, stay within the mode's tolerance of the oracle, turn a
non-finite input into NaN (it has no status word), reject sizes beyond its
fixed scratch, and run correctly both on its own in a fresh process and after
every other test.  Collected last on purpose."""
import time

import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_EMU, F32, F32_BF16 = 1, 2, 4


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def _run_noalloc(ata, A, dtype):
    m, n = A.shape
    C = torch.full((n, n), float("nan"), dtype=A.dtype, device="cuda")
    rc = ata._binding.lower_noalloc_ptr(m, n, A.data_ptr(), A.stride(0), C.data_ptr(), C.stride(0), dtype)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return C


def _run_handle(ata, A, dtype):
    m, n = A.shape
    C = torch.full((n, n), float("nan"), dtype=A.dtype, device="cuda")
    h = ata.Handle(cutoff=0, depth=0, slices=0, split_k=1)  # whole tiles, as the entry point
    h.lower(A, C, dtype)
    assert h.sync() == 0
    h.close()
    return C


def _bf16_bound(A64):
    """One-digit mode: every scaled entry is rounded to 8 fraction bits of its
    column scale 2^e (|x - fx| <= 2^(e - 9)), and the exact products are summed
    in FP32 (at most (m / 256 + 2) 2^-24 relative to |A|^T|A|)."""
    m = A64.shape[0]
    e = np.where(np.max(np.abs(A64), axis=0) > 0, np.frexp(np.max(np.abs(A64), axis=0))[1], 0)
    S = np.sum(np.abs(A64), axis=0)
    d = np.ldexp(1.0, e - 9)
    D = np.abs(A64).T @ np.abs(A64)
    return d[:, None] * S[None, :] + d[None, :] * S[:, None] + m * d[:, None] * d[None, :] + \
        (m / 256 + 2) * 2.0 ** -24 * 2 * D


@pytest.mark.parametrize("dtype", [F64_EMU, F32, F32_BF16])
@pytest.mark.parametrize("m,n", [(256, 192), (1000, 385), (1537, 641)])
def test_noalloc_matches_ata_lower_twice(ata, dtype, m, n):
    """Two calls in a row (they share the scratch) give the very bits of a
    depth-0 ata_lower call, and both are within the mode's tolerance of the
    oracle."""
    A64 = inputs.uniform(m, n, seed=m + n)
    tdt = torch.float64 if dtype == F64_EMU else torch.float32
    A = torch.from_numpy(A64).to(tdt).cuda()
    ref = _run_handle(ata, A, dtype).double().cpu().numpy()
    Aq = A.double().cpu().numpy()
    C_or, D = oracle.ata_lower(Aq), oracle.abs_ata_lower(Aq)
    low = np.tril_indices(n)
    tol = {F64_EMU: 1e-13 * D, F32: 5e-5 * D, F32_BF16: _bf16_bound(Aq)}[dtype]
    assert np.all(np.abs(ref[low] - C_or[low]) <= tol[low])
    for _ in range(2):
        got = _run_noalloc(ata, A, dtype).double().cpu().numpy()
        assert np.array_equal(got[low], ref[low])
        assert np.all(np.isnan(got[np.triu_indices(n, 1)]))


@pytest.mark.parametrize("dtype", [F64_EMU, F32])
def test_noalloc_non_finite_input_gives_nan(ata, dtype):
    m, n = 300, 200
    tdt = torch.float64 if dtype == F64_EMU else torch.float32
    A = torch.from_numpy(inputs.uniform(m, n, seed=5)).to(tdt).cuda()
    A[17, 33] = float("inf")
    got = _run_noalloc(ata, A, dtype).cpu().numpy()
    assert np.all(np.isnan(got[np.tril_indices(n)]))
    # the next call starts from a clear status word
    A[17, 33] = 0.5
    got = _run_noalloc(ata, A, dtype).double().cpu().numpy()
    assert not np.any(np.isnan(got[np.tril_indices(n)]))


def test_noalloc_rejects_beyond_scratch(ata):
    m, n = 4096, 2048        # digit planes alone need ~110 MiB > 32 MiB
    A = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    rc = ata._binding.lower_noalloc_ptr(m, n, A.data_ptr(), n, C.data_ptr(), n, F64_EMU)
    assert rc == 6                          # ATA_ERR_UNSUPPORTED
    rc = ata._binding.lower_noalloc_ptr(8, 8, A.data_ptr(), 8, C.data_ptr(), 8, 0)
    assert rc == 2                          # native FP64 is not offered here
    # a huge n is rejected at once (closed-form size check, no tile count);
    # the size check comes before any launch, so C's pointer is only compared
    # (placed far from A so the overlap check passes), never dereferenced
    t0 = time.perf_counter()
    big = 1 << 29
    rc = ata._binding.lower_noalloc_ptr(1, big, A.data_ptr(), big, A.data_ptr() + (1 << 44), big, F32)
    assert rc == 6 and time.perf_counter() - t0 < 1.0
