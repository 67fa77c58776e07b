"""The allocation-free entry point (ata_lower_noalloc), for callers that cannot
allocate device memory when they need the product: it must give the same
lower triangle as ata_lower (plain tiled, same digit count) on repeated calls,
reject sizes beyond its fixed scratch, and run correctly both on its own in a
fresh process and after every other test.  Collected last on purpose."""
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
    h = ata.Handle(cutoff=0, depth=0, slices=0)
    h.lower(A, C, dtype)
    assert h.sync() == 0
    h.close()
    return C


@pytest.mark.parametrize("dtype,tol", [(F64_EMU, 1e-13), (F32, 5e-5)])
@pytest.mark.parametrize("m,n", [(256, 192), (1000, 385), (1537, 641)])
def test_noalloc_matches_ata_lower_twice(ata, dtype, tol, m, n):
    A64 = inputs.uniform(m, n, seed=m + n)
    tdt = torch.float64 if dtype == F64_EMU else torch.float32
    A = torch.from_numpy(A64).to(tdt).cuda()
    ref = _run_handle(ata, A, dtype).double().cpu().numpy()
    D = oracle.abs_ata_lower(np.asarray(A.double().cpu().numpy()))
    low = np.tril_indices(n)
    for _ in range(2):                      # two calls in a row share the scratch
        got = _run_noalloc(ata, A, dtype).double().cpu().numpy()
        assert np.all(np.abs(got[low] - ref[low]) <= tol * D[low])
        assert np.all(np.isnan(got[np.triu_indices(n, 1)]))


def test_noalloc_rejects_beyond_scratch(ata):
    m, n = 4096, 2048        # digit planes alone need ~110 MiB > 32 MiB
    A = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    rc = ata._binding.lower_noalloc_ptr(m, n, A.data_ptr(), n, C.data_ptr(), n, F64_EMU)
    assert rc == 6                          # ATA_ERR_UNSUPPORTED
    rc = ata._binding.lower_noalloc_ptr(8, 8, A.data_ptr(), 8, C.data_ptr(), 8, 0)
    assert rc == 2                          # native FP64 is not offered here
