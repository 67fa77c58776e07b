"""Failure detection, in the host-made forms only (no GPU fault, trap or hang):

* an allocation failure injected on the host (ATA_TEST_FAIL_ALLOC=1, read at
  every workspace growth) gives ATA_ERR_ALLOC before anything is launched, and
  the same handle works once the injection is lifted;
* the bounded device wait that every persistent-kernel role uses runs out on
  a barrier that nothing completes (ata_check_wait_timeout): the kernel
  returns after its short budget, ata_sync reports ATA_ERR_TIMEOUT once, and
  the handle and the CUDA context stay usable for a correct product.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_EMU, F32 = 1, 2
ATA_ERR_INVALID, ATA_ERR_ALLOC, ATA_ERR_TIMEOUT = 1, 3, 5


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def check_product(A, C, tol):
    A64 = A.double().cpu().numpy()
    got = C.double().cpu().numpy()
    ref, D = oracle.ata_lower(A64), oracle.abs_ata_lower(A64)
    low = np.tril_indices(A64.shape[1])
    assert np.all(np.abs(got[low] - ref[low]) <= tol * D[low])


def test_injected_allocation_failure(ata, monkeypatch):
    m, n = 300, 200
    A = torch.from_numpy(inputs.uniform(m, n, seed=31)).cuda()
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    h = ata.Handle(depth=0)                    # fresh handle: no workspace yet
    monkeypatch.setenv("ATA_TEST_FAIL_ALLOC", "1")
    assert h.lower_ptr(m, n, A.data_ptr(), n, C.data_ptr(), n, F64_EMU) == ATA_ERR_ALLOC
    torch.cuda.synchronize()
    assert bool(torch.isnan(C).all())           # nothing was launched
    rc = h.batched_ptr([m], [n], [A.float().data_ptr()], [n], [C.data_ptr()], [n], F32)
    assert rc == ATA_ERR_ALLOC
    monkeypatch.delenv("ATA_TEST_FAIL_ALLOC")
    h.lower(A, C, F64_EMU)
    assert h.sync() == 0
    check_product(A, C, 1e-13)
    h.close()


def test_bounded_wait_reports_timeout(ata):
    h = ata.Handle(depth=0)
    budget_ns = 20_000_000                      # 20 ms
    t0 = time.perf_counter()
    assert h.check_wait_timeout(budget_ns) == 0
    assert h.sync() == ATA_ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    assert elapsed < 2.0, elapsed               # the kernel ended by itself
    assert h.sync() == 0                        # reported once, then cleared
    # the handle and the context still compute a correct product
    m, n = 257, 130
    A = torch.from_numpy(inputs.uniform(m, n, seed=32)).cuda()
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    h.lower(A, C, F64_EMU)
    assert h.sync() == 0
    check_product(A, C, 1e-13)
    assert h.check_wait_timeout(10) == ATA_ERR_INVALID
    assert h.check_wait_timeout(10 ** 11) == ATA_ERR_INVALID
    h.close()


def test_timeout_of_one_handle_does_not_leak_into_another(ata):
    h1, h2 = ata.Handle(depth=0), ata.Handle(depth=0)
    assert h1.check_wait_timeout(1_000_000) == 0
    assert h1.sync() == ATA_ERR_TIMEOUT
    assert h2.sync() == 0
    h1.close()
    h2.close()
