"""ata_syrk: low(C) <- alpha low(A^T A) + beta low(C) (Section 3.1: the BLAS
?syrk semantics; Algorithm 1 accumulates alpha A^T A into C).

Reference: alpha * (the FP64 definition) + beta * C0 in FP64.  Tolerance: the
mode's product tolerance scaled by |alpha|, plus a few roundings of the two
terms in the output precision.  Also: alpha = 1, beta = 0 is bit-identical to
ata_lower; beta = 0 never reads C; alpha = 0 and m = 0 scale C exactly;
accumulating two blocks of rows equals the product of the stacked matrix
(the accumulate form of Algorithm 1); exact integers stay exact; the strict
upper triangle is untouched."""
import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16, F32_FP8 = 0, 1, 2, 4, 5
MODES = [F64_EMU, F64, F32, F32_BF16, F32_FP8]
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


def f32(mode):
    return mode in (F32, F32_BF16, F32_FP8)


def dev(x, mode):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.float32 if f32(mode) else torch.float64).cuda()


def lower_c0(n, seed, mode):
    """Random lower triangle, NaN strict upper (the sentinel)."""
    C0 = inputs.uniform(n, n, seed=seed) * 3.0
    C0[np.triu_indices(n, 1)] = np.nan
    return C0.astype(np.float32).astype(np.float64) if f32(mode) else C0


def product_bound(A, mode, ref, D):
    if mode == F32_FP8:
        return fp8.fp8_error_bound(A)
    if mode == F32_BF16:
        m = A.shape[0]
        mx = np.max(np.abs(A), axis=0)
        _, e = np.frexp(mx)
        sc = np.where(mx > 0, np.ldexp(1.0, e), 0.0)
        S = np.sum(np.abs(A), axis=0)
        return 2.0 ** -8 * (sc[:, None] * S[None, :] + S[:, None] * sc[None, :]) + m * 2.0 ** -16 * sc[:, None] * sc[None, :]
    return TOL[mode] * D


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("depth", [0, 1])
def test_alpha_beta(h, mode, depth):
    m, n = 700, 300
    A = inputs.uniform(m, n, seed=31)
    if f32(mode):
        A = A.astype(np.float32).astype(np.float64)
    alpha, beta = -1.75, 0.625
    C0 = lower_c0(n, 32, mode)
    h.set_config(75, depth, 0, 2)
    Cd = dev(C0, mode)
    h.syrk(dev(A, mode), Cd, mode, alpha, beta)
    assert h.sync() == 0
    C = Cd.cpu().numpy().astype(np.float64)
    ref = oracle.ata_full(A)
    D = np.abs(A).T @ np.abs(A)
    want = alpha * ref + beta * C0
    u = 2.0 ** -24 if f32(mode) else 2.0 ** -53
    low = np.tril_indices(n)
    if mode == F32_FP8 and depth > 0:
        e = fp8.column_exponents(A)
        sc = np.ldexp(1.0, e)[:, None] * np.ldexp(1.0, e)[None, :]
        prod = abs(alpha) * fp8.fp8_strassen_bound(A, depth) * sc
    else:
        prod = abs(alpha) * product_bound(A, mode, ref, D)
    tol = prod + 4 * u * (abs(alpha) * (np.abs(ref) + prod) + abs(beta) * np.abs(np.nan_to_num(C0)))
    assert np.all(np.abs(C - want)[low] <= tol[low]), float(np.max((np.abs(C - want) / tol)[low]))
    assert np.all(np.isnan(C[np.triu_indices(n, 1)]))


@pytest.mark.parametrize("mode", MODES)
def test_alpha_one_beta_zero_is_ata_lower(h, mode):
    A = inputs.uniform(513, 200, seed=5)
    h.set_config(50, 1, 0, 2)
    C1 = torch.full((200, 200), float("nan"), dtype=torch.float32 if f32(mode) else torch.float64, device="cuda")
    C2 = torch.full_like(C1, float("nan"))
    Ad = dev(A, mode)
    h.lower(Ad, C1, mode)
    h.syrk(Ad, C2, mode, 1.0, 0.0)   # beta == 0: the NaNs in C2 are not read
    assert h.sync() == 0
    low = np.tril_indices(200)
    a, b = C1.cpu().numpy(), C2.cpu().numpy()
    assert np.array_equal(a[low], b[low])
    assert np.all(np.isfinite(b[low]))


@pytest.mark.parametrize("mode", [F64_EMU, F32])
def test_alpha_zero_and_empty_rows_scale_c(h, mode):
    n = 150
    C0 = lower_c0(n, 9, mode)
    A = inputs.uniform(40, n, seed=2)
    for m, alpha in ((40, 0.0), (0, 2.0)):
        Cd = dev(C0, mode)
        h.syrk(dev(A[:m], mode) if m else dev(A[:1], mode)[:0], Cd, mode, alpha, -0.5)
        assert h.sync() == 0
        C = Cd.cpu().numpy()
        low = np.tril_indices(n)
        want = (np.float32(-0.5) * C0.astype(np.float32)) if f32(mode) else -0.5 * C0
        assert np.array_equal(C[low], np.asarray(want)[low])
        assert np.all(np.isnan(C[np.triu_indices(n, 1)]))


@pytest.mark.parametrize("mode", [F64_EMU, F64])
def test_accumulating_row_blocks(h, mode):
    """Algorithm 1's accumulate form: C += A1^T A1, then C += A2^T A2, equals
    low([A1; A2]^T [A1; A2])."""
    A = inputs.uniform(900, 260, seed=44)
    h.set_config(65, 1, 0, 2)
    Cd = torch.zeros((260, 260), dtype=torch.float64, device="cuda")
    h.syrk(dev(A[:400], mode), Cd, mode, 1.0, 1.0)
    h.syrk(dev(A[400:], mode), Cd, mode, 1.0, 1.0)
    assert h.sync() == 0
    C = Cd.cpu().numpy()
    ref = oracle.ata_full(A)
    D = np.abs(A).T @ np.abs(A)
    low = np.tril_indices(260)
    assert np.all(np.abs(C - ref)[low] <= 2e-13 * D[low])


@pytest.mark.parametrize("mode", [F64_EMU, F64, F32, F32_BF16, F32_FP8])
def test_integers_exact(h, mode):
    A = inputs.integer_valued(300, 130, seed=3)
    C0 = inputs.integer_valued(130, 130, seed=4)
    C0[np.triu_indices(130, 1)] = np.nan
    h.set_config(40, 1, 0, 2)
    Cd = dev(C0, mode)
    h.syrk(dev(A, mode), Cd, mode, 2.0, -3.0)
    assert h.sync() == 0
    C = Cd.cpu().numpy().astype(np.float64)
    low = np.tril_indices(130)
    assert np.array_equal(C[low], (2.0 * oracle.ata_full(A) - 3.0 * C0)[low])


def test_non_finite_scalars_rejected(h):
    A = torch.ones((4, 4), dtype=torch.float64, device="cuda")
    C = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert h.syrk_ptr(4, 4, float("nan"), A.data_ptr(), 4, 0.0, C.data_ptr(), 4, F64_EMU) == 1
    assert h.syrk_ptr(4, 4, 1.0, A.data_ptr(), 4, float("inf"), C.data_ptr(), 4, F64_EMU) == 1
