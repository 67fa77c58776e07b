"""Columns at the ends of the floating-point range, through the C ABI, against
the FP64 oracle.

- Tiny FP32 columns (magnitude 2^-50 and 2^-45): the scale 2^(e_j + e_k) of
  their products lies below FP32's normal range, while C itself stays a
  normal number.
- Columns whose maximum is subnormal (FP32 about 2^-135, FP64 about 2^-1034)
  beside large columns: their digits come from a fixed point whose shift
  exceeds the significand's own, and their products with the large columns
  are normal numbers.

Entries whose |A|^T|A| is a normal number of the output type (with margin)
are held to the mode's tolerance; the others (products of two tiny or two
subnormal columns, which underflow) must be finite and no larger than
|A|^T|A| plus the output type's smallest normal number."""
import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16, F32_FP8 = 0, 1, 2, 4, 5


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    hd = pkg.Handle()
    yield hd
    hd.close()


def run(h, A, mode, depth=0, cutoff=0):
    h.set_config(cutoff, depth, 0, 2)
    dt = torch.float64 if mode in (F64, F64_EMU) else torch.float32
    n = A.shape[1]
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(dt).cuda()
    Cd = torch.full((n, n), float("nan"), dtype=dt, device="cuda")
    h.lower(Ad, Cd, mode)
    assert h.sync() == 0
    return Cd.cpu().numpy().astype(np.float64)


def tiny_f32(m, n, seed):
    """U[-1,1) FP32 columns; the first third scaled by 2^-50, the second by
    2^-45 (exact power-of-two scalings)."""
    A = inputs.uniform(m, n, seed=seed).astype(np.float32)
    A[:, : n // 3] *= np.float32(2.0 ** -50)
    A[:, n // 3: 2 * n // 3] *= np.float32(2.0 ** -45)
    return A.astype(np.float64)


def subnormal_f32(m, n, seed):
    """Two columns of subnormal FP32 values (about 2^-135, 14 significant
    bits), the rest U[-1,1) scaled by 2^40."""
    A = inputs.uniform(m, n, seed=seed) * 2.0 ** 40
    A[:, 3] *= 2.0 ** -175
    A[:, n - 2] *= 2.0 ** -176
    A = A.astype(np.float32)  # the two columns round to subnormal FP32 values
    assert 0 < np.max(np.abs(A[:, 3])) < 2.0 ** -126
    return A.astype(np.float64)


def subnormal_f64(m, n, seed):
    """Two columns of subnormal FP64 values (about 2^-1034), the rest
    U[-1,1) scaled by 2^20."""
    A = inputs.uniform(m, n, seed=seed) * 2.0 ** 20
    A[:, 5] = A[:, 5] * 2.0 ** -1054
    A[:, n - 1] = A[:, n - 1] * 2.0 ** -1060
    assert np.max(np.abs(A[:, 5])) < 2.0 ** -1022 and np.max(np.abs(A[:, 5])) > 0
    return A


def check(C, ref, D, tol, floor, tiny):
    """tol: componentwise bound (array or scalar x D) where D >= floor; tiny:
    the output type's smallest normal number."""
    n = ref.shape[0]
    low = np.tril_indices(n)
    c, r, d = C[low], ref[low], D[low]
    assert np.all(np.isfinite(c))
    big = d >= floor
    bound = tol[low] if isinstance(tol, np.ndarray) else tol * d
    err = np.abs(c - r)
    assert np.all(err[big] <= bound[big]), float(np.max(err[big] / np.maximum(d[big], 1e-300)))
    assert np.all(np.abs(c[~big]) <= d[~big] * (1 + 1e-6) + tiny)
    assert int(np.count_nonzero(big)) > n  # the checked entries include cross products


@pytest.mark.parametrize("depth", [0, 1])
@pytest.mark.parametrize("maker", ["tiny", "subnormal"])
def test_f32_extreme_columns(h, maker, depth):
    A = tiny_f32(700, 190, 31) if maker == "tiny" else subnormal_f32(700, 190, 32)
    ref, D = oracle.ata_lower(A), oracle.abs_ata_lower(A)
    C = run(h, A, F32, depth=depth, cutoff=96)
    check(C, ref, D, 5e-5, 2.0 ** -110, 2.0 ** -126)


@pytest.mark.parametrize("maker", ["tiny", "subnormal"])
def test_bf16_extreme_columns(h, maker):
    A = tiny_f32(700, 190, 33) if maker == "tiny" else subnormal_f32(700, 190, 34)
    ref = oracle.ata_lower(A)
    D = oracle.abs_ata_lower(A)
    m = A.shape[0]
    mx = np.max(np.abs(A), axis=0)
    _, e = np.frexp(mx)
    sc = np.where(mx > 0, np.ldexp(1.0, e), 0.0)
    S = np.sum(np.abs(A), axis=0)
    B = 2.0 ** -8 * (sc[:, None] * S[None, :] + S[:, None] * sc[None, :]) + m * 2.0 ** -16 * sc[:, None] * sc[None, :]
    C = run(h, A, F32_BF16)
    check(C, ref, D, B * (1 + 1e-6), 2.0 ** -110, 2.0 ** -126)


@pytest.mark.parametrize("maker", ["tiny", "subnormal"])
def test_fp8_extreme_columns(h, maker):
    A = tiny_f32(700, 190, 35) if maker == "tiny" else subnormal_f32(700, 190, 36)
    C8, D8 = fp8.fp8_ata_lower(A)
    C = run(h, A, F32_FP8)
    m = A.shape[0]
    # FP32 accumulation of the exact E4M3 products (as in the FP8 parity tests)
    tol = (512 + m / 512.0 + 2) * 2.0 ** -24 * D8
    check(C, C8, D8, tol, 2.0 ** -110, 2.0 ** -126)


@pytest.mark.parametrize("depth", [0, 1])
@pytest.mark.parametrize("mode", [F64_EMU, F64])
def test_f64_subnormal_columns(h, mode, depth):
    A = subnormal_f64(600, 170, 37 + depth)
    ref, D = oracle.ata_lower(A), oracle.abs_ata_lower(A)
    C = run(h, A, mode, depth=depth, cutoff=85)
    check(C, ref, D, 1e-13, 2.0 ** -1000, 2.0 ** -1022)
