"""Parity at the full sizes of the paper-style workloads, on sampled entries.

* rectangular, precision stress: tall 262144 x 2048 and wide 2048 x 65536,
  N(0,1) entries with columns scaled by 10^U(-3,3);
* precision at scale: 32768 x 32768 U[-1,1) plus a rank-16 component of
  magnitude 1e4 (cancellation stress), Strassen depth 2 and 3;
* the low-precision modes (one BF16 digit, FP8 E4M3) on the rectangular
  shapes, entry by entry within each mode's stated componentwise bound.

Inputs are drawn on the GPU (seeded); the sampled columns are copied back from
the device so the oracle uses exactly the library's inputs.  For a set of 64
columns every lower pair (2080 entries) is computed one by one by the oracle
and compared with max |C - C_ref| / (|A|^T|A|)_jk <= tol; sampled strict-upper
entries must still hold the sentinel."""
import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16, F32_FP8 = 0, 1, 2, 4, 5
TOL = {F64: 1e-13, F64_EMU: 1e-13, F32: 5e-5}


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def bf16_digit_bound(sub):
    """One BF16 digit per column: |C - C_ref| <= 2^-8 (2^e_j S_k + 2^e_k S_j)
    + m 2^-16 2^(e_j + e_k) (the digit rounds to 7 fraction bits of the
    column scale 2^e_j > max_i |a_ij|; S_j = sum_i |a_ij|)."""
    m = sub.shape[0]
    mx = np.max(np.abs(sub), axis=0)
    _, e = np.frexp(mx)
    sc = np.where(mx > 0, np.ldexp(1.0, e), 0.0)
    S = np.sum(np.abs(sub), axis=0)
    return 2.0 ** -8 * (sc[:, None] * S[None, :] + S[:, None] * sc[None, :]) + m * 2.0 ** -16 * sc[:, None] * sc[None, :]


def sampled_check(A, C, mode, ncols=64, seed=0, tol=None):
    n = A.shape[1]
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(n, size=min(ncols, n), replace=False))
    # always include the first and last columns (ragged edges)
    cols = np.unique(np.concatenate([cols, [0, n - 1]]))
    sub = A[:, torch.from_numpy(cols).to(A.device)].double().cpu().numpy()
    jj, kk = np.tril_indices(len(cols))
    vals, dens = oracle.dot_pairs(np.ascontiguousarray(sub[:, jj].T), np.ascontiguousarray(sub[:, kk].T))
    jt = torch.from_numpy(cols[jj]).to(C.device)
    kt = torch.from_numpy(cols[kk]).to(C.device)
    got = C[jt, kt].double().cpu().numpy()
    nz = dens > 0
    assert np.all(got[~nz] == 0)
    err = float(np.max(np.abs(got[nz] - vals[nz]) / dens[nz]))
    if mode in (F32_BF16, F32_FP8):
        # entry by entry within the mode's componentwise bound (depth 0)
        B = fp8.fp8_error_bound(sub) if mode == F32_FP8 else bf16_digit_bound(sub)
        bnd = np.maximum(B, B.T)[jj, kk]
        assert np.all(np.abs(got - vals) <= bnd), float(np.max(np.abs(got - vals) / bnd))
    else:
        assert err <= (tol if tol is not None else TOL[mode]), err
    # strict upper: untouched sentinel
    uj, uk = np.triu_indices(len(cols), 1)
    up = C[torch.from_numpy(cols[uj]).to(C.device), torch.from_numpy(cols[uk]).to(C.device)]
    assert bool(torch.isnan(up).all())
    return err


def run_dev(ata, A, mode, depth=-1, strassen_min=0):
    h = ata.Handle(depth=depth, strassen_min=strassen_min)
    try:
        n = A.shape[1]
        C = torch.full((n, n), float("nan"), dtype=A.dtype, device=A.device)
        h.lower(A, C, mode)
        assert h.sync() == 0
        return C
    finally:
        h.close()


@pytest.mark.parametrize("mode", [F64_EMU, F32, F64, F32_BF16, F32_FP8])
def test_tall_skinny_column_scaled(ata, mode):
    dt = torch.float32 if mode in (F32, F32_BF16, F32_FP8) else torch.float64
    A = inputs.device_column_scaled_normal(262144, 2048, 3, "cuda", dtype=dt)
    C = run_dev(ata, A, mode)
    print(f"tall 262144x2048 mode {mode}: max err {sampled_check(A, C, mode, seed=1):.3e}")


def test_wide_column_scaled(ata):
    A = inputs.device_column_scaled_normal(2048, 65536, 4, "cuda")
    C = run_dev(ata, A, F64_EMU, depth=1)  # Strassen on the 32768-wide top block
    print(f"wide 2048x65536 F64_EMU: max err {sampled_check(A, C, F64_EMU, seed=2):.3e}")


@pytest.mark.parametrize("mode", [F32_BF16, F32_FP8])
def test_wide_column_scaled_low_precision(ata, mode):
    """Plain tiles (depth 0), where the componentwise bounds apply; C is
    65536^2 FP32 (17 GB)."""
    A = inputs.device_column_scaled_normal(2048, 65536, 4, "cuda", dtype=torch.float32)
    C = run_dev(ata, A, mode, depth=0)
    print(f"wide 2048x65536 mode {mode}: max err {sampled_check(A, C, mode, seed=2):.3e}")
    del C


@pytest.mark.parametrize("depth", [2, 3])
def test_32768_rank16_stress(ata, depth):
    A = inputs.device_low_rank_stressed(32768, 32768, 5, "cuda")
    C = run_dev(ata, A, F64_EMU, depth=depth, strassen_min=2048)
    print(f"32768^2 rank-16 depth {depth}: max err {sampled_check(A, C, F64_EMU, seed=3 + depth):.3e}")
