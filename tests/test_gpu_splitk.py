"""Split contraction (ata_config.split_k): plain tiles computed as contraction
chunks whose exact partial products the combine pass sums in a fixed order.
Through the C ABI, against the oracle: within the mode's tolerance, exact on
integer inputs, run-to-run bit-identical, upper triangle untouched (the
combine masks the diagonal), with the packed output, the A A^T product,
alpha / beta, Strassen levels on the off-diagonal blocks, and the automatic
choice on a tall matrix."""
import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_EMU, F32, F32_BF16, FP8 = 1, 2, 4, 5
TRANS, PACKED = 1, 2


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def tdt(mode):
    return torch.float64 if mode == F64_EMU else torch.float32


def run(ata, A64, mode, flags=0, alpha=1.0, beta=0.0, C0=None, **cfg):
    A = torch.from_numpy(A64).to(tdt(mode)).cuda()
    m, n = A.shape
    nn = m if flags & TRANS else n
    C = torch.full((nn, nn), float("nan"), dtype=A.dtype, device="cuda") if C0 is None else C0.clone()
    h = ata.Handle(**cfg)
    h.syrk_ex(A, C, mode, flags=flags, alpha=alpha, beta=beta)
    assert h.sync() == 0
    info = ata.plan_info(n if flags & TRANS else m, nn, mode, h)
    h.close()
    return C.double().cpu().numpy(), info


def check_tol(C, X, mode):
    n = X.shape[1]
    low = np.tril_indices(n)
    assert np.all(np.isnan(C[np.triu_indices(n, 1)])), "upper triangle written"
    if mode == FP8:
        C8, D8 = fp8.fp8_ata_lower(X)
        err = np.abs(C[low] - C8[low])
        assert np.all(err <= (512 + X.shape[0] / 512 + 2) * 2.0 ** -24 * D8[low] + 1e-30)
        return
    ref, D = oracle.ata_lower(X), oracle.abs_ata_lower(X)
    if mode == F32_BF16:
        e = np.where(np.max(np.abs(X), axis=0) > 0, np.frexp(np.max(np.abs(X), axis=0))[1], 0)
        d = np.ldexp(1.0, e - 9)
        S = np.sum(np.abs(X), axis=0)
        B = d[:, None] * S[None, :] + d[None, :] * S[:, None] + X.shape[0] * d[:, None] * d[None, :] + \
            (X.shape[0] / 256 + 4) * 2.0 ** -24 * 2 * D
        assert np.all(np.abs(C[low] - ref[low]) <= B[low])
        return
    tol = 1e-13 if mode == F64_EMU else 5e-5
    assert float(np.max(np.abs(C[low] - ref[low]) / D[low])) <= tol


@pytest.mark.parametrize("mode", [F64_EMU, F32, F32_BF16, FP8])
@pytest.mark.parametrize("split", [2, 3, 5, 16])
def test_forced_split_within_tolerance(ata, mode, split):
    m, n = 3000, 333
    A = inputs.uniform(m, n, seed=split + 10 * mode).astype(np.float32 if mode != F64_EMU else np.float64)
    A = A.astype(np.float64)
    C, info = run(ata, A, mode, depth=0, split_k=split)
    assert info["split_k"] == split
    check_tol(C, A, mode)
    C2, _ = run(ata, A, mode, depth=0, split_k=split)
    low = np.tril_indices(n)
    assert np.array_equal(C[low], C2[low])


@pytest.mark.parametrize("mode", [F64_EMU, F32])
@pytest.mark.parametrize("m", [2600, 16384])
def test_split_integer_inputs_exact(ata, mode, m):
    """The chunks' exact sum can exceed int64 (m 2^(43 + h) >= 2^63 with h
    the chunks' extra fraction bits), so these regions are summed in int128:
    bit-exact on integer inputs."""
    A = inputs.integer_valued(m, 257, seed=7, lo=-4, hi=4)
    C, _ = run(ata, A, mode, depth=0, split_k=4)
    low = np.tril_indices(257)
    assert np.array_equal(C[low], oracle.ata_lower(A)[low])


@pytest.mark.parametrize("flags", [PACKED, TRANS, TRANS | PACKED])
def test_split_with_layout_flags(ata, flags):
    m, n = 700, 2600   # TRANS: the product is 700 x 700 over 2600 columns
    if not flags & TRANS:
        m, n = n, m
    A = inputs.uniform(m, n, seed=flags)
    X = A.T if flags & TRANS else A
    nn = X.shape[1]
    Aref, _ = run(ata, A, F64_EMU, flags=flags & TRANS, depth=0, split_k=4)
    if flags & PACKED:
        h = ata.Handle(depth=0, split_k=4)
        Ad = torch.from_numpy(A).cuda()
        P = torch.full((nn * (nn + 1) // 2,), float("nan"), dtype=torch.float64, device="cuda")
        h.syrk_ex(Ad, P, F64_EMU, flags=flags)
        assert h.sync() == 0
        h.close()
        j, k = np.tril_indices(nn)
        assert np.array_equal(P.cpu().numpy(), Aref[j, k])
    check_tol(Aref, X, F64_EMU)


def test_split_alpha_beta_and_strassen(ata):
    m, n = 3000, 700
    A = inputs.uniform(m, n, seed=5)
    C0 = torch.from_numpy(np.tril(inputs.uniform(n, n, seed=6))).cuda()
    C0 = torch.where(torch.tril(torch.ones_like(C0)) > 0, C0, torch.full_like(C0, float("nan")))
    C, _ = run(ata, A, F64_EMU, alpha=-0.5, beta=2.0, C0=C0, cutoff=160, depth=1, strassen_min=2, split_k=3)
    ref, D = oracle.ata_lower(A), oracle.abs_ata_lower(A)
    low = np.tril_indices(n)
    want = -0.5 * ref + 2.0 * C0.cpu().numpy()
    den = 0.5 * D + 2.0 * np.abs(C0.cpu().numpy())
    assert np.all(np.abs(C[low] - want[low]) <= 1e-13 * den[low])
    assert np.all(np.isnan(C[np.triu_indices(n, 1)]))


def test_automatic_split_on_a_tall_matrix(ata):
    m, n = 65536, 640
    Ad = inputs.device_uniform(m, n, 9, "cuda")
    h = ata.Handle(depth=-1)
    info = ata.plan_info(m, n, F64_EMU, h)
    assert info["split_k"] > 1
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    h.lower(Ad, C, F64_EMU)
    assert h.sync() == 0
    h.close()
    rng = np.random.default_rng(0)
    j = np.concatenate([[0, n - 1, n - 1], rng.integers(0, n, 60)])
    k = np.concatenate([[0, 0, n - 1], (rng.random(60) * (j[3:] + 1)).astype(np.int64)])
    cols = torch.from_numpy(np.concatenate([j, k])).cuda()
    X = Ad[:, cols].cpu().numpy()
    ref, den = oracle.dot_pairs(np.ascontiguousarray(X[:, :len(j)].T), np.ascontiguousarray(X[:, len(j):].T))
    got = C[torch.from_numpy(j).cuda(), torch.from_numpy(k).cuda()].cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-13 * den)
    assert bool(torch.isnan(C[torch.triu_indices(n, n, 1, device="cuda")[0],
                              torch.triu_indices(n, n, 1, device="cuda")[1]]).all())
