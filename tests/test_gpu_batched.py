"""ata_batched (one persistent launch over many problems) against the FP64
oracle and against one ata_lower call per problem.

Tolerances as in the single-call parity tests (relative to |A|^T|A|):
F64_EMU <= 1e-13, F32 <= 5e-5, F32_BF16 within the one-digit rounding bound.
Every problem of a batch is done as plain tiles of the same shape and digit
arithmetic as a depth-0 ata_lower call, so the two must agree bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16 = 0, 1, 2, 4


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def h(ata):
    hd = ata.Handle(depth=0, split_k=1)
    yield hd
    hd.close()


def dt(mode):
    return torch.float32 if mode in (F32, F32_BF16) else torch.float64


def make_batch(count, seed, mode, m_range=(1, 700), n_range=(1, 400), extra=()):
    ms, ns = inputs.batch_shapes(count, seed, m_range, n_range)
    shapes = [(int(a), int(b)) for a, b in zip(ms, ns)] + list(extra)
    As = [inputs.uniform(m, n, seed + 17 * i) for i, (m, n) in enumerate(shapes)]
    if mode in (F32, F32_BF16):
        As = [a.astype(np.float32) for a in As]
    return As


def to_dev(As, mode):
    Ad = [torch.from_numpy(np.ascontiguousarray(a)).to(dt(mode)).cuda() for a in As]
    Cd = [torch.full((a.shape[1], a.shape[1]), float("nan"), dtype=dt(mode), device="cuda") for a in As]
    return Ad, Cd


def bf16_bound(A):
    A = np.asarray(A, np.float64)
    m = A.shape[0]
    mx = np.max(np.abs(A), axis=0) if m else np.zeros(A.shape[1])
    _, e = np.frexp(mx)
    sc = np.where(mx > 0, np.ldexp(1.0, e), 0.0)
    S = np.sum(np.abs(A), axis=0)
    return 2.0 ** -8 * (sc[:, None] * S[None, :] + S[:, None] * sc[None, :]) + \
        m * 2.0 ** -16 * sc[:, None] * sc[None, :]


def check_against_oracle(A, C, mode):
    n = A.shape[1]
    low = np.tril_indices(n)
    assert np.all(np.isnan(C[np.triu_indices(n, 1)])), "strict upper triangle written"
    A64 = np.asarray(A, np.float64)
    ref = oracle.ata_lower(A64)
    D = oracle.abs_ata_lower(A64)
    e = np.abs(C[low] - ref[low])
    if mode == F32_BF16:
        B = bf16_bound(A)
        assert np.all(e <= B[low] * (1 + 1e-6) + 1e-30)
        return
    d = D[low]
    assert np.all(e[d == 0] == 0)
    if np.any(d > 0):
        tol = 1e-13 if mode == F64_EMU else 5e-5
        assert float(np.max(e[d > 0] / d[d > 0])) <= tol


@pytest.mark.parametrize("mode", [F64_EMU, F32, F32_BF16])
def test_batched_matches_oracle_and_single_calls(ata, h, mode):
    extra = [(0, 5), (7, 0), (1, 1), (1, 130), (300, 1), (97, 257)]
    As = make_batch(60, 11, mode, extra=extra)
    Ad, Cd = to_dev(As, mode)
    h.batched(Ad, Cd, mode)
    assert h.sync() == 0
    for A, Ct in zip(As, Cd):
        C = Ct.cpu().numpy().astype(np.float64)
        if A.shape[1] == 0:
            continue
        if A.shape[0] == 0:
            n = A.shape[1]
            assert np.all(C[np.tril_indices(n)] == 0) and np.all(np.isnan(C[np.triu_indices(n, 1)]))
            continue
        check_against_oracle(A, C, mode)
    # one ata_lower per problem (depth 0): identical bits
    single = ata.Handle(depth=0, split_k=1)
    try:
        for A, Ab, Cb in zip(As, Ad, Cd):
            if A.shape[0] == 0 or A.shape[1] == 0:
                continue
            Cs = torch.full_like(Cb, float("nan"))
            single.lower(Ab, Cs, mode)
            assert single.sync() == 0
            low = torch.tril_indices(A.shape[1], A.shape[1], device="cuda")
            assert torch.equal(Cs[low[0], low[1]], Cb[low[0], low[1]])
    finally:
        single.close()


def test_batched_repeatable_and_graph_capturable(h):
    mode = F32
    As = make_batch(40, 3, mode, m_range=(16, 2000), n_range=(8, 600))
    Ad, Cd = to_dev(As, mode)
    h.batched(Ad, Cd, mode)
    assert h.sync() == 0
    first = [c.clone() for c in Cd]
    for c in Cd:
        c.fill_(float("nan"))
    h.batched(Ad, Cd, mode)  # cached plan: no host work, same bits
    assert h.sync() == 0
    for a, b in zip(first, Cd):
        assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0))
    # the same call captured in a CUDA graph and replayed
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    for c in Cd:
        c.fill_(float("nan"))
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        h.batched(Ad, Cd, mode, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert h.sync() == 0
    for a, b in zip(first, Cd):
        assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0))


def test_batched_errors(ata, h):
    A = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    C = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert h.batched_ptr([], [], [], [], [], [], F64_EMU) == 0
    # native FP64 is not a batched mode
    assert h.batched_ptr([8], [4], [A.data_ptr()], [4], [C.data_ptr()], [4], F64) == 6
    # leading dimension below n
    assert h.batched_ptr([8], [4], [A.data_ptr()], [3], [C.data_ptr()], [4], F64_EMU) == 1
    # A overlapping C
    assert h.batched_ptr([8], [4], [A.data_ptr()], [4], [A.data_ptr()], [4], F64_EMU) == 1
    # unknown dtype
    assert h.batched_ptr([8], [4], [A.data_ptr()], [4], [C.data_ptr()], [4], 9) == 2


def ptr_table(tensors):
    return torch.tensor([t.data_ptr() for t in tensors], dtype=torch.int64, device="cuda")


@pytest.mark.parametrize("mode", [F64_EMU, F32])
def test_batched_dev_graph_replay_on_new_buffers(ata, mode):
    """Device-resident pointer arrays (ata_batched_dev): one call captured in
    a CUDA graph, the arrays rewritten with a second set of buffers of the same
    shapes, the graph replayed: the second set gets its products (oracle
    parity, and the same bits as the host-array form), the first set is not
    touched.  Problems with m == 0 are zero-filled through the device table."""
    extra = [(0, 5), (1, 130), (97, 257)]
    As1 = make_batch(30, 41, mode, m_range=(16, 900), n_range=(8, 300), extra=extra)
    As2 = make_batch(30, 41, mode, m_range=(16, 900), n_range=(8, 300), extra=extra)
    As2 = [a * 0.75 - 0.125 for a in As2]   # same shapes, other values
    A1, C1 = to_dev(As1, mode)
    A2, C2 = to_dev(As2, mode)
    ms = [a.shape[0] for a in As1]
    ns = [a.shape[1] for a in As1]
    ldas = [max(n, 1) for n in ns]
    ta, tc = ptr_table(A1), ptr_table(C1)
    hd = ata.Handle(depth=0, split_k=1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    assert hd.batched_dev_ptr(ms, ns, ta.data_ptr(), ldas, tc.data_ptr(), ldas, mode, s) == 0  # plan + workspace
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert hd.batched_dev_ptr(ms, ns, ta.data_ptr(), ldas, tc.data_ptr(), ldas, mode, s) == 0
    for c in C1:
        c.fill_(float("nan"))
    ta.copy_(ptr_table(A2))
    tc.copy_(ptr_table(C2))
    g.replay()
    torch.cuda.synchronize()
    assert hd.sync() == 0
    for c in C1:
        assert bool(torch.isnan(c).all())
    for A, Ct in zip(As2, C2):
        n = A.shape[1]
        C = Ct.cpu().numpy().astype(np.float64)
        if A.shape[0] == 0:
            assert np.all(C[np.tril_indices(n)] == 0)
            continue
        check_against_oracle(A, C, mode)
    # the host-array form on the same buffers gives the same bits
    C3 = [torch.full_like(c, float("nan")) for c in C2]
    hd.batched(A2, C3, mode)
    assert hd.sync() == 0
    for a, b in zip(C2, C3):
        assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0))
    # and so does the pre-marshalled call on a third output table, twice
    C4 = [torch.full_like(c, float("nan")) for c in C2]
    t4 = ptr_table(C4)
    call = hd.batched_dev_call(ms, ns, ta.data_ptr(), ldas, t4.data_ptr(), ldas, mode)
    for _ in range(2):
        call()
        assert hd.sync() == 0
        for a, b in zip(C2, C4):
            assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0))
    hd.close()


def test_batched_host_form_follows_new_pointers(h):
    """The plan is keyed on shapes only: a second call with other buffers of
    the same shapes reuses it and writes the new buffers."""
    mode = F32
    As1 = make_batch(25, 77, mode, m_range=(16, 600), n_range=(8, 200))
    As2 = [a[::-1].copy() for a in As1]
    A1, C1 = to_dev(As1, mode)
    A2, C2 = to_dev(As2, mode)
    h.batched(A1, C1, mode)
    h.batched(A2, C2, mode)
    assert h.sync() == 0
    for A, Ct in list(zip(As1, C1)) + list(zip(As2, C2)):
        check_against_oracle(A, Ct.cpu().numpy().astype(np.float64), mode)


def test_batched_full_workload_sampled(ata):
    """The benchmarked batch: 4096 FP32 problems, m log-uniform in [64, 4096],
    n log-uniform in [32, 1024], U[-1, 1) drawn on the device.  For every
    problem: both corners of the diagonal, the last row (first and last
    column), the first column of the last row block, and three random lower
    entries, against the oracle at 5e-5 of (|A|^T|A|)_jk."""
    count, seed = 4096, 2110
    ms, ns = inputs.batch_shapes(count, seed, (64, 4096), (32, 1024))
    ms, ns = [int(v) for v in ms], [int(v) for v in ns]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    abuf = torch.rand(sum(a * b for a, b in zip(ms, ns)), generator=g, device="cuda") * 2 - 1
    cbuf = torch.full((sum(b * b for b in ns),), float("nan"), device="cuda")
    As, Cs, oa, oc = [], [], 0, 0
    for a, b in zip(ms, ns):
        As.append(abuf[oa:oa + a * b].view(a, b))
        Cs.append(cbuf[oc:oc + b * b].view(b, b))
        oa += a * b
        oc += b * b
    hb = ata.Handle(depth=0, split_k=1)
    hb.batched(As, Cs, F32)
    assert hb.sync() == 0
    hb.close()
    rng = np.random.default_rng(seed)
    worst = 0.0
    for i, (m, n) in enumerate(zip(ms, ns)):
        j = [0, n - 1, n - 1, n - 1, n - 1]
        k = [0, n - 1, 0, max(0, n - 129), n // 2]
        for _ in range(3):
            jj = int(rng.integers(0, n))
            j.append(jj)
            k.append(int(rng.integers(0, jj + 1)))
        j, k = np.array(j), np.array(k)
        cols = torch.from_numpy(np.concatenate([j, k])).cuda()
        X = As[i][:, cols].double().cpu().numpy()
        got = Cs[i][torch.from_numpy(j).cuda(), torch.from_numpy(k).cuda()].double().cpu().numpy()
        ref, den = oracle.dot_pairs(np.ascontiguousarray(X[:, :len(j)].T), np.ascontiguousarray(X[:, len(j):].T))
        err = np.abs(got - ref) / den
        worst = max(worst, float(np.max(err)))
        assert np.all(err <= 5e-5), (i, m, n, float(np.max(err)))
    assert worst > 0  # the FP32 mode is not exact on random data
