"""The static partition over streams (ata_config.streams > 1) through the C
ABI: every tile is computed by the same kernel with the same arithmetic, only
on another CTA of another launch, so the lower triangle must be bit-identical
to the single persistent launch in every mode, with Strassen levels, and when
the forked call is captured in a CUDA graph and replayed."""
import ctypes

import numpy as np
import pytest

from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64, F64_EMU, F32, F32_BF16, FP8 = 0, 1, 2, 4, 5


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


def handle(ata, streams, **cfg):
    return ata.Handle(streams=streams, **cfg)


def product(ata, A, mode, streams, **cfg):
    n = A.shape[1]
    C = torch.full((n, n), float("nan"), dtype=A.dtype, device="cuda")
    h = handle(ata, streams, **cfg)
    h.lower(A, C, mode)
    assert h.sync() == 0
    h.close()
    return C


@pytest.mark.parametrize("mode", [F64_EMU, F32, F32_BF16, FP8, F64])
@pytest.mark.parametrize("streams", [2, 4, 7])
def test_partition_bit_identical(ata, mode, streams):
    m, n = (700, 900) if mode != F64 else (300, 500)
    dt = torch.float64 if mode in (F64, F64_EMU) else torch.float32
    A = torch.from_numpy(inputs.uniform(m, n, seed=streams + mode)).to(dt).cuda()
    cfg = dict(cutoff=150, depth=2, strassen_min=2)
    C1 = product(ata, A, mode, 1, **cfg)
    Cp = product(ata, A, mode, streams, **cfg)
    assert torch.equal(torch.nan_to_num(C1, nan=-9.0), torch.nan_to_num(Cp, nan=-9.0))


def test_partition_graph_capture(ata):
    m, n = 1024, 1300
    A = torch.from_numpy(inputs.uniform(m, n, seed=3)).cuda()
    ref = product(ata, A, F64_EMU, 1, cutoff=0, depth=1, strassen_min=256)
    h = handle(ata, 4, cutoff=0, depth=1, strassen_min=256)
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    h.lower(A, C, F64_EMU, stream=s)          # plan, workspace and side streams outside capture
    torch.cuda.synchronize()
    C.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.lower(A, C, F64_EMU, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert h.sync() == 0
    assert torch.equal(torch.nan_to_num(ref, nan=-9.0), torch.nan_to_num(C, nan=-9.0))
    h.close()


def test_streams_out_of_range_rejected(ata):
    h = ata.Handle()
    c = ata._binding._config()
    c.streams = 17
    assert ata.load().ata_set_config(h._h, ctypes.byref(c)) == 1
    h.close()
