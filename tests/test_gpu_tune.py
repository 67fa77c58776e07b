"""ata_tune: timed choice among planned candidates, stored per shape.

The tuned configuration only changes the plan, never the result beyond the
stated tolerance: C after tuning is the product of the chosen plan, equal bit
for bit to a later ata_lower of that shape."""
import numpy as np
import pytest

import oracle
from paper_2110_13042_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_EMU, F32 = 1, 2


@pytest.fixture(scope="module")
def ata():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_13042_gb300 as pkg
    return pkg


@pytest.mark.parametrize("mode", [F64_EMU, F32])
def test_tune_picks_a_candidate_and_is_used(ata, mode):
    m, n = 1536, 2304
    A = inputs.uniform(m, n, 31)
    dt = torch.float64 if mode == F64_EMU else torch.float32
    Ad = torch.from_numpy(A).to(dt).cuda()
    Ct = torch.full((n, n), float("nan"), dtype=dt, device="cuda")
    h = ata.Handle()
    try:
        ch = h.tune(Ad, Ct, mode, budget_ms=2000)
        assert ch["candidates"] >= 2
        assert ch["depth"] in (0, 1, 2, 3)
        info = ata.plan_info(m, n, mode, h)
        assert info["depth"] == ch["depth"]
        # C holds the chosen plan's product; a later call reproduces it
        C2 = torch.full_like(Ct, float("nan"))
        h.lower(Ad, C2, mode)
        assert h.sync() == 0
        low = torch.tril_indices(n, n, device="cuda")
        assert torch.equal(Ct[low[0], low[1]], C2[low[0], low[1]])
        assert bool(torch.isnan(Ct[torch.triu_indices(n, n, 1, device="cuda").unbind()]).all())
        ref = oracle.ata_lower(np.asarray(Ad.cpu().numpy(), np.float64))
        D = oracle.abs_ata_lower(np.asarray(Ad.cpu().numpy(), np.float64))
        C = Ct.cpu().numpy().astype(np.float64)
        l = np.tril_indices(n)
        tol = 1e-13 if mode == F64_EMU else 5e-5
        assert np.max(np.abs(C[l] - ref[l]) / D[l]) <= tol
        # an explicit configuration wins over the tuned one; clearing forgets it
        h.set_config(depth=0)
        assert ata.plan_info(m, n, mode, h)["depth"] == 0
        h.set_config()
        h.tune_clear()
        assert ata.plan_info(m, n, mode, h)["depth"] == ata.plan_info(m, n, mode)["depth"]
    finally:
        h.close()
