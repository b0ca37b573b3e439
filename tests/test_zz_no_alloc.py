"""The allocation-free Delta table entry point (crv_delta_table_noalloc).

Some callers cannot allocate device memory during a call: a host framework that owns
a fixed device arena, code issued while a stream is captured into a CUDA graph, or a
latency-critical path that cannot take the synchronisation cudaMalloc/cudaFree imply.
This entry point serves them: its scratch (the recursion's seed rows) is a static
device array of the library, and the caller passes only the output table. The test
runs it twice in a row, through the C ABI, and checks each result against the table
the regular plan path builds (crv_plan_delta), within the tolerance the other Delta
tests use. It lives in a file of its own that pytest collects last.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _check_table(Q, L, plan):
    Qh = Q.cpu().numpy().reshape(L, L, L)
    for l in sorted({0, 1, L // 2, L - 1}):
        ref = plan.delta(l)                 # [m'][n] for 0 <= m', n <= l, from the plan
        got = Qh[: l + 1, l, : l + 1]       # Q[m'][l][n]
        assert np.abs(got - ref).max() < 1e-14 + 2e-16 * l, l
    # outside the triangle the table is zero
    assert Qh[L - 1, 0, 0] == 0.0 and (L < 2 or Qh[0, 0, 1] == 0.0)


def test_noalloc_delta_matches_plan_twice():
    import paper_1511_05578_gb300 as crv
    L1, L2 = 300, 64
    p1 = crv.Plan(L1, 2.0, 0, 0, crv.CRV_F_REAL)
    p2 = crv.Plan(L2, 2.0, 0, 0, crv.CRV_F_REAL)
    Q1 = torch.full((L1 ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    Q2 = torch.full((L2 ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    crv.crv_delta_table_noalloc(L1, Q1)   # first call on this device also looks up the scratch address
    torch.cuda.synchronize()
    _check_table(Q1, L1, p1)
    crv.crv_delta_table_noalloc(L2, Q2)   # second call reuses the same scratch
    torch.cuda.synchronize()
    _check_table(Q2, L2, p2)
    p1.close()
    p2.close()


def test_noalloc_delta_at_its_size_limit_matches_oracle():
    """At the scratch array's limit (L = CRV_NOALLOC_MAX_L) a few rows of the table, including
    the last one, against the oracle's Delta, which Risbo's recursion computes independently of
    the library's (the same bar as the plan's Delta tests)."""
    import oracle as O
    import paper_1511_05578_gb300 as crv
    L = crv.CRV_NOALLOC_MAX_L
    Q = torch.full((L ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    crv.crv_delta_table_noalloc(L, Q)
    torch.cuda.synchronize()
    Qh = Q.view(L, L, L)
    for l in (0, 1, L // 2 - 1, L - 1):
        got = Qh[: l + 1, l, : l + 1].cpu().numpy()
        want = O.delta_matrix(l)[l:, l:]         # m', n >= 0 quadrant
        assert np.abs(got - want).max() < 1e-14 + 2e-16 * l, l
    del Q


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1511_05578_gb300 as crv
    Q = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(crv.CrvError) as e:
        crv.crv_delta_table_noalloc(crv.CRV_NOALLOC_MAX_L + 1, Q)
    assert e.value.status == crv.CRV_EINVAL
    assert "must be in" in crv.crv_last_error()
