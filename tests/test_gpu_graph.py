"""A map's analysis + synthesis through the C ABI captured once in a CUDA graph and replayed
on new inputs (same buffers) gives the results of the eager calls (bitwise; the FP64 path's
synthesis sums with atomics, so there up to summation order): the per-call path issues
only kernels and asynchronous memsets on the caller's stream (no allocation, no host
synchronisation), so serving and batching loops can replay it."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

import oracle as O  # noqa: E402
import paper_1511_05578_gb300 as crv  # noqa: E402
from paper_1511_05578_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("flags", [crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32, crv.CRV_F_REAL])
def test_round_trip_replays_in_a_cuda_graph(flags):
    L = 40
    p = crv.Plan(L, 2.0, 2, 0, flags)
    maps_h = [O.sht_inverse(inputs.flm_gaussian(L, 50 + k, 0, True), L, 0).real for k in range(3)]
    m = p.map_tensor(1)
    W, Wphi, out = p.W_tensors(1), p.Wphi_tensor(1), p.map_tensor(1)
    eager = []
    for mh in maps_h:  # eager results (also warms up every kernel's attributes)
        m.copy_(torch.from_numpy(mh[None]))
        crv.crv_analysis(p.handle, m, W, Wphi, 1)
        crv.crv_synthesis(p.handle, W, Wphi, out, 1)
        torch.cuda.synchronize()
        eager.append((out.clone(), [w.clone() if w is not None else None for w in W]))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g):
            crv.crv_analysis(p.handle, m, W, Wphi, 1)
            crv.crv_synthesis(p.handle, W, Wphi, out, 1)
    torch.cuda.synchronize()
    for k in (2, 0, 1):
        m.copy_(torch.from_numpy(maps_h[k][None]))
        g.replay()
        torch.cuda.synchronize()
        if flags & crv.CRV_F_MIXED:
            assert torch.equal(out, eager[k][0])
        else:  # the FP64 synthesis accumulates f_lm with atomics: equal up to summation order
            assert (torch.linalg.norm(out - eager[k][0]) / torch.linalg.norm(eager[k][0])).item() < 1e-13
        for j in range(p.J0, p.J + 1):
            assert torch.equal(W[j], eager[k][1][j])
    crv.crv_plan_check(p.handle)
    p.close()
