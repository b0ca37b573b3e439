"""Map workers of a batched call (NEXT-1 batching form): a plan with max_batch > 1 and a small
workspace runs the maps of one call on worker instances that share its tables, each on its own
stream forked from and joined back into the call's stream. Results are bitwise those of one map
per call (same kernels, deterministic reductions); the autotuner (CRV_F_TUNE) records its
choice; a batched call captures into a CUDA graph and replays on new inputs; clones keep the
workers."""
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

MIXED = crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _maps(L, n, seed):
    return torch.tensor(np.stack([O.sht_inverse(inputs.flm_gaussian(L, seed + k, 0, True), L, 0).real for k in range(n)]),
                        device="cuda")


def _one_by_one(L, maps):
    p = crv.Plan(L, 2.0, 2, 0, MIXED, max_batch=1)
    assert crv.crv_plan_tuning(p.handle)["workers"] == 1
    Ws, outs = [], []
    for b in range(maps.shape[0]):
        W, Wphi, out = p.W_tensors(1), p.Wphi_tensor(1), p.map_tensor(1)
        crv.crv_analysis(p.handle, maps[b:b + 1], W, Wphi, 1)
        crv.crv_synthesis(p.handle, W, Wphi, out, 1)
        Ws.append(W)
        outs.append(out)
    torch.cuda.synchronize()
    p.close()
    return Ws, outs


def _check_same(p, maps, Ws, outs):
    B = maps.shape[0]
    W, Wphi, out = p.W_tensors(B), p.Wphi_tensor(B), p.map_tensor(B)
    crv.crv_analysis(p.handle, maps, W, Wphi, B)
    crv.crv_synthesis(p.handle, W, Wphi, out, B)
    crv.crv_plan_check(p.handle)
    for b in range(B):
        for j in range(p.J0, p.J + 1):
            assert torch.equal(W[j][b], Ws[b][j][0]), (b, j)
        assert torch.equal(out[b], outs[b][0]), b


def test_batched_call_on_workers_matches_single_map_calls():
    L, B = 48, 5
    maps = _maps(L, B, 300)
    Ws, outs = _one_by_one(L, maps)
    p = crv.Plan(L, 2.0, 2, 0, MIXED, max_batch=B)
    assert crv.crv_plan_tuning(p.handle)["workers"] == 4  # up to 4 workers, 5 maps: uneven split
    _check_same(p, maps, Ws, outs)
    q = p.clone()  # a clone keeps the workers
    assert crv.crv_plan_tuning(q.handle)["workers"] == 4
    p.close()
    _check_same(q, maps, Ws, outs)
    q.close()


def test_autotuned_plan_records_its_choice_and_gives_the_same_results():
    L, B = 64, 4
    maps = _maps(L, B, 400)
    Ws, outs = _one_by_one(L, maps)
    p = crv.Plan(L, 2.0, 2, 0, MIXED | crv.CRV_F_TUNE, max_batch=B)
    t = crv.crv_plan_tuning(p.handle)
    assert t["tuned"] and t["workers"] in (1, 2, 4) and t["ring_bytes"] > 0
    _check_same(p, maps, Ws, outs)
    p.close()


def test_batched_call_on_workers_replays_in_a_cuda_graph():
    L, B = 40, 2
    p = crv.Plan(L, 2.0, 2, 0, MIXED, max_batch=B)
    assert crv.crv_plan_tuning(p.handle)["workers"] == 2
    inputs_ = [_maps(L, B, 500 + 10 * k) for k in range(2)]
    m = p.map_tensor(B)
    W, Wphi, out = p.W_tensors(B), p.Wphi_tensor(B), p.map_tensor(B)
    eager = []
    for x in inputs_:
        m.copy_(x)
        crv.crv_analysis(p.handle, m, W, Wphi, B)
        crv.crv_synthesis(p.handle, W, Wphi, out, B)
        torch.cuda.synchronize()
        eager.append(out.clone())
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g):
            crv.crv_analysis(p.handle, m, W, Wphi, B)
            crv.crv_synthesis(p.handle, W, Wphi, out, B)
    torch.cuda.synchronize()
    for k in (1, 0):
        m.copy_(inputs_[k])
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager[k])
    crv.crv_plan_check(p.handle)
    p.close()
