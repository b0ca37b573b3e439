"""Serving on the GPU (continuous batching of round-trip requests): each request gives the same
result alone and in a concurrent mix of band limits, spins and batch sizes, and the round trip
reproduces its maps within the mixed-precision tolerance."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))

import oracle as O  # noqa: E402
from paper_1511_05578_gb300 import inputs  # noqa: E402
from paper_1511_05578_gb300 import serving as S  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _maps(L, spin, B, seed):
    real = spin == 0
    out = []
    for b in range(B):
        f = inputs.flm_gaussian(L, seed + b, spin, real, 3.0 if spin else 2.0)
        m = O.sht_inverse(f, L, spin)
        out.append(m.real if real else np.stack([m.real, m.imag], -1))
    return np.stack(out)


def _mix():
    spec = [(16, 0, 2), (32, 2, 1), (48, 0, 1), (16, 2, 2), (32, 0, 2), (48, 2, 1), (512, 0, 1), (32, 0, 1)]
    return [S.Request(rid=i, L=L, spin=s, B=B, arrival=0.002 * i, maps=_maps(L, s, B, 100 * i))
            for i, (L, s, B) in enumerate(spec)]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_results_same_alone_and_in_mix():
    budget = 0.5 * torch.cuda.mem_get_info()[0]
    mix = _mix()
    sch = S.Scheduler(S.CudaExecutor(), budget, max_running=4)
    S.run(sch, mix)
    assert len(sch.done) == len(mix) and not sch.rejected
    # several requests were on the device at once, by their CUDA events (device time)
    def dev_overlap(a, b):
        a0, a1 = a.dev_events
        b0, b1 = b.dev_events
        return a0.elapsed_time(b1) > 0 and b0.elapsed_time(a1) > 0
    overlaps = sum(1 for a in mix for b in mix if a.rid < b.rid and dev_overlap(a, b))
    assert overlaps >= 1
    for r in mix:
        alone = S.Request(rid=r.rid, L=r.L, spin=r.spin, B=r.B, arrival=0.0, maps=r.maps)
        s1 = S.Scheduler(S.CudaExecutor(), budget, max_running=1)
        S.run(s1, [alone])
        assert _rel(r.result, alone.result) < 1e-12, (r.rid, _rel(r.result, alone.result))
        assert _rel(r.result, r.maps) < 1e-5, (r.rid, _rel(r.result, r.maps))
    st = sch.stats(max(r.finish for r in mix) - min(r.arrival for r in mix))
    assert st["p50_ms"] <= st["p99_ms"]


def test_clone_shares_tables_and_gives_identical_results():
    """crv_plan_clone: the second instance holds the same table set (no new table bytes), a
    workspace of its own, gives bitwise the same coefficients on the same map, and keeps
    working after the plan it was cloned from is destroyed."""
    import paper_1511_05578_gb300 as crv
    from gpu_util import case, map_from_device, map_to_device, rel_l2
    L, lam, J0 = 64, 2.0, 2
    p = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED | crv.CRV_F_W_FP32)
    free0 = torch.cuda.mem_get_info()[0]
    q = p.clone()
    free1 = torch.cuda.mem_get_info()[0]
    assert q.table_bytes() == p.table_bytes() > 0
    assert q.own_bytes() == p.own_bytes()
    assert free0 - free1 < p.table_bytes() + 2 * q.own_bytes()  # no second copy of the tables
    _, fmap = case(L, lam, J0, 0, True, seed=17)
    m = map_to_device(fmap, True)
    Wp, Wq = p.W_tensors(1), q.W_tensors(1)
    crv.crv_analysis(p.handle, m, Wp, None, 1)
    crv.crv_analysis(q.handle, m, Wq, None, 1)
    torch.cuda.synchronize()
    for j in range(J0, p.J + 1):
        assert torch.equal(Wp[j], Wq[j]), j
    p.close()
    out = q.map_tensor(1)
    crv.crv_synthesis(q.handle, Wq, None, out, 1)
    crv.crv_plan_check(q.handle)
    # without the scaling term the round trip misses only the scaling part; compare with it
    Wphi = q.Wphi_tensor(1)
    crv.crv_analysis(q.handle, m, Wq, Wphi, 1)
    crv.crv_synthesis(q.handle, Wq, Wphi, out, 1)
    crv.crv_plan_check(q.handle)
    assert rel_l2(map_from_device(out, True), fmap) < 1e-5
    q.close()
