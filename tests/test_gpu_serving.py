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
    spec = [(16, 0, 2), (32, 2, 1), (48, 0, 1), (16, 2, 2), (32, 0, 2), (48, 2, 1)]
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
    # several requests were on the device at once
    overlaps = sum(1 for a in mix for b in mix if a.rid < b.rid and b.start < a.finish and a.start < b.finish)
    assert overlaps >= 1
    for r in mix:
        alone = S.Request(rid=r.rid, L=r.L, spin=r.spin, B=r.B, arrival=0.0, maps=r.maps)
        s1 = S.Scheduler(S.CudaExecutor(), budget, max_running=1)
        S.run(s1, [alone])
        assert _rel(r.result, alone.result) < 1e-12, (r.rid, _rel(r.result, alone.result))
        assert _rel(r.result, r.maps) < 1e-5, (r.rid, _rel(r.result, r.maps))
    st = sch.stats(max(r.finish for r in mix) - min(r.arrival for r in mix))
    assert st["p50_ms"] <= st["p99_ms"]
