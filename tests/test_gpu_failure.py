"""Failure detection without a GPU fault: every device-side wait of the library is bounded and
reports through crv_plan_check. A probe thread waits on a barrier that nothing arrives at, with
a short limit; the next check reports CRV_ETIMEOUT once, and the plan and context stay usable
(a round trip afterwards is exact)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(__file__))

import paper_1511_05578_gb300 as crv  # noqa: E402
from gpu_util import case, map_from_device, map_to_device, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_bounded_wait_gives_up_and_reports_then_plan_still_works():
    L, lam, J0 = 32, 2.0, 2
    p = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED)
    crv.crv_plan_check(p.handle)  # clean state
    crv.crv_debug_bounded_wait(p.handle, 2000)
    with pytest.raises(crv.CrvError) as e:
        crv.crv_plan_check(p.handle)
    assert e.value.status == crv.CRV_ETIMEOUT
    crv.crv_plan_check(p.handle)  # the condition was cleared
    with pytest.raises(crv.CrvError):
        crv.crv_debug_bounded_wait(p.handle, 0)  # argument check, nothing launched
    # the context and the plan are intact: a mixed round trip still reconstructs
    _, fmap = case(L, lam, J0, 0, True, seed=5)
    W, Wphi, out = p.W_tensors(1), p.Wphi_tensor(1), p.map_tensor(1)
    crv.crv_analysis(p.handle, map_to_device(fmap, True), W, Wphi, 1)
    crv.crv_synthesis(p.handle, W, Wphi, out, 1)
    crv.crv_plan_check(p.handle)
    assert rel_l2(map_from_device(out, True), fmap) < 1e-5
    p.close()


def test_stream_ordered_check_reports_and_leaves_other_streams_alone():
    """crv_plan_check_stream reads the error flag in the order of one stream: a probe that
    gives up on stream s1 is reported by the check on s1, once; a check of a second plan on
    its own stream s2 is clean meanwhile."""
    L, lam, J0 = 32, 2.0, 2
    p1 = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED)
    p2 = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL | crv.CRV_F_MIXED)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    crv.crv_plan_check(p1.handle)
    crv.crv_debug_bounded_wait(p1.handle, 2000, s1)
    crv.crv_plan_check_stream(p2.handle, s2)  # the other plan's flag is clean
    with pytest.raises(crv.CrvError) as e:
        crv.crv_plan_check_stream(p1.handle, s1)
    assert e.value.status == crv.CRV_ETIMEOUT
    crv.crv_plan_check_stream(p1.handle, s1)  # cleared
    p1.close()
    p2.close()
