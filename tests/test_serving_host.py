"""Serving scheduler logic on the host (no GPU): admission by memory footprint, plan reuse and
extra instances, passing of a request that does not fit, rejection of unsupported band limits,
latency percentiles and the Poisson arrival stream."""
import numpy as np
import pytest

from paper_1511_05578_gb300 import serving as S


class FakeExecutor:
    """Virtual clock; a request runs for B * L / 1000 seconds; plans cost L^2 bytes."""

    def __init__(self):
        self.t = 0.0
        self.created = []
        self.destroyed = []

    def plan_bytes(self, key):
        return key[0] ** 2

    def create_plan(self, key):
        if key[0] > S.MAX_L:
            raise ValueError("unsupported")
        self.created.append(key)
        return object()

    def destroy_plan(self, plan):
        self.destroyed.append(plan)

    def start(self, req, plan):
        return {"end": self.t + req.B * req.L / 1000.0, "rid": req.rid}

    def done(self, h):
        return self.t >= h["end"]

    def finish(self, h):
        return h["rid"]

    def now(self):
        return self.t

    def sleep(self, s):
        self.t += 0.01


def _req(rid, L, B=1, spin=0, t=0.0):
    return S.Request(rid=rid, L=L, spin=spin, B=B, arrival=t)


def test_concurrent_admission_and_completion():
    ex = FakeExecutor()
    budget = 3 * (S.request_bytes(_req(0, 64)) + 64 ** 2)
    sch = S.Scheduler(ex, budget, max_running=8)
    reqs = [_req(i, 64) for i in range(3)]
    wall = S.run(sch, reqs)
    assert len(sch.done) == 3 and not sch.rejected
    # all three fit at once: three plan instances, all started at t = 0
    assert len(ex.created) == 3
    assert all(r.start == 0.0 for r in reqs)
    assert wall == pytest.approx(0.07, abs=0.02)
    assert sch.used == sum(e[0] ** 2 for e in [(64,)] * 3)  # plans stay resident


def test_plan_reuse_when_memory_allows_one_instance():
    ex = FakeExecutor()
    budget = S.request_bytes(_req(0, 64)) + 64 ** 2  # one plan + one request
    sch = S.Scheduler(ex, budget)
    reqs = [_req(i, 64) for i in range(3)]
    S.run(sch, reqs)
    assert len(sch.done) == 3
    assert ex.created == [(64, 0, True)]  # one instance, reused in turn
    starts = sorted(r.start for r in reqs)
    assert starts[1] >= starts[0] + 0.064 - 1e-9 and starts[2] >= starts[1] + 0.064 - 1e-9


def test_small_request_passes_one_that_does_not_fit():
    ex = FakeExecutor()
    first, big, small = _req(0, 128, B=4), _req(1, 128, B=4), _req(2, 32)
    budget = S.request_bytes(big) + 128 ** 2 + S.request_bytes(small) + 32 ** 2
    sch = S.Scheduler(ex, budget)
    S.run(sch, [first, big, small])
    # `big` waits for `first` (second 128 plan does not fit), `small` starts at once
    assert small.start == 0.0 and first.start == 0.0
    assert big.start >= first.start + 0.512 - 1e-9
    assert len(sch.done) == 3


def test_rejections():
    ex = FakeExecutor()
    sch = S.Scheduler(ex, 10 ** 9)
    too_large_L = _req(0, 2048)
    too_big = _req(1, 1024, B=8)  # W alone is 37 GB > 1 GB budget
    ok = _req(2, 16)
    S.run(sch, [too_large_L, too_big, ok])
    assert {r.rid for r in sch.rejected} == {0, 1}
    assert "2048" in too_large_L.reason and "budget" in too_big.reason
    assert [r.rid for r in sch.done] == [2]


def test_percentiles_and_stats():
    assert S.percentile([5, 1, 3, 2, 4], 50) == 3
    assert S.percentile(list(range(1, 101)), 99) == 99
    assert S.percentile([7], 99) == 7
    ex = FakeExecutor()
    sch = S.Scheduler(ex, 10 ** 9)
    S.run(sch, [_req(i, 32, t=0.1 * i) for i in range(5)])
    st = sch.stats(1.0)
    assert st["requests_done"] == 5 and st["maps_done"] == 5
    assert st["p50_ms"] <= st["p99_ms"]


def test_poisson_stream_is_seeded():
    a = S.poisson_requests(50, 4.0, [128, 256], [0, 2], (1, 8), seed=3)
    b = S.poisson_requests(50, 4.0, [128, 256], [0, 2], (1, 8), seed=3)
    assert [(r.L, r.spin, r.B, r.arrival) for r in a] == [(r.L, r.spin, r.B, r.arrival) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert gaps.min() > 0 and abs(gaps.mean() - 0.25) < 0.1
    assert {r.L for r in a} == {128, 256} and all(1 <= r.B <= 8 for r in a)


def test_w_bytes_matches_grid_sizes():
    # L = 1024, lambda = 2, J0 = 2: scales j = 2..10 with L_j = 8, 16, ..., 1024, 1024
    Ls = [8, 16, 32, 64, 128, 256, 512, 1024, 1024]
    assert S.w_bytes(1024, 0) == sum(Lb * (2 * Lb - 1) ** 2 * 4 for Lb in Ls)
    assert S.w_bytes(1024, 2) == 2 * S.w_bytes(1024, 0)


def test_idle_resident_plans_are_evicted_when_a_request_would_not_fit():
    """Plans stay resident after their requests; a request of another band limit that fits only
    without them frees the idle ones instead of waiting for ever."""
    ex = FakeExecutor()
    a, b = _req(0, 64), _req(1, 96, t=0.5)
    budget = max(S.request_bytes(a) + 64 ** 2, S.request_bytes(b) + 96 ** 2) + 10
    assert S.request_bytes(a) + 64 ** 2 + S.request_bytes(b) + 96 ** 2 > budget
    sch = S.Scheduler(ex, budget, max_running=4)
    S.run(sch, [a, b])
    assert len(sch.done) == 2 and not sch.rejected
    assert sch.evicted == 1 and len(ex.destroyed) == 1
    assert b.start >= a.finish
    assert sch.used == 96 ** 2  # only b's plan stays resident
    assert sch.stats(1.0)["plans_evicted"] == 1


class SharingExecutor(FakeExecutor):
    """Instances of a key share tables of L^2 bytes; each has a workspace of L bytes."""

    def __init__(self):
        super().__init__()
        self.live = {}

    def plan_bytes(self, key):
        return key[0] if self.live.get(key) else key[0] ** 2 + key[0]

    def create_plan(self, key):
        plan = super().create_plan(key)
        self.live.setdefault(key, []).append(plan)
        self.keys = getattr(self, "keys", {})
        self.keys[id(plan)] = key
        return plan

    def _key(self, plan):
        return self.keys[id(plan)]

    def added_bytes(self, plan):
        k = self._key(plan)
        return k[0] + (k[0] ** 2 if len(self.live[k]) == 1 else 0)

    def freed_bytes(self, plan):
        k = self._key(plan)
        return k[0] + (k[0] ** 2 if len(self.live[k]) == 1 else 0)

    def destroy_plan(self, plan):
        freed = self.freed_bytes(plan)
        k = self._key(plan)
        self.live[k] = [q for q in self.live[k] if q is not plan]
        super().destroy_plan(plan)
        return freed


def test_shared_tables_admit_concurrent_instances_for_their_workspace():
    """With tables shared between instances of a key, a second concurrent request of the same
    key needs only a workspace: two fit at once in a budget that holds one table set, and the
    accounting returns to the tables alone once everything but one instance is evicted."""
    ex = SharingExecutor()
    L = 64
    rb = S.request_bytes(_req(0, L))
    budget = L ** 2 + 2 * L + 2 * rb  # one table set, two workspaces, two requests
    sch = S.Scheduler(ex, budget, max_running=8)
    reqs = [_req(i, L) for i in range(2)]
    S.run(sch, reqs)
    assert len(sch.done) == 2 and all(r.start == 0.0 for r in reqs)
    assert len(ex.created) == 2
    assert sch.used == L ** 2 + 2 * L
    # a request of another key that needs the room evicts both idle instances: the clone frees
    # its workspace, the last one the tables too, and the accounting comes back to zero + new
    big = _req(9, 32, B=1)
    sch.budget = S.request_bytes(big) + 32 ** 2 + 32
    S.run(sch, [big])
    assert len(ex.destroyed) == 2 and sch.used == 32 ** 2 + 32
