"""Serving loop for curvelet round trips of mixed band limit and spin.

A request asks for B maps of band limit L and spin s to be analysed into curvelet
coefficients (Sec. II-D, Eq. wav_analysis_harmonic) and synthesised back (Eq.
wav_synthesis_harmonic); the coefficients stay on the device for the duration of the request
and the reconstructed maps go back to the host. Requests arrive over time. The scheduler
admits a request as soon as a plan for its (L, s) is idle (or another instance fits) and its
transient buffers fit in the device-memory budget; admitted requests run concurrently, each on
its own CUDA stream with its own plan instance (a plan serves one stream at a time), and
completions are detected with CUDA events. Instances of the same (L, s) share the plan's
read-only tables (Delta, the tensor-core Delta Psi tables, FFT tables: crv_plan_clone), so a
second concurrent request of a key costs only a workspace. Requests that arrive while others run are thereby
admitted as plans and memory free up (continuous batching at request granularity); the queue is
served first-come first-served, except that a request that does not fit may be passed by later
ones that do. Band limits the library does not support are rejected at admission.

The scheduling logic (`Scheduler`) is plain Python over an executor interface, so it can be
exercised without a GPU; `CudaExecutor` runs requests through the C ABI.
"""
import heapq
import math
import time
from dataclasses import dataclass

import numpy as np

from . import inputs

MAX_L = 1024  # crv_plan_create returns CRV_EUNSUPPORTED above this band limit
BATCH_L = 256  # up to this band limit a request's maps go through one call (the plan's map
MAX_B = 8      # workers run them concurrently); above it one map per call reuses one W


class NoMemory(Exception):
    """A plan instance could not be allocated now (device memory held by others)."""


@dataclass
class Request:
    rid: int
    L: int
    spin: int
    B: int
    arrival: float                  # seconds on the scheduler's clock
    maps: object = None             # host array [B][L][2L-1] (real) or [B][L][2L-1][2]; None: generated
    seed: int = 0
    # filled by the scheduler
    start: float = None
    finish: float = None
    status: str = "pending"         # pending | running | done | rejected
    reason: str = ""
    result: object = None           # host array of the reconstructed maps
    dev_events: object = None       # (start, end) CUDA events of the request's device work


def plan_key(req, mixed):
    return (req.L, req.spin, mixed)


def w_bytes(L, spin, lam=2.0, J0=2, w_fp32=True):
    """Device bytes of one map's curvelet coefficients W_j for all scales j >= J0 (Sec. III-A:
    L_j x (2L_j - 1) x (2L_j - 1) samples per scale), real for spin 0, complex otherwise."""
    J = 0
    while lam ** J < L * (1 - 1e-14):
        J += 1
    el = (4 if w_fp32 else 8) * (1 if spin == 0 else 2)
    tot = 0
    for j in range(J0, J + 1):
        v = lam ** (j + 1)
        Lb = min(L, int(round(v)) if abs(v - round(v)) < 1e-9 * max(1.0, v) else int(math.ceil(v)))
        N = 2 * Lb - 1
        tot += Lb * N * N * el
    return tot


def plan_estimate(L, spin, mixed=True):
    """Device bytes of a first plan instance before one exists (tables + workspace), from the
    library's allocations: Delta^l(pi/2) for l < L (L^3 doubles, and floats when mixed); the
    tensor-core Delta Psi tables of both directions (about 17 L^2 Nc bytes over all scales);
    two (m, n, m') volumes; the per-map A tables of the tensor-core analysis; the ring buffer.
    m runs over L values (real spin 0) or 2L - 1; n over about L (spin 0: even n) or 2L - 1."""
    mc = L if spin == 0 else 2 * L - 1
    nc = L if spin == 0 else 2 * L - 1
    ring = min(L * (2 * L) * max(mc, nc) * (8 if mixed else 16), 256 << 20)
    if mixed:
        return 12 * L ** 3 + 17.2 * L * L * nc + 2 * 8 * L * mc * nc + 8 * L * L * mc + ring
    return 8 * L ** 3 + 2 * 16 * L * mc * nc + ring


def request_bytes(req, w_fp32=True):
    """Transient device bytes of a request: the coefficients W of one map (maps processed one
    after the other, W reused), or of all B maps when they go through one call (L <= BATCH_L),
    plus the B input and B output maps and the scaling coefficients."""
    mapb = req.L * (2 * req.L - 1) * 8 * (1 if req.spin == 0 else 2)
    nw = req.B if req.L <= BATCH_L else 1
    return nw * w_bytes(req.L, req.spin, w_fp32=w_fp32) + 2 * req.B * mapb + 2 * nw * mapb


def percentile(xs, q):
    """Nearest-rank percentile (q in [0, 100]) of a non-empty list."""
    s = sorted(xs)
    k = max(0, min(len(s) - 1, int(math.ceil(q / 100.0 * len(s))) - 1))
    return s[k]


class Scheduler:
    """Admission and accounting. The executor provides:
        plan_bytes(key) -> bytes a new plan instance of this key would add (with tables shared
                           between instances: the workspace alone once an instance exists)
        create_plan(key) -> plan object (or raises ValueError with a reason when unsupported)
        destroy_plan(plan) -> bytes freed or None (then the bytes it added are assumed); idle
                           plans are evicted, largest first, when a request would not fit
                           otherwise
        freed_bytes(plan) -> bytes destroy_plan would free (optional; default: bytes it added)
        added_bytes(plan) -> bytes a just-created instance holds beyond what existed (optional;
                           replaces the estimate plan_bytes gave before it existed)
        start(req, plan) -> handle;  done(handle) -> bool;  finish(handle) -> result
        now() -> seconds
    """

    def __init__(self, executor, budget_bytes, mixed=True, max_running=8):
        self.ex = executor
        self.budget = budget_bytes
        self.mixed = mixed
        self.max_running = max_running
        self.used = 0                      # bytes held by plans and running requests
        self.plans = {}                    # key -> list of [plan, busy, bytes added]
        self.queue = []                    # admitted order: list of requests waiting
        self.running = []                  # (req, plan_entry, handle, bytes)
        self.done = []
        self.rejected = []
        self.evicted = 0                   # idle plan instances freed to admit a request

    def _idle_plan(self, key):
        for e in self.plans.get(key, []):
            if not e[1]:
                return e
        return None

    def _try_start(self, req):
        key = plan_key(req, self.mixed)
        if req.L > MAX_L or req.L < 2:
            req.status, req.reason = "rejected", f"band limit {req.L} outside 2..{MAX_L}"
            return "rejected"
        rb = request_bytes(req)
        e = self._idle_plan(key)
        need = rb + (0 if e else self.ex.plan_bytes(key))
        if need > self.budget and not self.running:
            req.status, req.reason = "rejected", f"needs {need / 1e9:.1f} GB, budget {self.budget / 1e9:.1f} GB"
            return "rejected"
        if len(self.running) >= self.max_running:
            return "wait"
        if self.used + need > self.budget and not self._evict_idle(need, keep=e):
            # resident idle plans freed and it still does not fit: wait for running requests
            # (it fits alone, since need <= budget)
            return "wait"
        if e is None:
            added = self.ex.plan_bytes(key)
            try:
                plan = self.ex.create_plan(key)
            except ValueError as err:
                req.status, req.reason = "rejected", str(err)
                return "rejected"
            except NoMemory as err:
                # the estimate was short: free every idle plan and try once more, else wait for
                # the running requests (or reject when nothing else holds memory)
                self._evict_idle(self.budget + 1)
                try:
                    plan = self.ex.create_plan(key)
                except NoMemory:
                    if self.running:
                        return "wait"
                    req.status, req.reason = "rejected", f"no device memory for the plan: {err}"
                    return "rejected"
            measured = getattr(self.ex, "added_bytes", None)
            if measured is not None:  # what the new instance actually holds
                added = measured(plan)
            e = [plan, False, added]
            self.plans.setdefault(key, []).append(e)
            self.used += added
        e[1] = True
        self.used += rb
        req.status, req.start = "running", self.ex.now()
        self.running.append((req, e, self.ex.start(req, e[0]), rb))
        return "started"

    def _evict_idle(self, need, keep=None):
        """Free idle plan instances (largest first; never `keep`) until `need` more bytes fit.
        Returns whether they fit."""
        destroy = getattr(self.ex, "destroy_plan", None)
        if destroy is None:
            return False
        freed_of = getattr(self.ex, "freed_bytes", None)

        def frees(e):
            return freed_of(e[0]) if freed_of is not None else e[2]
        idle = [(k, e) for k, lst in self.plans.items() for e in lst if not e[1] and e is not keep]
        idle.sort(key=lambda ke: -frees(ke[1]))
        for k, e in idle:
            if self.used + need <= self.budget:
                break
            self.plans[k].remove(e)
            freed = destroy(e[0])
            self.used -= e[2] if freed is None else freed
            self.evicted += 1
        return self.used + need <= self.budget

    def submit(self, req):
        self.queue.append(req)

    def step(self):
        """Retire finished requests, then admit from the queue in order (later requests may
        pass one that does not fit). Returns True if anything changed."""
        changed = False
        still = []
        for (req, e, h, rb) in self.running:
            if self.ex.done(h):
                req.result = self.ex.finish(h)
                req.finish, req.status = self.ex.now(), "done"
                e[1] = False
                self.used -= rb
                self.done.append(req)
                changed = True
            else:
                still.append((req, e, h, rb))
        self.running = still
        waiting = []
        for req in self.queue:
            r = self._try_start(req)
            if r == "rejected":
                self.rejected.append(req)
                changed = True
            elif r == "started":
                changed = True
            else:
                waiting.append(req)
        self.queue = waiting
        return changed

    def idle(self):
        return not self.queue and not self.running

    def stats(self, wall_s):
        lat = [r.finish - r.arrival for r in self.done]
        maps = sum(r.B for r in self.done)
        out = {"requests_done": len(self.done), "requests_rejected": len(self.rejected), "maps_done": maps,
               "maps_per_s": maps / wall_s if wall_s > 0 else 0.0, "plans_evicted": self.evicted}
        if lat:
            out.update({"p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
                        "mean_ms": 1e3 * sum(lat) / len(lat)})
        return out


def poisson_requests(n, rate_per_s, Ls, spins, B_range, seed=0):
    """n requests with exponential inter-arrival times (Poisson stream), L, spin and B drawn
    uniformly; deterministic for a seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        out.append(Request(rid=i, L=int(rng.choice(Ls)), spin=int(rng.choice(spins)),
                           B=int(rng.integers(B_range[0], B_range[1] + 1)), arrival=t, seed=1000 * 4 + i))
    return out


def run(scheduler, requests, clock_start=None, poll_s=0.0005):
    """Feed requests to the scheduler at their arrival times (relative to the clock at the
    call) and drive it until every request is done or rejected. Returns the wall time."""
    ex = scheduler.ex
    t0 = ex.now() if clock_start is None else clock_start
    pending = [(r.arrival, r.rid, r) for r in requests]
    heapq.heapify(pending)
    while pending or not scheduler.idle():
        now = ex.now() - t0
        while pending and pending[0][0] <= now:
            _, _, r = heapq.heappop(pending)
            r.arrival = t0 + r.arrival
            scheduler.submit(r)
        if not scheduler.step():
            ex.sleep(poll_s)
    return ex.now() - t0


class CudaExecutor:
    """Runs requests through the C ABI: one CUDA stream and one plan instance per running
    request, results read back on that stream, completion by CUDA event."""

    def __init__(self, lam=2.0, J0=2, mixed=True, share_tables=True):
        import torch
        import paper_1511_05578_gb300 as crv
        self.torch, self.crv = torch, crv
        self.lam, self.J0, self.mixed = lam, J0, mixed
        self.share = share_tables
        self._plan_bytes = {}     # key -> (table bytes, workspace bytes) measured on an instance
        self._live = {}           # key -> live plan instances (they share one table set)

    def flags(self, L, spin):
        c = self.crv
        f = c.CRV_F_REAL if spin == 0 else 0
        if self.mixed:
            f |= c.CRV_F_MIXED | c.CRV_F_W_FP32
        return f

    def plan_bytes(self, key):
        """Bytes the next instance of `key` adds: its workspace when an instance exists (tables
        shared), tables and workspace otherwise (measured once an instance has existed)."""
        if key in self._plan_bytes:
            tb, wb = self._plan_bytes[key]
            return wb if (self.share and self._live.get(key)) else tb + wb
        L, spin, mixed = key
        # estimate before the first instance exists (the plan's own count replaces it once one
        # does): Delta tables (FP64, + FP32, the tensor-core B tables of both directions and the
        # per-map A tables when mixed) and the two (m, n, m') workspaces, complex, m over
        # 2L - 1 values for spin != 0
        return plan_estimate(L, spin, mixed)

    def _key_of(self, plan):
        for k, lst in self._live.items():
            if any(q is plan for q in lst):
                return k
        return None

    def freed_bytes(self, plan):
        """Bytes destroy_plan(plan) would free: its workspace, and the tables when it is the
        last instance of its key."""
        k = self._key_of(plan)
        tb, wb = plan.table_bytes(), plan.own_bytes()
        return wb + (tb if (k is None or len(self._live[k]) == 1 or not self.share) else 0)

    def added_bytes(self, plan):
        """Bytes a just-created instance added: its workspace, and the tables if it is the
        only instance of its key."""
        k = self._key_of(plan)
        tb, wb = plan.table_bytes(), plan.own_bytes()
        return wb + (tb if (k is None or len(self._live[k]) == 1 or not self.share) else 0)

    def destroy_plan(self, plan):
        freed = self.freed_bytes(plan)
        k = self._key_of(plan)
        if k is not None:
            self._live[k] = [q for q in self._live[k] if q is not plan]
        plan.close()
        return freed

    def create_plan(self, key):
        L, spin, mixed = key
        if L > MAX_L:
            raise ValueError(f"band limit {L} > {MAX_L} (unsupported by the library)")
        J0 = self.J0
        while self.lam ** J0 < abs(spin):  # theta^j needs lambda^J0 >= |s|
            J0 += 1
        live = self._live.setdefault(key, [])
        try:
            if self.share and live:
                p = live[0].clone()
            else:
                p = self.crv.Plan(L, self.lam, J0, spin, self.flags(L, spin), max_batch=MAX_B if L <= BATCH_L else 1)
        except self.crv.CrvError as err:
            if err.status == self.crv.CRV_ENOMEM:
                raise NoMemory(str(err)) from err
            raise
        self._plan_bytes[key] = (p.table_bytes(), p.own_bytes())
        live.append(p)
        return p

    def now(self):
        return time.perf_counter()

    def sleep(self, s):
        time.sleep(s)

    def start(self, req, plan):
        """Queue the request on a new stream: inputs (given maps from pinned host memory, or
        f_lm from the package's seeded generator turned into maps by the library's inverse
        SHT), analysis and synthesis of each map, and the read-back of the results."""
        torch, crv = self.torch, self.crv
        s = torch.cuda.Stream()
        real = req.spin == 0
        shape = (req.B, req.L, 2 * req.L - 1) + (() if real else (2,))
        out_host = torch.empty(shape, dtype=torch.float64).pin_memory()
        keep = [s]
        with torch.cuda.stream(s):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(s)
            if req.maps is not None:
                host = torch.from_numpy(np.ascontiguousarray(req.maps, dtype=np.float64)).pin_memory()
                dmaps = host.to("cuda", non_blocking=True)
                keep.append(host)
            else:
                power = 3.0 if req.spin == 2 else 2.0
                f = np.stack([inputs.flm_gaussian(req.L, req.seed + b, req.spin, real, power) for b in range(req.B)])
                fh = torch.from_numpy(f).pin_memory()
                fd = fh.to("cuda", non_blocking=True)
                dmaps = torch.empty(shape, dtype=torch.float64, device="cuda")
                for b in range(req.B):
                    crv.crv_sht_inv(plan.handle, fd[b:b + 1], dmaps[b:b + 1], 1, stream=s)
                keep += [fh, fd]
            nb = req.B if (req.L <= BATCH_L and req.B <= plan.max_batch) else 1  # maps per call
            W = plan.W_tensors(nb)
            Wphi = plan.Wphi_tensor(nb)
            dout = torch.empty_like(dmaps)
            for b in range(0, req.B, nb):
                crv.crv_analysis(plan.handle, dmaps[b:b + nb], W, Wphi, nb, stream=s)
                crv.crv_synthesis(plan.handle, W, Wphi, dout[b:b + nb], nb, stream=s)
            out_host.copy_(dout, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        req.dev_events = (ev0, ev)
        keep += [dmaps, W, Wphi, dout]
        return {"ev": ev, "out": out_host, "keep": keep, "plan": plan, "inputs": dmaps, "stream": s}

    def done(self, h):
        return h["ev"].query()

    def finish(self, h):
        """Reconstructed maps (host), after checking the plan's device-side error flag on the
        request's own stream (already complete: no wait, and no device-wide synchronisation
        that would stall the other running requests)."""
        self.crv.crv_plan_check_stream(h["plan"].handle, h["stream"])
        out = h["out"].numpy().copy()
        h.clear()
        return out


def main(argv=None):
    """Poisson-arrival serving run on cuda:0 (round trips of mixed L and spin); prints one JSON
    line with p50/p99 latency and maps/s. Plans for every (L, spin) in the mix are created
    before the clock starts (resident plans)."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--rate", type=float, default=2.0, help="mean arrivals per second")
    ap.add_argument("--Ls", default="128,256,512,1024")
    ap.add_argument("--spins", default="0,2")
    ap.add_argument("--B", default="1,8", help="batch range per request, inclusive")
    ap.add_argument("--budget-gb", type=float, default=0.0, help="device-memory budget (0: 90%% of free)")
    ap.add_argument("--max-running", type=int, default=4)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    Ls = [int(x) for x in a.Ls.split(",")]
    spins = [int(x) for x in a.spins.split(",")]
    b0, b1 = (int(x) for x in a.B.split(","))
    free, _ = torch.cuda.mem_get_info()
    budget = a.budget_gb * 1e9 if a.budget_gb > 0 else 0.9 * free
    ex = CudaExecutor()
    sch = Scheduler(ex, budget, mixed=True, max_running=a.max_running)
    for L in Ls:
        if L > MAX_L:
            continue
        for sp in spins:
            key = (L, sp, True)
            added = ex.plan_bytes(key)
            if sch.used + added + request_bytes(Request(0, L, sp, b1, 0.0)) <= budget:
                pl = ex.create_plan(key)
                added = ex.added_bytes(pl)
                sch.plans.setdefault(key, []).append([pl, False, added])
                sch.used += added
    torch.cuda.synchronize()
    reqs = poisson_requests(a.requests, a.rate, Ls, spins, (b0, b1), seed=a.seed)
    wall = run(sch, reqs)
    st = sch.stats(wall)
    st.update({"metric": "curvelet round-trip serving, Poisson arrivals", "unit": "maps/s", "wall_s": wall,
               "config": {"requests": a.requests, "rate_per_s": a.rate, "Ls": Ls, "spins": spins, "B": [b0, b1],
                          "budget_gb": budget / 1e9, "max_running": a.max_running, "precision": "mixed"},
               "rejected_reasons": sorted({r.reason for r in sch.rejected})})
    print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
