#!/usr/bin/env python3
"""Benchmark: curvelet analysis + synthesis throughput (maps/s) on one or more GPUs.

Workload (default): 32 real spin-0 maps per GPU, band limit L = 1024, lambda = 2,
J0 = 2, mixed precision (split-FP32 contraction, FP32 FFTs and W storage; FP64
Delta tables and FP64 f_lm accumulation). One step = for every map: forward SHT ->
curvelet analysis onto all SO(3) scale grids (W materialised in HBM) -> synthesis
-> inverse SHT. Inputs are seeded synthetic band-limited maps (Gaussian f_lm with
C_l = (l+1)^-2, seed 1000*2 + map index), 16.8 MB each, so one step's inputs (537 MB)
exceed the 126 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--L 1024] [--B 32]
                  [--mode mixed|fp64] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank runs its own 32 maps
(independent problems: weak scaling, no data-path collective); value = all ranks'
maps / max-over-ranks time.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PROF_MAPS = 2  # maps of the separate per-kind timing pass
METRIC = "maps/s analysis+synthesis at L=1024, mixed vs FP64 (err<=1e-5); p50/p99 ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--L", type=int, default=1024)
    ap.add_argument("--B", type=int, default=32)
    ap.add_argument("--lam", type=float, default=2.0)
    ap.add_argument("--J0", type=int, default=2)
    ap.add_argument("--mode", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--fp64-tc", action="store_true",
                    help="with --mode fp64: the contractions on the tensor cores at FP64 accuracy (CRV_F_FP64_TC)")
    ap.add_argument("--unrotated", action="store_true",
                    help="coefficients of the unrotated curvelets (CRV_F_UNROTATED: single-term l = |n| contraction)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-sample-maps", type=int, default=1,
                    help="maps timed on the plain FP64 path for the mixed/FP64 speedup (0 = skip)")
    ap.add_argument("--breakdown", action="store_true", help="print per-kernel-kind device time to stderr")
    ap.add_argument("--batch-calls", action="store_true",
                    help="one analysis and one synthesis call per step for all B maps (the plan's map workers run "
                         "them concurrently; small band limits), instead of one call per map")
    ap.add_argument("--maps-per-call", type=int, default=2,
                    help="maps per analysis/synthesis call (a divisor of B); with 2 or more the plan runs two "
                         "maps at once on two instances where memory allows")
    ap.add_argument("--tune", action="store_true", help="create the plan with CRV_F_TUNE (autotuned workers and ring chunks)")
    ap.add_argument("--graph", action="store_true",
                    help="capture one step (all its calls) into a CUDA graph after the warm-up and replay it "
                         "(no host launch cost per kernel; small band limits)")
    ap.add_argument("--serving-requests", type=int, default=24,
                    help="requests of the serving leg (Poisson arrivals; 0 = skip)")
    ap.add_argument("--serving-rate", type=float, default=0.5, help="mean arrivals per second of the serving leg")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per map (for the roofline object)
# ---------------------------------------------------------------------------
def plan_shapes(L, lam, J0, real=True, spin=0, unrot=False):
    J = 0
    while lam ** J < L * (1 - 1e-14):
        J += 1
    out = []
    for j in range(J0, J + 1):
        v = lam ** (j + 1)
        r = round(v)
        Lb = min(L, int(r) if abs(v - r) < 1e-9 * max(1, v) else int(math.ceil(v)))
        N = 2 * Lb - 1
        Mc = Lb if real else N
        if spin == 0 and not unrot:
            n0 = -(Lb - 1) + ((Lb - 1) % 2)
            Nc = (-n0 - n0) // 2 + 1
        else:
            Nc = N
        out.append((j, Lb, N, Mc, Nc))
    return J, out


def support_start(lam, j):
    """First l with kappa^(j)(l) > 0: the smallest integer above lam^(j-1) (kappa^(j) vanishes
    for l <= lam^(j-1), where both k_lambda arguments are at most 1/lam)."""
    v = lam ** (j - 1)
    r = round(v)
    return (int(r) if abs(v - r) < 1e-9 * max(1, v) else int(math.floor(v))) + 1


def contraction_terms(Lb, lmin=0, real=True, spin=0):
    """Number of (l, m, n, m'>=0) terms of the Delta contraction of one scale, over the l of the
    kernel's support (l >= lmin; Psi_ln = 0 below it)."""
    tot = 0
    for l in range(lmin, Lb):
        nm = (l + 1) if real else (2 * l + 1)       # m in the m-set with |m| <= l
        nn = 2 * (l // 2) + 1 if spin == 0 else 2 * l + 1  # even n (spin 0) with |n| <= l
        tot += (l + 1) * nm * nn                     # m' = 0..l
    return tot


def fft_flops(n):
    """Conventional algorithmic flop count of a complex DFT of length n: 5 n log2 n."""
    return 5.0 * n * math.log2(n) if n > 1 else 0.0


def kind_work(L, lam, J0, el_bytes, w_bytes, unrot=False):
    """Algorithmic bytes (input read + output written, once) and flops per map for each
    kernel kind of the Wigner pipelines. DFT flops use the conventional 5 N log2 N per
    complex length-N transform (half that for a real-input or real-output one); the
    beta quadrature adds its weight correlation as two length-Q transforms."""
    J, shapes = plan_shapes(L, lam, J0, unrot=unrot)
    w = {}

    def add(k, b=0.0, f=0.0):
        B0, F0 = w.get(k, (0.0, 0.0))
        w[k] = (B0 + b, F0 + f)
    for (j, Lb, N, Mc, Nc) in shapes:
        vol = Lb * Mc * Nc * el_bytes           # X, Xb, Y volumes (complex)
        wv = Lb * N * N * w_bytes               # W_j
        terms = contraction_terms(Lb, support_start(lam, j))
        Q = 1 << max(3, (4 * Lb - 4).bit_length())
        if unrot:
            # single term l = |n|: the volume is written (analysis) or read (synthesis) once
            terms = Lb * Lb * Lb
        add("contract_analysis", vol, 4.0 * terms)
        add("oz_analysis", vol, 4.0 * terms)
        add("tc_analysis", vol, 4.0 * terms)
        Nh = (Nc + 1) // 2                      # columns n >= 0 (real signals: F_{-m,-n} = conj F_{m,n})
        ring_h = Lb * N * Nh * el_bytes         # ring buffer [b][a][h]
        add("beta_synth", 2 * vol, Mc * Nc * fft_flops(N))
        add("ring_inv_m", vol + ring_h, Lb * Nh * fft_flops(N))
        add("ring_inv_n", ring_h + wv, Lb * N * 0.5 * fft_flops(N))
        add("ring_fwd_g", wv + ring_h, Lb * N * 0.5 * fft_flops(N))
        add("ring_fwd_a", ring_h + vol, Lb * Nh * fft_flops(N))
        add("beta_quad", 2 * vol, Mc * Nc * (fft_flops(N) + 2 * fft_flops(Q) + 6 * Q))
        add("contract_synthesis", vol, 4.0 * terms)
        add("oz_synthesis", vol, 4.0 * terms)
        add("tc_synthesis", vol, 4.0 * terms)
    return w


# The sources that define each kernel kind's device code: recorded DRAM traffic of a kind is
# used only while these are unchanged since the ncu capture that produced it.
KIND_SOURCES = {
    "fft": ["common.cuh", "fft.cuh", "transforms.cuh"],
    "tc": ["common.cuh", "fft.cuh", "transforms.cuh", "tc_gemm.cuh", "tc_contract.cuh", "tc_contract.cu"],
}


def kernel_source_hash(kind="fft"):
    """Hash of the CUDA sources that define a kernel kind (`fft` for the DFT and beta kinds,
    `tc` for the tensor-core contractions)."""
    d = os.path.join(ROOT, "paper_1511_05578_gb300", "csrc")
    files = KIND_SOURCES["tc" if kind.startswith("tc_") or kind == "tc" else "fft"]
    h = hashlib.sha256()
    for n in files:
        h.update(n.encode())
        with open(os.path.join(d, n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_workload(L, lam, J0, mode, unrot):
    """Key of the workload a recorded traffic figure belongs to."""
    return f"L={L},lambda={float(lam):g},J0={J0},{mode}" + (",unrotated" if unrot else "")


def recorded_traffic(kind, workload):
    """DRAM bytes (read + write) per launch of a kernel kind on a workload (from
    profiles/traffic.json), or None if absent, recorded for another workload, or taken on
    other sources of that kind."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(kind)
    if not e or e.get("source_hash") != kernel_source_hash(kind) or e.get("workload") != workload:
        return None
    return e.get("dram_bytes_per_launch")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


def fp32_alu_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flop per FMA at the sampled SM clock
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def fp64_alu_peak_tflops(sm_mhz):
    # FP64 FMA rate measured on this machine: 1.01 TFLOP/s at 1995 MHz (0.5 lane-FMA/clk/SM x 64)
    return 1.0124 * (sm_mhz or 1995.0) / 1995.0


# ---------------------------------------------------------------------------
# the oracle arm (CPU)
# ---------------------------------------------------------------------------
def oracle_maps_per_s(L, lam, J0, rings_per_sample=1, seed=2000, unrot=False):
    """Time the FP64 oracle's curvelet analysis on sampled rings of the top scale and
    extrapolate to one full map round trip: analysis cost per ring scales as L_j^3
    (Risbo recursion at beta_b plus the per-ring sums), summed over all rings of all
    scales; synthesis is taken as equal to analysis (its adjoint, same order of work);
    the two O(L^3) SHTs are left out (under 1% here)."""
    import numpy as np
    import oracle as O
    from paper_1511_05578_gb300 import inputs
    f = inputs.flm_gaussian(L, seed, real=True)
    J = O.J_max(lam, L)
    Lt = O.band_limit(lam, J, L)
    ps = O.psi(lam, J, 0, Lt, unrot)
    rings = list(np.linspace(0, Lt - 1, rings_per_sample + 2).astype(int)[1:-1])
    t0 = time.perf_counter()
    O.analysis_rings(f, lam, J, 0, L, rings=rings, psi_j=ps)
    dt = (time.perf_counter() - t0) / len(rings)
    total = 0.0
    for j in range(J0, J + 1):
        Lb = O.band_limit(lam, j, L)
        total += Lb * dt * (Lb / Lt) ** 3
    per_map = 2.0 * total
    return 1.0 / per_map, {"ring_s": dt, "rings": len(rings), "per_map_s": per_map}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def max_over_ranks(x, world, device):
    """The largest x over all ranks, known to every rank (x itself when world == 1): the
    whole-job time of a replicated run is that of its slowest rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, maps_per_rank, steps, t_ms):
    """Maps per second of the whole job: every rank's maps over the max-over-ranks time."""
    return world * maps_per_rank * steps / (t_ms / 1000.0)


def rank_map_seeds(rank, B):
    """Seeds of a rank's B maps: ranks draw disjoint maps of the same distribution."""
    from paper_1511_05578_gb300 import inputs
    return [inputs.seed_for(2, rank * B + b) for b in range(B)]


def run_reference(args, rank, world):
    # the oracle runs on rank 0 only
    if rank != 0:
        return
    vals = []
    rings = 4  # ~2-3 s of oracle work per step on 16 host cores at L = 1024
    for _ in range(args.warmup):
        oracle_maps_per_s(args.L, args.lam, args.J0, 1, unrot=args.unrotated)
    for _ in range(args.steps):
        v, info = oracle_maps_per_s(args.L, args.lam, args.J0, rings, unrot=args.unrotated)
        vals.append(v)
    v = sorted(vals)[len(vals) // 2]
    sample = (f"{rings} rings of the top scale (L_j={args.L}) per step, extrapolated by L_j^3 over all rings of "
              f"all scales, synthesis = analysis; {info['ring_s']:.2f} s per ring")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "maps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * args.B / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args),
        "cpu_baseline": {"value": v, "unit": "maps/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def serving_leg(args):
    """Continuous-batching serving of round-trip requests (the serving workload: Poisson
    arrivals, L uniform in {128, 256, 512, 1024, 2048}, spin in {0, 2}, 1-8 maps per request,
    mixed precision), run after the headline plans are freed. Plans for every (L, spin) are
    built before the clock (resident plans); instances of a key share their tables. Returns
    p50/p99 request latency, maps/s over the wall time, requests done and rejected (with the
    reasons: L = 2048 is beyond this build's band limit)."""
    import torch
    from paper_1511_05578_gb300 import serving as S
    Ls, spins, Bs = [128, 256, 512, 1024, 2048], [0, 2], (1, 8)
    free = torch.cuda.mem_get_info()[0]
    budget = 0.9 * free
    ex = S.CudaExecutor(lam=args.lam, J0=args.J0)
    sch = S.Scheduler(ex, budget, mixed=True, max_running=4)
    for L in Ls:
        if L > S.MAX_L:
            continue
        for sp in spins:
            key = (L, sp, True)
            if sch.used + ex.plan_bytes(key) + S.request_bytes(S.Request(0, L, sp, Bs[1], 0.0)) <= budget:
                pl = ex.create_plan(key)
                added = ex.added_bytes(pl)
                sch.plans.setdefault(key, []).append([pl, False, added])
                sch.used += added
    torch.cuda.synchronize()
    reqs = S.poisson_requests(args.serving_requests, args.serving_rate, Ls, spins, Bs, seed=0)
    wall = S.run(sch, reqs)
    st = sch.stats(wall)
    out = {"p50_ms": st.get("p50_ms"), "p99_ms": st.get("p99_ms"), "maps_per_s": st["maps_per_s"],
           "admitted": st["requests_done"], "rejected": st["requests_rejected"], "maps_done": st["maps_done"],
           "wall_s": wall, "plans_evicted": st["plans_evicted"],
           "rejected_reasons": sorted({r.reason for r in sch.rejected}),
           "config": {"requests": args.serving_requests, "rate_per_s": args.serving_rate, "Ls": Ls, "spins": spins,
                      "maps_per_request": list(Bs), "budget_gb": budget / 1e9, "max_running": 4,
                      "precision": "mixed", "latency": "arrival to reconstructed maps on the host"}}
    for lst in sch.plans.values():
        for e in lst:
            ex.destroy_plan(e[0])
    return out


def config_dict(args):
    return {"workload": f"curvelet analysis+synthesis, {args.B} real spin-0 maps, L={args.L}, lambda={args.lam:g}, "
                        f"J0={args.J0}, {'mixed precision (split-FP32 contraction, FP32 FFT/W)' if args.mode == 'mixed' else 'plain FP64'}"
                        + (", FP64-accurate contractions on tensor cores" if args.mode == "fp64" and args.fp64_tc else "")
                        + (", unrotated curvelets (O(L^3) single-term contraction)" if args.unrotated else ""),
            "L": args.L, "maps_per_gpu": args.B, "lambda": args.lam, "J0": args.J0, "spin": 0, "real": True,
            "precision": args.mode, "unrotated": bool(args.unrotated), "maps_per_call": args.maps_per_call if not args.batch_calls else args.B,
            "cuda_graph": bool(args.graph),
            "l2": "inputs larger than L2 (537 MB maps per step; W_j 36.8 GB per map)" if args.L >= 1024 else
                  "inputs of a step smaller than L2 at this band limit"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1511_05578_gb300 as crv
    from paper_1511_05578_gb300 import build, inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    L, lam, J0, B = args.L, args.lam, args.J0, args.B
    flags = crv.CRV_F_REAL | (crv.CRV_F_MIXED | crv.CRV_F_W_FP32 if args.mode == "mixed" else 0)
    if args.mode == "fp64" and args.fp64_tc:
        flags |= crv.CRV_F_FP64_TC
    unrot_flag = crv.CRV_F_UNROTATED if args.unrotated else 0
    flags |= unrot_flag
    if args.tune:
        flags |= crv.CRV_F_TUNE
    nb = B if args.batch_calls else max(1, args.maps_per_call)  # maps per call
    nb = math.gcd(B, min(nb, B))  # a divisor of B (B = 1: one map per call)
    args.maps_per_call = nb
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = crv.Plan(L, lam, J0, 0, flags, max_batch=nb, stream=stream.cuda_stream)
        # seeded inputs: f_lm on the host -> maps through our inverse SHT (not timed)
        maps = torch.empty((B, L, 2 * L - 1), dtype=torch.float64, device="cuda")
        f1 = plan.flm_tensor(1)
        for b, seed in enumerate(rank_map_seeds(rank, B)):
            f1.copy_(torch.from_numpy(inputs.flm_gaussian(L, seed, real=True)[None]))
            crv.crv_sht_inv(plan.handle, f1, maps[b:b + 1], 1, stream.cuda_stream)
        tuning = crv.crv_plan_tuning(plan.handle)
        out = torch.empty_like(maps)
        W = plan.W_tensors(nb)
        Wphi = plan.Wphi_tensor(nb)
    torch.cuda.synchronize()

    def step(src, dst):
        for b in range(0, B, nb):
            crv.crv_analysis(plan.handle, src[b:b + nb], W, Wphi, nb, stream.cuda_stream)
            crv.crv_synthesis(plan.handle, W, Wphi, dst[b:b + nb], nb, stream.cuda_stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(maps, out)
    torch.cuda.synchronize()
    # accuracy of the round trip on this rank's last map (FP32 W / mixed: <= 1e-5 relative)
    recon = float(torch.linalg.vector_norm(out[-1] - maps[-1]) / torch.linalg.vector_norm(maps[-1]))

    graph = None
    if args.graph:
        # one step's calls captured once (the plan's per-call path allocates nothing and never
        # synchronises, its worker streams fork and join by events), replayed every step
        graph = torch.cuda.CUDAGraph()
        lc0 = crv.crv_launch_count()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                step(maps, out)
        graph_launches = crv.crv_launch_count() - lc0  # kernels in the graph (counted at capture)
        with torch.cuda.stream(stream):
            graph.replay()  # one more warm-up, as the replays below
        torch.cuda.synchronize()
    kinds = crv.crv_profile_kinds()
    l0 = crv.crv_launch_count()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_step, per_map = [], []
    ev0.record(stream)
    for _ in range(args.steps):
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if graph is not None:
            with torch.cuda.stream(stream):
                graph.replay()
            per_map.append((a, None))
        else:
            for b in range(0, B, nb):  # one step = all B maps; per-call events give the latency distribution
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                crv.crv_analysis(plan.handle, maps[b:b + nb], W, Wphi, nb, stream.cuda_stream)
                crv.crv_synthesis(plan.handle, W, Wphi, out[b:b + nb], nb, stream.cuda_stream)
                e1.record(stream)
                per_map.append((e0, e1))
        b_.record(stream)
        per_step.append((a, b_))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = crv.crv_launch_count() - l0
    if graph is not None:
        launches = graph_launches * args.steps  # replays launch the captured kernels
    ms_total = ev0.elapsed_time(ev1)
    step_ms = [a.elapsed_time(b_) for a, b_ in per_step]
    # per-kind device times from a pass of their own after the timed region (no event records
    # in the timed steps): PROF_MAPS maps, one per call on one plan instance, so that no kernel
    # shares the GPU with a concurrent map's
    prof_maps = min(B, PROF_MAPS)
    crv.crv_profile_reset()
    crv.crv_profile_enable((1 << len(kinds)) - 1)
    for b in range(prof_maps):
        crv.crv_analysis(plan.handle, maps[b:b + 1], W, Wphi, 1, stream.cuda_stream)
        crv.crv_synthesis(plan.handle, W, Wphi, out[b:b + 1], 1, stream.cuda_stream)
    torch.cuda.synchronize()
    crv.crv_profile_enable(0)
    kind_ms = {}
    kind_n = {}
    for k, name in enumerate(kinds):
        n, t = crv.crv_profile_read(k)
        if n:
            kind_ms[name], kind_n[name] = t / prof_maps, n / prof_maps  # per map
    t_max = max_over_ranks(ms_total, world, "cuda")
    ms_per_step = t_max / args.steps
    value = whole_job_rate(world, B, args.steps, t_max)

    # per-map latency (p50 / p99) from the per-map events of the timed steps
    if graph is not None:  # a graph replay is one step: its duration is the latency
        per_map = per_step
    lat_ms = sorted(a.elapsed_time(b_) for a, b_ in per_map)
    p50 = lat_ms[len(lat_ms) // 2]
    p99 = lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)]

    # end to end through the public API with host buffers (pinned), copies in the timed region
    e2e = None
    if not args.no_e2e:
        host_in = maps.cpu().pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        dev_in = torch.empty((nb, L, 2 * L - 1), dtype=torch.float64, device="cuda")
        dev_out = torch.empty_like(dev_in)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for b in range(0, B, nb):  # the calls of the timed steps: nb maps per call
                dev_in.copy_(host_in[b:b + nb], non_blocking=True)
                crv.crv_analysis(plan.handle, dev_in, W, Wphi, nb, stream.cuda_stream)
                crv.crv_synthesis(plan.handle, W, Wphi, dev_out, nb, stream.cuda_stream)
                host_out[b:b + nb].copy_(dev_out, non_blocking=True)
        stream.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        nbytes = B * L * (2 * L - 1) * 8
        e2e = {"value": whole_job_rate(world, B, 1, 1000.0 * t_e2e), "unit": "maps/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}

    # plain FP64 GPU path on a sample of maps: the mixed/FP64 speedup, and the per-scale error
    # of the mixed coefficients against the FP64 path's on the same map (the FP64 path matches
    # the FP64 oracle to 1e-10 per scale at this size: tests/test_gpu_fullsize.py)
    fp64 = None
    if args.mode == "mixed" and args.fp64_sample_maps > 0 and rank == 0:
        with torch.cuda.stream(stream):
            crv.crv_analysis(plan.handle, maps[0:1], W, Wphi, 1, stream.cuda_stream)  # mixed W of map 0
        torch.cuda.synchronize()
        plan.close()
        torch.cuda.empty_cache()
        with torch.cuda.stream(stream):
            p64 = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL | unrot_flag, max_batch=1, stream=stream.cuda_stream)
            W64 = p64.W_tensors(1)
            P64 = p64.Wphi_tensor(1)
            o64 = torch.empty_like(maps[:1])
        torch.cuda.synchronize()
        n64 = args.fp64_sample_maps
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        crv.crv_profile_reset()
        crv.crv_profile_enable((1 << len(kinds)) - 1)
        a.record(stream)
        for i in range(n64):
            crv.crv_analysis(p64.handle, maps[i:i + 1], W64, P64, 1, stream.cuda_stream)
            crv.crv_synthesis(p64.handle, W64, P64, o64, 1, stream.cuda_stream)
        b_.record(stream)
        torch.cuda.synchronize()
        crv.crv_profile_enable(0)
        ms64 = a.elapsed_time(b_) / n64
        cc64 = sum(crv.crv_profile_read(kinds.index(k))[1] for k in ("contract_analysis", "contract_synthesis")) / n64
        rec64 = float(torch.linalg.vector_norm(o64[0] - maps[n64 - 1]) / torch.linalg.vector_norm(maps[n64 - 1]))
        if n64 > 1:
            with torch.cuda.stream(stream):
                crv.crv_analysis(p64.handle, maps[0:1], W64, P64, 1, stream.cuda_stream)
            torch.cuda.synchronize()
        per_scale = {}
        rings64 = {}
        for j in range(J0, plan.J + 1):
            ref = W64[j]
            per_scale[str(j)] = float(torch.linalg.vector_norm(W[j][:1].double() - ref) / torch.linalg.vector_norm(ref))
            Lb = plan.Lj[j]
            rings64[j] = ref[:, sorted({0, Lb // 3, Lb - 1})].clone()
        fp64 = {"maps_per_s": 1000.0 / ms64, "ms_per_map": ms64, "sample_maps": n64,
                "speedup_mixed_over_fp64": (1000.0 / ms64 and value / world / (1000.0 / ms64)),
                "roundtrip_rel_l2": rec64, "mixed_vs_fp64_rel_l2_per_scale": per_scale,
                "mixed_vs_fp64_rel_l2_max": max(per_scale.values())}
        p64.close()
        del W64, P64
        torch.cuda.empty_cache()
        if not args.unrotated:
            # the same map with the contractions on the tensor cores at FP64 accuracy: time per
            # map, and its coefficients on sampled rings of every scale against the CUDA-core path
            with torch.cuda.stream(stream):
                ptc = crv.Plan(L, lam, J0, 0, crv.CRV_F_REAL | crv.CRV_F_FP64_TC, max_batch=1,
                               stream=stream.cuda_stream)
                Wtc = ptc.W_tensors(1)
                Ptc = ptc.Wphi_tensor(1)
            torch.cuda.synchronize()
            crv.crv_profile_reset()
            crv.crv_profile_enable((1 << len(kinds)) - 1)
            a.record(stream)
            crv.crv_analysis(ptc.handle, maps[0:1], Wtc, Ptc, 1, stream.cuda_stream)
            crv.crv_synthesis(ptc.handle, Wtc, Ptc, o64, 1, stream.cuda_stream)
            b_.record(stream)
            torch.cuda.synchronize()
            crv.crv_profile_enable(0)
            mstc = a.elapsed_time(b_)
            kind_tc = {}
            for k, name in enumerate(kinds):
                n, t = crv.crv_profile_read(k)
                if n:
                    kind_tc[name] = t
            crv.crv_plan_check(ptc.handle)
            rtc = {}
            for j in range(J0, plan.J + 1):
                Lb = plan.Lj[j]
                got = Wtc[j][:, sorted({0, Lb // 3, Lb - 1})]
                rtc[str(j)] = float(torch.linalg.vector_norm(got - rings64[j]) / torch.linalg.vector_norm(rings64[j]))
            fp64["fp64_tc"] = {
                "ms_per_map": mstc, "speedup_over_fp64_cuda_cores": ms64 / mstc,
                "contraction_ms": kind_tc.get("oz_analysis", 0.0) + kind_tc.get("oz_synthesis", 0.0),
                "cuda_core_contraction_ms": cc64,
                "roundtrip_rel_l2": float(torch.linalg.vector_norm(o64[0] - maps[0]) / torch.linalg.vector_norm(maps[0])),
                "vs_fp64_cuda_cores_sampled_rings_rel_l2_max": max(rtc.values()),
                "kernels_ms": kind_tc}
            ptc.close()
            del Wtc, Ptc
        del rings64

    # roofline of the dominant kernel kind
    peaks = measured_peaks()
    el = 8 if args.mode == "mixed" else 16
    wb = 4 if args.mode == "mixed" else 8
    work = kind_work(L, lam, J0, el, wb, args.unrotated)
    dom = max(kind_ms, key=kind_ms.get) if kind_ms else None
    twl = traffic_workload(L, lam, J0, args.mode, args.unrotated)
    roof = None
    if dom:
        avg_ms = kind_ms[dom] / kind_n[dom]
        per_launch_units = kind_n[dom]  # launches of this kind per map
        bytes_map, flops_map = work.get(dom, (0.0, 0.0))
        if dom in ("contract_analysis", "contract_synthesis"):
            flops_launch = flops_map / per_launch_units
            peak = fp32_alu_peak_tflops(clk.get("sm_mhz")) if args.mode == "mixed" else fp64_alu_peak_tflops(clk.get("sm_mhz"))
            ach = flops_launch / (avg_ms * 1e-3) / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": recorded_traffic(dom, twl),
                    "peak_src": "FP32 FMA lanes x clock" if args.mode == "mixed" else "FP64 FMA rate measured on this pool"}
        elif dom in ("oz_analysis", "oz_synthesis"):
            flops_launch = flops_map / per_launch_units
            peak = peaks["bf16_tflops_sustained"] / 2.0  # TF32 = bf16 / 2 (nominal ratio)
            ach = flops_launch / (avg_ms * 1e-3) / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": recorded_traffic(dom, twl),
                    "peak_src": f"{peaks['src']} bf16 sustained / 2 (tf32); achieved counts FP64-accurate flops "
                                "(each one 28 TF32 slice products; slicing included)"}
        elif dom in ("tc_analysis", "tc_synthesis"):
            flops_launch = flops_map / per_launch_units
            peak = peaks["bf16_tflops_sustained"] / 2.0  # TF32 = bf16 / 2 (nominal ratio)
            ach = flops_launch / (avg_ms * 1e-3) / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": recorded_traffic(dom, twl),
                    "peak_src": f"{peaks['src']} bf16 sustained / 2 (tf32); achieved counts FP32-accurate flops"}
        else:
            # the DFT kernels are bound by FP32 (FP64) arithmetic, not by HBM: their
            # algorithmic bytes per launch are reported beside the ALU roofline
            bytes_launch = bytes_map / per_launch_units
            flops_launch = flops_map / per_launch_units
            peak = fp32_alu_peak_tflops(clk.get("sm_mhz")) if args.mode == "mixed" else fp64_alu_peak_tflops(clk.get("sm_mhz"))
            ach = flops_launch / (avg_ms * 1e-3) / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": recorded_traffic(dom, twl),
                    "peak_src": ("FP32 FMA lanes x clock" if args.mode == "mixed" else "FP64 FMA rate measured on this pool")
                    + "; achieved counts 5 N log2 N per DFT",
                    "hbm_gbs_algorithmic": bytes_launch / (avg_ms * 1e-3) / 1e9}
        roof["avg_launch_ms"] = avg_ms
        roof["launches"] = int(round(kind_n[dom] * prof_maps))
        roof["launches_per_map"] = per_launch_units
        roof["timing"] = f"CUDA events around each launch, separate pass of {prof_maps} maps, one per call"
    # whole-map roofline: per kernel kind the larger of its algorithmic flops over its pipe's
    # peak and its algorithmic bytes over HBM, summed over the kinds, against the measured time
    # per map
    roof_map = None
    if kind_ms:
        sm = clk.get("sm_mhz")
        hbm = peaks["hbm_gbs"] * 1e9
        t_roof = 0.0
        parts = {}
        for k, (bts, fl) in work.items():
            if k not in kind_ms:
                continue
            if k.startswith(("tc_", "oz_")):  # tensor-core contractions: the TF32 pipe
                pk = peaks["bf16_tflops_sustained"] / 2.0 * 1e12
            elif args.mode == "mixed":
                pk = fp32_alu_peak_tflops(sm) * 1e12
            else:
                pk = fp64_alu_peak_tflops(sm) * 1e12
            t = max(fl / pk, bts / hbm) * 1e3
            parts[k] = t
            t_roof += t
        t_meas = ms_per_step / B
        roof_map = {"t_roof_ms": t_roof, "t_measured_ms": t_meas, "frac": t_roof / t_meas, "per_kind_roof_ms": parts,
                    "rule": "sum over kernel kinds of max(algorithmic flops / pipe peak, algorithmic bytes / HBM)"}

    line = {
        "metric": METRIC, "value": value, "unit": "maps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.mode == "mixed" else "f64", "data": "synthetic",
        "config": config_dict(args), "p50_ms": p50, "p99_ms": p99,
        "latency_unit": (f"ms per step ({B} maps, one CUDA graph replay)" if args.graph else
                         "ms per map (analysis+synthesis)" if nb == 1 else f"ms per call of {nb} maps (analysis+synthesis)"),
        "launches_per_map": launches / (args.steps * B), "plan_tuning": tuning,
        "roundtrip_rel_l2": recon, "gpu_launches": launches, "clocks": clk, "roofline": roof, "roofline_map": roof_map,
        "e2e": e2e,
        "fp64_path": fp64, "step_ms": step_ms,
        "kernels_ms_per_map": {k: v for k, v in sorted(kind_ms.items(), key=lambda kv: -kv[1])},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, info = oracle_maps_per_s(L, lam, J0, 20, unrot=args.unrotated)  # ~10-15 s of oracle work on 16 host cores
        line["cpu_baseline"] = {"value": v, "unit": "maps/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"FP64 oracle analysis of {info['rings']} rings of the top scale (L_j={L}, "
                                          f"{info['ring_s']:.2f} s per ring), extrapolated by L_j^3 over all rings of "
                                          f"all scales; synthesis taken equal to analysis"}
    if rank == 0 and world == 1 and args.serving_requests > 0:
        if plan.handle is not None:
            plan.close()
        del maps, out, W, Wphi
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        try:
            line["serving"] = serving_leg(args)
        except Exception as err:  # the bench line is printed whatever the serving leg does
            line["serving"] = {"error": f"{type(err).__name__}: {err}"}
    if args.breakdown and rank == 0:
        for k, v in sorted(kind_ms.items(), key=lambda kv: -kv[1]):
            sys.stderr.write(f"{k:20s} {v:10.2f} ms/map  {kind_n[k]:7.0f} launches/map\n")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if plan.handle is not None:
        plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
