#!/usr/bin/env python3
"""Throughput of the FOSSILS least-squares hot path on GB300.

One step = one complete FOSSILS solve (sketch S[A b], Householder QR of the
sketch, sketch-and-solve start, two refinement steps with the Polyak inner
solver) of the 1,000,000 x 500 FP64 problem A = (G/sqrt(m)) diag(sigma) V^T,
sigma log-spaced 1..1e-10, b = A x + 1e-4 g, d = 12n, zeta = 8, with A and b
resident in HBM.  A (4 GB) is larger than the 129 MB L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own replica of the problem on its own GPU ("replicas only": the solve has no
cross-GPU exchange); only the step timer is reduced (max over ranks).

--impl reference times the CPU oracle (oracle/, plain FP64 loops and numpy
BLAS) on the host cores, on a bounded row sample of the same problem, scaled
to the full problem's solves/s.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FOSSILS solves/s & HBM GB/s at BE≤1e-13 vs plain GPU; served p50/p99 latency"
UNIT = "solves/s"
M, N, KAPPA, NOISE, SEED = 1_000_000, 500, 1e10, 1e-4, 5
SKETCH_SEED = 9
WORKLOAD = "fossils_fp64_m1000000_n500_kappa1e10_d6000_zeta8"
REF_SAMPLE_ROWS = 100_000      # oracle sample per reference step
CPU_BASELINE_ROWS = 250_000    # oracle sample for the cpu_baseline object


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tier", action="store_true",
                    help="skip the tier / many-RHS / served comparisons")
    ap.add_argument("--profile-case", default="", choices=["", "tier", "multi"],
                    help="run small solves of one path for ncu captures (no bench line)")
    ap.add_argument("--rows", type=int, default=0,
                    help="override m (small cases for ncu captures; not a bench line)")
    ap.add_argument("--cols", type=int, default=0,
                    help="override n (small cases for ncu captures; not a bench line)")
    args = ap.parse_args()
    global M, N, WORKLOAD
    if args.rows:
        M = args.rows
    if args.cols:
        N = args.cols
    if args.rows or args.cols:
        WORKLOAD = "fossils_fp64_m%d_n%d_kappa1e10_d%d_zeta8" % (M, N, 12 * N)
    return args


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def config(extra=None):
    c = {"workload": WORKLOAD, "m": M, "n": N, "d": 12 * N, "zeta": 8, "kappa": KAPPA,
         "method": "fossils", "refinement_steps": 2,
         "l2": "A is %.1f GB, larger than L2: no flush needed" % (8.0 * M * N / 1e9),
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


def make_problem(rows=None):
    from lsq_problems import problem_gaussian
    return problem_gaussian(rows or M, N, KAPPA, NOISE, seed=SEED)


# --------------------------------------------------------------------------
# oracle (CPU) timing: the cpu_baseline object and the reference arm
# --------------------------------------------------------------------------

def oracle_time(P, rows, reps=1):
    """Seconds per oracle FOSSILS solve on the first `rows` rows of P."""
    import oracle
    A = P["A"][:rows]
    b = P["b"][:rows]
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.fossils(A, b, seed=SKETCH_SEED)
        ts.append(time.perf_counter() - t0)
    return ts


def cpu_baseline_obj(P, rows):
    ts = oracle_time(P, rows, reps=1)
    per_solve_full = ts[0] * (M / rows)
    return {"value": 1.0 / per_solve_full, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "oracle FOSSILS (numpy BLAS + plain C, FP64) on the first %d of %d rows "
                      "of the same A, b; %.2f s, time scaled by m/rows (passes are O(mn))"
                      % (rows, M, ts[0])}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    P = make_problem(REF_SAMPLE_ROWS)
    oracle_time(P, REF_SAMPLE_ROWS, reps=max(0, args.warmup))
    ts = oracle_time(P, REF_SAMPLE_ROWS, reps=args.steps)
    per_full = statistics.mean(ts) * (M / REF_SAMPLE_ROWS)
    value = 1.0 / per_full
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_full * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"sample_rows": REF_SAMPLE_ROWS}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "each step: oracle FOSSILS on %d of %d rows, time "
                                       "scaled by m/rows" % (REF_SAMPLE_ROWS, M)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpus):
        self.gpus = set(gpus)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or not f[0].isdigit() or int(f[0]) not in self.gpus:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_per_launch():
    """dram read+write bytes per launch of the inner pass from the committed
    ncu summary, or None when the kernel source changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "atax_df_kernel_traffic.txt")
    src = os.path.join(ROOT, "paper_2406_03468_gb300", "csrc", "k_pass.cu")
    try:
        rec = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("k_pass_sha256") != h:
            return None
        return float(rec["bytes_per_launch_full"])
    except (OSError, ValueError, KeyError):
        return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def tier_compare(lsq, torch, dev, steps):
    """Config 5: 1e6 x 1000, A built as for the Fig. 1 problems at kappa = 1e4,
    solved by FOSSILS on the all-FP64 path and on the FP32-inner tier (AUTO),
    and the automatic FP64 fallback at kappa = 1e10."""
    from lsq_problems import problem_svd_torch
    m, n = 1_000_000, 1000
    out = {"workload": "fossils_m1000000_n1000_kappa1e4_d12000_zeta8", "steps": steps}
    P = problem_svd_torch(m, n, 1e4, 1e-4, seed=31, device=dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    for name, prec in (("fp64", lsq.LSQ_PREC_FP64), ("auto", lsq.LSQ_PREC_AUTO)):
        plan = lsq.Plan(m, n, seed=7, precision=prec, timing=1)
        lsq.lsq_solve_fossils(plan.handle, P["A"], P["b"], x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = []
        for _ in range(steps):
            st, inf = lsq.lsq_solve_fossils(plan.handle, P["A"], P["b"], x)
            infos.append(inf.as_dict())
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        last = infos[-1]
        out[name] = {"solves_per_s": 1.0 / dt, "ms_per_solve": dt * 1e3, "path": last["path"],
                     "refine_steps": last["refine_steps"], "iters": last["iters"],
                     "bytes_a_gb": last["bytes_a"] / 1e9,
                     "phase_ms": {"sketch": last["ms_sketch"], "qr": last["ms_qr"],
                                  "refine": last["ms_refine"]},
                     "inner_pass_ms": (last["ms_inner_pass"] / max(1, last["n_inner_pass"]))}
        plan.close()
    del P
    torch.cuda.empty_cache()
    P = problem_svd_torch(m, n, 1e10, 1e-4, seed=32, device=dev)
    plan = lsq.Plan(m, n, seed=7, precision=lsq.LSQ_PREC_AUTO)
    st, inf = lsq.lsq_solve_fossils(plan.handle, P["A"], P["b"], x)
    out["auto_kappa1e10_path"] = inf.as_dict()["path"]
    out["auto_kappa1e10_condest"] = inf.as_dict()["condest"]
    plan.close()
    del P
    torch.cuda.empty_cache()
    return out


def multi_compare(lsq, torch, dev, steps):
    """Config 4: 2e6 x 200, k = 64 right-hand sides sharing one sketch and QR.
    The default plan runs the inner pass for all k vectors as one batched
    double-float launch on the hi / lo planes (HBM roofline over k 8mn
    bytes per pass); a strict-FP64 plan (inner_fp64_fma = 1) runs it as the
    FP64 tensor-core (DMMA) contraction (tensor roofline); both against the
    single-RHS path solving one column."""
    from lsq_problems import problem_multi_rhs_torch
    m, n, k = 2_000_000, 200, 64
    P = problem_multi_rhs_torch(m, n, k, 1e8, 1e-5, seed=41, device=dev)
    X = torch.empty((n, k), dtype=torch.float64, device=dev)
    pk, kind = peaks()

    def run(opts, nsteps):
        plan = lsq.Plan(m, n, seed=6, nrhs=k, timing=1, **opts)
        lsq.lsq_solve_fossils_multi(plan.handle, P["A"], P["B"], k, X)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = []
        for _ in range(nsteps):
            st, inf = lsq.lsq_solve_fossils_multi(plan.handle, P["A"], P["B"], k, X)
            infos.append(inf.as_dict())
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / nsteps
        plan.close()
        last = infos[-1]
        return dt, last, last["ms_inner_pass"] / max(1, last["n_inner_pass"])

    dt, last, pass_ms = run({}, steps)
    hbm_bytes = 8.0 * m * n * k
    achieved = hbm_bytes / (pass_ms / 1e3) / 1e9
    dt64, last64, pass64_ms = run({"inner_fp64_fma": 1}, 1)
    flops = 4.0 * m * n * k
    # FP64 tensor peak: the measured BF16 peak times the nominal FP64 / BF16 ratio (1.25 / 2250)
    fp64_peak = pk.get("bf16_tflops", 1900.0) * 1.25 / 2250.0
    achieved64 = flops / (pass64_ms / 1e3) / 1e12
    b0 = P["B"][:, 0].contiguous()
    x1 = torch.empty(n, dtype=torch.float64, device=dev)
    plan1 = lsq.Plan(m, n, seed=6)
    lsq.lsq_solve_fossils(plan1.handle, P["A"], b0, x1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        lsq.lsq_solve_fossils(plan1.handle, P["A"], b0, x1)
    torch.cuda.synchronize()
    dt1 = (time.perf_counter() - t0) / steps
    plan1.close()
    del P
    torch.cuda.empty_cache()
    return {"workload": "fossils_multi_m2000000_n200_k64_kappa1e8_d2400_zeta8",
            "solves_per_s": 1.0 / dt, "rhs_solves_per_s": k / dt, "ms_per_solve": dt * 1e3,
            "inner_kernel": last["inner_kernel"],
            "iters": last["iters"], "phase_ms": {"sketch": last["ms_sketch"], "qr": last["ms_qr"],
                                                 "refine": last["ms_refine"]},
            "single_rhs_solves_per_s": 1.0 / dt1,
            "inner_pass": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                           "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "ms": pass_ms,
                           "bytes": hbm_bytes, "peak_kind": kind},
            "fp64_dmma": {"rhs_solves_per_s": k / dt64, "inner_kernel": last64["inner_kernel"],
                          "pass": {"bound": "tensor", "achieved": achieved64, "peak": fp64_peak,
                                   "unit": "TFLOP/s", "frac": achieved64 / fp64_peak,
                                   "ms": pass64_ms, "flops": flops,
                                   "peak_note": "measured bf16 x nominal fp64/bf16 (1.25/2250), "
                                   + kind}}}


def serve_compare(lsq, torch, dev, count=512, slots=8):
    """Config 3: a stream of `count` independent problems (m log-uniform in
    [2e4, 4e5], n in {32, 64, 128, 256}, kappa log-uniform in [1e2, 1e12],
    b = A x + 1e-6 g), solved one at a time on one plan (plain), then through
    the request server: closed loop (all submitted at once) for the capacity
    C, and Poisson arrivals at 0.5 C and 0.9 C for p50 / p99 latency."""
    import math
    import numpy as np
    from lsq_problems import problem_svd_torch
    rng = np.random.default_rng(2026)
    probs = []
    for i in range(count):
        m = int(math.exp(rng.uniform(math.log(2e4), math.log(4e5))))
        n = int(rng.choice([32, 64, 128, 256]))
        kappa = 10.0 ** rng.uniform(2, 12)
        P = problem_svd_torch(m, n, kappa, 1e-6, seed=5000 + i, device=dev)
        probs.append((m, n, P["A"], P["b"]))
    torch.cuda.synchronize()
    # plain: one plan of the largest size, re-targeted per problem (no
    # allocation), one solve at a time on one stream (first 128 problems)
    nplain = min(128, count)
    x = torch.empty(256, dtype=torch.float64, device=dev)
    plan = lsq.Plan(400000, 256, seed=1)
    for (m, n, A, b) in probs[:4]:
        lsq.lsq_plan_configure(plan.handle, lsq.lsq_options_default(m=m, n=n, seed=1))
        lsq.lsq_solve_fossils(plan.handle, A, b, x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (m, n, A, b) in probs[:nplain]:
        lsq.lsq_plan_configure(plan.handle, lsq.lsq_options_default(m=m, n=n, seed=1))
        lsq.lsq_solve_fossils(plan.handle, A, b, x)
    torch.cuda.synchronize()
    plain_rate = nplain / (time.perf_counter() - t0)
    plan.close()
    foot = [8 * (m * n + m + n) + 768 for (m, n, _, _) in probs]
    arena = int(min(sum(foot), 48 << 30))
    srv = lsq.lsq_server_create(arena, slots, 400000, 256)

    def run(gaps):
        xb = np.empty(256)
        t_start = time.perf_counter()
        due = t_start + np.cumsum(gaps)
        pending, lat, i = {}, [], 0
        while i < count or pending:
            now = time.perf_counter()
            while i < count and due[i] <= now:
                m, n, A, b = probs[i]
                o = lsq.lsq_options_default(m=m, n=n, seed=1)
                pending[lsq.lsq_submit(srv, o, 0, A, b, 1)] = i
                i += 1
            for t in list(pending):
                st, info, l = lsq.lsq_poll(srv, t, xb)
                if st != lsq.LSQ_PENDING:
                    lat.append(l)
                    del pending[t]
            if not pending and i < count:
                time.sleep(max(0.0, min(0.001, due[i] - time.perf_counter())))
        el = time.perf_counter() - t_start
        return count / el, float(np.percentile(lat, 50)), float(np.percentile(lat, 99))

    run(np.zeros(count))  # warm-up
    cap, _, _ = run(np.zeros(count))
    out = {"workload": "served_stream_512_m2e4-4e5_n32-256_kappa1e2-1e12", "slots": slots,
           "arena_gb": arena / 1e9, "plain_solves_per_s": plain_rate,
           "capacity_solves_per_s": cap}
    for frac in (0.5, 0.9):
        rate = frac * cap
        gaps = np.random.default_rng(7).exponential(1.0 / rate, count)
        thr, p50, p99 = run(gaps)
        out["rate_%.1fC" % frac] = {"offered_per_s": rate, "solves_per_s": thr,
                                    "p50_ms": p50 * 1e3, "p99_ms": p99 * 1e3}
    out["stats"] = lsq.lsq_server_stats(srv)
    lsq.lsq_server_destroy(srv)
    del probs
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import paper_2406_03468_gb300 as lsq

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    P = make_problem()
    dev = torch.device("cuda", local)
    A = torch.from_numpy(P["A"]).to(dev)
    b = torch.from_numpy(P["b"]).to(dev)
    x = torch.empty(N, dtype=torch.float64, device=dev)
    plan = lsq.Plan(M, N, seed=SKETCH_SEED, timing=1)
    h = plan.handle

    for _ in range(args.warmup):
        lsq.lsq_solve_fossils(h, A, b, x)
    torch.cuda.synchronize()

    sampler = ClockSampler(range(args.gpus)) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    infos = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        st, inf = lsq.lsq_solve_fossils(h, A, b, x)
        infos.append(inf.as_dict())
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = args.steps * world / (ms / 1e3)

    # roofline of the dominant kernel: the fused A^T(A z) pass
    n_in = sum(i["n_inner_pass"] for i in infos)
    ms_in = sum(i["ms_inner_pass"] for i in infos)
    pk, pk_kind = peaks()
    bytes_pass = 8.0 * M * N
    avg_s = (ms_in / n_in) / 1e3
    achieved = bytes_pass / avg_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic_per_launch(),
            "kernel": {0: "atax_kernel", 1: "atax_eft_kernel", 2: "atax32_kernel",
                       3: "atax_df_kernel"}[infos[-1]["inner_kernel"]]
                      + " (fused A^T(A z) inner pass)", "launches_timed": n_in,
            "avg_launch_ms": avg_s * 1e3, "peak_kind": pk_kind}
    passes = statistics.mean(i["passes"] for i in infos)
    hbm_solve = passes * bytes_pass / (ms / args.steps / 1e3) / 1e9

    # SPIR on the same plan (context)
    xs = torch.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    spir_infos = []
    for _ in range(max(1, args.steps // 2)):
        st, inf = lsq.lsq_solve_spir(h, A, b, xs)
        spir_infos.append(inf.as_dict())
    torch.cuda.synchronize()
    spir_rate = len(spir_infos) / (time.perf_counter() - t0)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(P["A"]).pin_memory()
        hb = torch.from_numpy(P["b"]).pin_memory()
        hx = torch.empty(N, dtype=torch.float64).pin_memory()
        lsq.lsq_solve_host(h, 0, hA, hb, hx)
        torch.cuda.synchronize()
        # the host link's own rate on these buffers (context for the e2e number)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record()
        A.copy_(hA, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        link_gbs = 8 * M * N / (c0.elapsed_time(c1) * 1e-3) / 1e9
        k2 = max(1, args.steps // 2)
        host_infos = []
        t0 = time.perf_counter()
        for _ in range(k2):
            _, hinf = lsq.lsq_solve_host(h, 0, hA, hb, hx)
            host_infos.append(hinf.as_dict())
        dt = time.perf_counter() - t0
        rate = k2 * world / dt
        if dist:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            rate = k2 * world / float(t.item())
        e2e = {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 8 * M * N + 8 * M,
               "d2h_bytes_per_step": 8 * N, "h2d_link_gbs": link_gbs,
               "sketch_ms_incl_copy": statistics.median(i["ms_sketch"] for i in host_infos),
               "device_ms_per_solve": statistics.median(i["ms_total"] for i in host_infos)}

    tier = None
    multi = None
    served = None
    if not args.no_tier and not args.rows and not args.cols:
        del A
        torch.cuda.empty_cache()
        tier = tier_compare(lsq, torch, dev, max(2, args.steps // 3))
        multi = multi_compare(lsq, torch, dev, 2)
        served = serve_compare(lsq, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_obj(P, CPU_BASELINE_ROWS)

    if rank == 0:
        last = infos[-1]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": config({"hbm_gbs_per_solve": hbm_solve,
                                  "passes_per_solve": passes,
                                  "iters": last["iters"], "condest": last["condest"],
                                  "phase_ms": {"sketch": last["ms_sketch"], "qr": last["ms_qr"],
                                               "refine": last["ms_refine"]},
                                  "sketch_pass_ms": last["ms_sketch_pass"],
                                  "spir_solves_per_s": spir_rate,
                                  "spir_iters": spir_infos[-1]["iters"],
                                  "fp32_tier_1e6x1000": tier,
                                  "multi_rhs_2e6x200_k64": multi,
                                  "served_stream": served}),
                "clocks": clocks, "e2e": e2e,
                "gpu_launches": int(sum(i["launches"] for i in infos)),
                "roofline": roof, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """Small cases for ncu captures: `tier` = FP32-inner FOSSILS on 2e5 x 1000
    (kappa 1e4), `multi` = 64 right-hand sides on 2e5 x 200 (kappa 1e8)."""
    import numpy as np
    import torch
    import paper_2406_03468_gb300 as lsq
    from lsq_problems import problem_gaussian
    dev = torch.device("cuda", 0)
    if args.profile_case == "tier":
        P = problem_gaussian(200000, 1000, 1e4, 1e-4, seed=31)
        A, b = torch.from_numpy(P["A"]).to(dev), torch.from_numpy(P["b"]).to(dev)
        plan = lsq.Plan(200000, 1000, seed=7, precision=lsq.LSQ_PREC_AUTO)
        x = torch.empty(1000, dtype=torch.float64, device=dev)
        for _ in range(max(1, args.steps)):
            st, info = lsq.lsq_solve_fossils(plan.handle, A, b, x)
    else:
        P = problem_gaussian(200000, 200, 1e8, 1e-5, seed=41)
        A = torch.from_numpy(P["A"]).to(dev)
        Xt = torch.from_numpy(np.random.default_rng(3).standard_normal((200, 64))).to(dev)
        B = (A @ Xt).contiguous()
        plan = lsq.Plan(200000, 200, seed=6, nrhs=64)
        X = torch.empty((200, 64), dtype=torch.float64, device=dev)
        for _ in range(max(1, args.steps)):
            st, info = lsq.lsq_solve_fossils_multi(plan.handle, A, B, 64, X)
    torch.cuda.synchronize()
    plan.close()
    print(json.dumps({"profile_case": args.profile_case, "info": info.as_dict()}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
