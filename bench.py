"""Throughput of the multi-chain HMC sampler on one GB300 (or N, one process
per GPU, each sampling its own replica of the posterior: chains are
independent, so ranks share nothing on the data path; weak scaling).

A step is one full sample_chain call (bootstrap, burn-in transitions with
dual-averaging step-size adaptation, kept transitions with every kept state
written to HBM) of the correlated-Gaussian workload: D = 256,
P = A A^T / D + 0.1 I, 4096 chains from N(0, 1), 16 leapfrog steps,
adaptation to accept 0.65, 1000 burn-in + 2000 kept transitions.
Metric: leapfrog gradient evaluations per second (one chain's grad log p is
one evaluation; bootstrap adds one per chain), plus min-ESS/s of the kept
draws.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload corr_gauss|logreg|funnel|std_normal] [--plain]

--impl reference times the float64 oracle (a deliberately plain CPU
program, the only reference this method has) on the host cores, on a bounded
sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# nominal dense tensor ratio tf32 : bf16 (1.1 : 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from the committed
# ncu capture of the same kernel on the same workload (profiles/); keyed by
# (kernel, target, chains, dim, leapfrog steps).  Absent -> traffic is null.
PROFILED_TRAFFIC = {}

# NUTS (Section 2.3): default maximum tree depth
NUTS_MAX_DEPTH = 10
NUTS_LABEL = " NUTS max_depth=10"

L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="corr_gauss",
                    choices=["corr_gauss", "logreg", "funnel", "std_normal", "uneven_batch", "serve"])
    ap.add_argument("--plain", action="store_true", help="one launch per op per leapfrog step")
    ap.add_argument("--proposal", default="leapfrog", choices=["leapfrog", "random_walk", "nuts"],
                    help="inner kernel of the Metropolis-Hastings composition (random_walk runs "
                         "the plain path; one target evaluation per transition) or NUTS "
                         "(funnel / std_normal; maximum tree depth 10)")
    ap.add_argument("--max-transitions-per-launch", type=int, default=0,
                    help="dense Gaussian: cap on transitions per kernel launch (0: whole chain; "
                         "1 for profilers that cannot replay cooperative cluster launches)")
    ap.add_argument("--streaming", type=int, default=0, metavar="BATCH",
                    help="streaming driver: running moments and batch-means ESS (batches of BATCH "
                         "kept draws) on the device instead of the kept-sample trace")
    ap.add_argument("--replicas", type=int, default=1, metavar="K",
                    help="replica exchange (Section 2.2): the chains form chains/K sets of K "
                         "tempered replicas, inverse temperatures 4^(-k/(K-1)), fixed step size")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain-baseline", action="store_true",
                    help="skip the comparison run of the plain one-launch-per-operation path "
                         "(same workload, same GPU) that fills vs_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-scale", type=float, default=0.04,
                    help="uneven_batch: fraction of the 500 + 1000 transitions run per posterior")
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-duration", type=float, default=10.0)
    ap.add_argument("--serve-scale", type=float, default=0.1,
                    help="serve: scale of chains, samples and data rows of every request")
    ap.add_argument("--serve-workers", type=int, default=4,
                    help="serve: admission threads (context creation, graph capture, teardown)")
    ap.add_argument("--serve-max-wall", type=float, default=0.0,
                    help="serve: stop after this many seconds (0: 6 x the duration, at least 60)")
    ap.add_argument("--small", action="store_true",
                    help="20 burn-in + 20 kept transitions (profiling runs)")
    ap.add_argument("--logreg-shape", default=None, metavar="D,N,C",
                    help="logreg: dim, data rows and chains instead of 128, 20000, 2048 (e.g. one "
                         "of the uneven batch's shapes, for profiling)")
    return ap.parse_args()


def make_problem(name, logreg_shape=None):
    from paper_2002_01184_gb300 import workloads
    if name == "corr_gauss":
        return workloads.corr_gauss(), "corr_gauss D=256 P=AA^T/D+0.1I C=4096 L=16 DA(0.65) B=1000 K=2000"
    if name == "logreg" and logreg_shape:
        D, N, C = (int(v) for v in logreg_shape.split(","))
        return (workloads.logreg(n_data=N, dim=D, num_chains=C),
                f"logreg N={N} D={D} C={C} L=10 DA(0.8) B=500 K=1000")
    if name == "logreg":
        return workloads.logreg(), "logreg N=20000 D=128 C=2048 L=10 DA(0.8) B=500 K=1000"
    if name == "funnel":
        p = workloads.funnel(dim=100, num_chains=4096)
        return p, "funnel d=100 C=4096 L=10 DA(0.8) B=500 K=1000"
    return workloads.std_normal(), "std_normal D=1 C=100 L=3 eps=1.5 B=300 K=100"


class ReplicaSet:
    """A replica-exchange context over the workload's chains: chains / K sets
    of K replicas (rows c K + k), inverse temperatures 4^(-k / (K - 1)); the
    step size is fixed at the workload's adapted value."""

    def __init__(self, p, K, impl, stream, proposal):
        from paper_2002_01184_gb300 import hmc
        import torch
        if p.num_chains % K:
            raise SystemExit(f"--replicas {K} must divide the {p.num_chains} chains")
        self.betas = [4.0 ** (-k / (K - 1)) for k in range(K)]
        self.P = None if p.P is None else torch.as_tensor(p.P).cuda().contiguous()
        self.X = None if p.X is None else torch.as_tensor(p.X).cuda().contiguous()
        self.y = None if p.y is None else torch.as_tensor(p.y).cuda().contiguous()
        if p.kind == "corr_gauss":
            p.step_size = 0.445            # the adapted step size of the untempered chains
        p.adapt = False
        target = hmc.make_target(p.kind, p.dim, self.P, self.X, self.y)
        cfg = hmc.make_config(p.num_leapfrog, p.step_size, p.seed, False, p.target_accept, 0, impl,
                              proposal=proposal)
        self.ctx = hmc.hmc_remc_create(target, p.num_chains // K, self.betas, cfg, stream)

    def close(self):
        from paper_2002_01184_gb300 import hmc
        if self.ctx:
            hmc.hmc_destroy(self.ctx)
            self.ctx = None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK), "fallback"


def nuts_leaf_latency(p, eps, transitions=64):
    """Seconds per leaf of one NUTS chain alone (one warp on the GPU) on the
    workload's target and dim at step size eps: `transitions` fixed-step
    transitions in one launch, timed on the device."""
    import copy
    import torch
    from paper_2002_01184_gb300 import hmc
    from paper_2002_01184_gb300.sampler import Sampler
    q = copy.copy(p)
    q.num_chains, q.x0 = 1, p.x0[:1].copy()
    s = Sampler(q, adapt=False, step_size=eps, proposal=hmc.HMC_PROPOSAL_NUTS)
    x = torch.as_tensor(q.x0).cuda()
    s.sample_chain(x, 0, 4)                    # warm-up
    l0 = hmc.hmc_nuts_leapfrog_count(s.ctx)
    hmc.hmc_profile_dominant_kernel(s.ctx, 1)
    s.sample_chain(x, 0, transitions)
    torch.cuda.synchronize()
    pr = hmc.hmc_profile_read(s.ctx)
    leaves = hmc.hmc_nuts_leapfrog_count(s.ctx) - l0
    s.close()
    return pr["avg_ms"] * pr["samples"] / 1000.0 / max(leaves, 1)


def grad_flops_per_eval(p):
    """Algorithmic flops of one chain's gradient (the dense products)."""
    if p.kind == "corr_gauss":
        return 2.0 * p.dim * p.dim
    if p.kind == "logreg":
        return 4.0 * p.n_data * p.dim
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(ms, units, device=None):
    """Whole-job throughput of weakly scaled replicas: the slowest rank's time
    and the units summed over ranks (each rank runs its own replica)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The float64 oracle on the host cores, on a bounded sample."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    p, wl = make_problem(args.workload, args.logreg_shape)
    if args.proposal == "nuts":
        p.num_leapfrog = NUTS_MAX_DEPTH
        wl += NUTS_LABEL
    res = cpu_oracle_rate(p, args.cpu_seconds, args.proposal)
    line = {"impl": "reference", "metric": "leapfrog grad-evals/s", "value": res["value"],
            "unit": "grad-evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_transition"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl, "sample": res["sample"]},
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "grad-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_oracle_rate(p, seconds, proposal="leapfrog"):
    """Time the oracle's transitions on a prefix of the workload until about
    `seconds` of CPU work; rate = target evaluations (chains x L per HMC
    transition, one per random-walk transition, the leaves built by NUTS) /
    wall time."""
    import numpy as np
    from oracle import hmc as ohmc, mh as omh, nuts as onuts, targets as otargets
    tgt = otargets.make(p.kind, **p.data())
    C = p.num_chains
    if proposal == "nuts":
        C = min(C, 64)                 # the oracle builds each chain's tree in a Python loop
    x = p.x0[:C].astype(np.float64)
    lp, g = ohmc.bootstrap(x, tgt)
    eps = p.step_size
    t0 = time.perf_counter()
    n = evals = 0
    while True:
        if proposal == "nuts":
            r = onuts.one_step(x, lp, g, eps, p.num_leapfrog, p.seed, n, tgt)
            evals += int(r["leaves"].sum())
        elif proposal == "random_walk":
            r = omh.rw_one_step(x, lp, g, eps, p.seed, n, tgt)
            evals += C
        else:
            r = ohmc.one_step(x, lp, g, eps, p.num_leapfrog, p.seed, n, tgt)
            evals += C * p.num_leapfrog
        x, lp, g = r["x"], r["lp"], r["g"]
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= p.num_burnin + p.num_results:
            break
    kind = {"nuts": "NUTS", "random_walk": "random-walk"}.get(proposal, "HMC")
    return {"value": evals / el, "unit": "grad-evals/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {n} {kind} transitions of the workload ({C} of {p.num_chains} chains, "
                      f"fixed step size), numpy float64 with BLAS on all host cores",
            "ms_per_transition": 1000.0 * el / n}


def plain_baseline(p, stream, x, x0, samples, eps, acc, value, min_ess_per_s):
    """One untimed warm-up and one timed sample_chain of the plain path
    (HMC_IMPL_PLAIN) on the same workload, reusing the bench's buffers after
    its own figures are taken; returns the vs_baseline object (per GPU)."""
    import torch
    from paper_2002_01184_gb300 import diagnostics, hmc
    from paper_2002_01184_gb300.sampler import Sampler
    C, K, B = p.num_chains, p.num_results, p.num_burnin
    s = Sampler(p, impl=hmc.HMC_IMPL_PLAIN, stream=stream)
    try:
        def run():
            x.copy_(x0)
            hmc.hmc_sample_chain(s.ctx, x, B, K, samples, eps, acc)
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        evals = C * p.num_leapfrog * (B + K) + C
        plain_value = evals / (ms / 1000.0)
        plain_ess = float(diagnostics.ess(samples).min())
        plain_ess_s = plain_ess / (ms / 1000.0)
        return {"baseline": "plain HMC on the same GPU: one kernel launch per operation per "
                            "leapfrog step (SIMT float32 products), same workload, seed, L and "
                            "dual averaging; 1 warm-up + 1 timed step",
                "value": plain_value, "unit": "grad-evals/s", "ms_per_step": ms,
                "min_ess": plain_ess, "min_ess_per_s": plain_ess_s,
                "accept_rate": float(acc.float().mean().item()) if K else None,
                "ratio": value / plain_value,
                "min_ess_per_s_ratio": (min_ess_per_s / plain_ess_s) if plain_ess_s else None}
    finally:
        s.close()


def run_uneven_batch(args):
    """64 logistic regressions + 16 funnels of uneven size in one grouped
    launch per transition (ours) or one posterior after another through the
    plain one-launch-per-operation path (--plain)."""
    import numpy as np
    import torch
    from paper_2002_01184_gb300 import build as libbuild
    libbuild.build()
    from paper_2002_01184_gb300 import diagnostics, hmc, workloads
    from paper_2002_01184_gb300.sampler import Sampler
    torch.cuda.set_device(0)
    B = max(1, int(round(500 * args.batch_scale)))
    K = max(2, int(round(1000 * args.batch_scale)))
    probs = workloads.uneven_batch(num_burnin=B, num_results=K)
    dev = lambda a: None if a is None else torch.as_tensor(a).cuda().contiguous()
    data = [(dev(p.X), dev(p.y)) for p in probs]
    xs0 = [dev(p.x0) for p in probs]
    xs = [torch.empty_like(x) for x in xs0]
    samples = [torch.empty((K, p.num_chains, p.dim), device="cuda") for p in probs]
    evals = sum(p.num_chains * p.num_leapfrog * (B + K) + p.num_chains for p in probs)
    stream = torch.cuda.current_stream()
    if args.plain:
        samplers = [Sampler(p, impl=hmc.HMC_IMPL_PLAIN, stream=stream) for p in probs]

        def step():
            for s_, x, x0, smp, p in zip(samplers, xs, xs0, samples, probs):
                x.copy_(x0)
                hmc.hmc_sample_chain(s_.ctx, x, B, K, smp, None, None)
    else:
        targets = [hmc.make_target(p.kind, p.dim, None, X, y) for p, (X, y) in zip(probs, data)]
        configs = [hmc.make_config(p.num_leapfrog, p.step_size, p.seed, p.adapt, p.target_accept, B)
                   for p in probs]
        t_tune = time.perf_counter()
        batch = hmc.hmc_batch_create_autotuned(targets, [p.num_chains for p in probs], configs, stream)
        t_tune = time.perf_counter() - t_tune
        paths = [hmc.hmc_batch_member_path(batch, i)[0] for i in range(len(probs))]
        tuner = {"create_s": t_tune,
                 "grouped": sum(1 for q in paths if q == 0),
                 "tensor_core_contexts": sum(1 for q in paths if q == 1),
                 "other_contexts": sum(1 for q in paths if q == 2)}

        def step():
            for x, x0 in zip(xs, xs0):
                x.copy_(x0)
            hmc.hmc_batch_sample_chain(batch, xs, [B] * len(probs), [K] * len(probs), samples)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    if args.plain:
        tuner = None
    launches0 = hmc.hmc_kernel_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    t_enq = time.perf_counter() - t_host
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    launches = hmc.hmc_kernel_launch_count() - launches0
    ess = min(float(diagnostics.ess(smp, max_dims=16).min()) for smp in samples)
    # the GEMM share: the logistic regressions' algorithmic flops (4 N D per
    # gradient evaluation) over the whole step's time, against the 3xTF32
    # peak -- a lower bound on the products' own fraction, since the step's
    # time also holds the funnels and the leapfrog updates
    pk, src = peaks()
    gemm = sum(4.0 * p.n_data * p.dim * (p.num_chains * p.num_leapfrog * (B + K) + p.num_chains)
               for p in probs if p.kind == "logreg")
    peak = pk["bf16_tflops"] * TF32_PER_BF16 / 3.0
    achieved = gemm / (ms / 1000.0) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "scope": "the logistic regressions' algorithmic flops over the whole step",
            "peak_source": f"{src} bf16 {pk['bf16_tflops']:.0f} TFLOP/s x (1.1/2.25 nominal tf32:bf16) / 3"}
    line = {"metric": "leapfrog grad-evals/s", "value": evals / (ms / 1000.0), "unit": "grad-evals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"uneven batch: 64 logreg (D,N,C log-uniform [8,512],[500,20000],"
                                   f"[64,4096]) + 16 funnels (d in [10,200]), L=10, DA(0.8), "
                                   f"B={B} K={K} (fraction {args.batch_scale} of 500+1000)",
                       "impl": "plain, one posterior after another" if args.plain
                       else "autotuned: grouped members in one persistent launch, tensor-core members on their own streams",
                       "posteriors": len(probs), "autotuner": tuner},
            "min_ess_per_s": ess / (ms / 1000.0), "min_ess": ess,
            "host_enqueue_ms_per_step": 1000.0 * t_enq / args.steps,
            "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "cpu_baseline": None,
            "e2e": None}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson request stream through the continuous-batching server."""
    import torch
    from paper_2002_01184_gb300 import build as libbuild
    libbuild.build()
    from paper_2002_01184_gb300 import hmc, serve, workloads
    torch.cuda.set_device(0)
    reqs = workloads.serve_stream(rate=args.serve_rate, duration=args.serve_duration,
                                  size_scale=args.serve_scale)
    # warm-up: a few requests through a throwaway server
    serve.Server(hbm_budget_bytes=150 * 2 ** 30, slots=16).run(reqs[:4], time_scale=1e9)
    launches0 = hmc.hmc_kernel_launch_count()
    clocks = ClockSampler(0)
    clocks.start()
    server = serve.Server(hbm_budget_bytes=150 * 2 ** 30, slots=32, workers=args.serve_workers)
    max_wall = args.serve_max_wall or max(60.0, 6 * args.serve_duration)
    jobs = server.run(reqs, max_wall=max_wall)
    clk = clocks.stop()
    summ = serve.summarize(jobs, server.wall)
    summ["host_s"] = dict(server.host_s)
    summ["backlog_at_end"] = server.backlog
    summ["stopped_at_max_wall"] = server.backlog > 0
    line = {"metric": "leapfrog grad-evals/s", "value": summ["grad_evals_per_s"],
            "unit": "grad-evals/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1000.0 * server.wall, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"served stream: Poisson {args.serve_rate}/s for "
                                   f"{args.serve_duration} s, requests from corr_gauss / logreg / "
                                   f"uneven families, chains/samples/data rows scaled by "
                                   f"{args.serve_scale}, HBM budget 150 GB, 32 slots, "
                                   f"{args.serve_workers} admission threads, run stopped after "
                                   f"{max_wall:.0f} s of wall time at the latest",
                       "impl": "continuous batching (slot streams, admission by HBM budget)"},
            "serve": summ, "min_ess_per_s": summ["ess_per_s"],
            "gpu_launches": int(hmc.hmc_kernel_launch_count() - launches0), "clocks": clk,
            "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "uneven_batch":
        run_uneven_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    import numpy as np
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2002_01184_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2002_01184_gb300 import diagnostics, hmc
    from paper_2002_01184_gb300.sampler import Sampler

    p, wl = make_problem(args.workload, args.logreg_shape)
    if args.small:
        p.num_burnin, p.num_results = 20, 20
        wl += " (profiling run: B=20 K=20)"
    p.seed = p.seed + 1000 * rank          # each rank samples its own replica
    impl = hmc.HMC_IMPL_PLAIN if args.plain else hmc.HMC_IMPL_FUSED
    stream = torch.cuda.current_stream()
    proposal = {"random_walk": hmc.HMC_PROPOSAL_RANDOM_WALK,
                "nuts": hmc.HMC_PROPOSAL_NUTS}.get(args.proposal, hmc.HMC_PROPOSAL_LEAPFROG)
    if proposal == hmc.HMC_PROPOSAL_RANDOM_WALK:
        p.num_leapfrog = 1                 # one target evaluation per transition
        wl += " (random-walk Metropolis-Hastings)"
    elif proposal == hmc.HMC_PROPOSAL_NUTS:
        p.num_leapfrog = NUTS_MAX_DEPTH    # the context's num_leapfrog is the maximum tree depth
        wl += NUTS_LABEL
    if args.replicas > 1:
        s = ReplicaSet(p, args.replicas, impl, stream, proposal)
        wl += (f" (replica exchange: {p.num_chains // args.replicas} x {args.replicas} replicas, "
               f"betas {', '.join(f'{b:.3f}' for b in s.betas)}, step size {p.step_size} fixed)")
    else:
        s = Sampler(p, impl=impl, stream=stream, max_transitions_per_launch=args.max_transitions_per_launch,
                    proposal=proposal)
    C, D, K, B = p.num_chains, p.dim, p.num_results, p.num_burnin
    x0 = torch.as_tensor(p.x0).cuda()
    x = torch.empty_like(x0)
    streaming = args.streaming > 0
    samples = None if streaming else torch.empty((K, C, D), dtype=torch.float32, device="cuda")
    eps = torch.empty(K, dtype=torch.float32, device="cuda")
    acc = torch.empty((K, C), dtype=torch.uint8, device="cuda")
    if streaming:
        wl += f" (streaming: moments + batch-means ESS, batches of {args.streaming})"
        mean, m2 = torch.empty_like(x0), torch.empty_like(x0)
        ess_d = torch.empty(D, dtype=torch.float32, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        x.copy_(x0)
        if streaming:
            flush.zero_()            # no trace is written: flush L2 explicitly
            hmc.hmc_sample_chain_streaming_ess(s.ctx, x, B, K, args.streaming, mean, m2, ess_d, eps, acc)
        else:
            hmc.hmc_sample_chain(s.ctx, x, B, K, samples, eps, acc)

    hmc.hmc_profile_dominant_kernel(s.ctx, 8)      # before the graph is captured
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evals_per_step = C * p.num_leapfrog * (B + K) + C
    nuts = proposal == hmc.HMC_PROPOSAL_NUTS
    nuts_dense = nuts and p.kind in ("corr_gauss", "logreg")
    if nuts:
        leaves0 = hmc.hmc_nuts_leapfrog_count(s.ctx)
    if nuts_dense:
        iters0 = hmc.hmc_nuts_leaf_iterations(s.ctx)
    clocks = ClockSampler(local)
    clocks.start()
    hmc.hmc_profile_dominant_kernel(s.ctx, 8)
    launches0 = hmc.hmc_kernel_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms_local = e0.elapsed_time(e1)
    launches = hmc.hmc_kernel_launch_count() - launches0
    if nuts:
        # the trees' sizes vary: count the leapfrog steps the timed steps built
        # (identical every step: same start, same seed) and the bootstrap
        evals_per_step = (hmc.hmc_nuts_leapfrog_count(s.ctx) - leaves0) / args.steps + C
    nuts_info = None
    if nuts_dense:
        # lockstep leaves: each loop iteration is one batched gradient (tile
        # products of the chains still building) and one leaf kernel; the
        # launch count above has each transition's loop body once
        iters = (hmc.hmc_nuts_leaf_iterations(s.ctx) - iters0) / args.steps
        per_iter = 2 if p.kind == "corr_gauss" else 3
        launches += int(round((iters - (B + K)) * per_iter * args.steps))
        nuts_info = {"leaf_iterations_per_step": iters, "leapfrog_steps_per_step": evals_per_step - C,
                     "useful_row_fraction": (evals_per_step - C) / (iters * C)}
    try:
        prof = hmc.hmc_profile_read(s.ctx)
    except hmc.HMCError as exc:              # timing support only
        print(f"dominant-kernel timing unavailable: {exc}", file=sys.stderr)
        prof = {"avg_ms": 0.0, "samples": 0, "launches": 0}
    clk = clocks.stop()
    ms, total_evals = reduce_over_ranks(ms_local, evals_per_step * args.steps, device="cuda")
    ms_per_step = ms / args.steps
    value = total_evals / (ms / 1000.0)

    # min-ESS/s of the last step's kept draws over every dimension (not timed)
    ess = ess_d.double().cpu().numpy() if streaming else diagnostics.ess(samples).numpy()
    min_ess = float(ess.min())
    min_ess_per_s = min_ess / (ms_per_step / 1000.0) * world
    final_eps = float(eps[-1].item()) if K else None
    accept_rate = float(acc.float().mean().item()) if K else None

    pk, src = peaks()
    flops = grad_flops_per_eval(p)
    kname, evals_per_launch = hmc.hmc_dominant_kernel_info(s.ctx)
    if nuts:
        # launches of unequal work (one adapting transition each, then the
        # fixed-step-size run): one more, untimed step with every launch
        # timed gives the k_nuts time of a whole step
        hmc.hmc_profile_dominant_kernel(s.ctx, 1)
        crit0 = hmc.hmc_nuts_leaf_iterations(s.ctx)
        step()
        torch.cuda.synchronize()
        crit_per_step = hmc.hmc_nuts_leaf_iterations(s.ctx) - crit0
        pn = hmc.hmc_profile_read(s.ctx)
        prof = {"samples": 0}
        if pn["samples"] and pn["samples"] == pn["launches"]:
            prof = {"avg_ms": pn["avg_ms"] * pn["samples"], "samples": pn["samples"]}
        elif pn["samples"]:
            # more launches than the timer keeps (the last 2048): their mean
            # times the step's launch count
            prof = {"avg_ms": pn["avg_ms"] * pn["launches"], "samples": pn["samples"],
                    "sampled_of": pn["launches"]}
        evals_per_launch = evals_per_step - C              # per step
    roof = None
    if prof["samples"]:
        kernel_s = prof["avg_ms"] / 1000.0
        traffic = PROFILED_TRAFFIC.get((kname, p.kind, C, D, p.num_leapfrog))
        common = {"kernel": kname, "avg_launch_ms": prof["avg_ms"],
                  "timed_launches": prof["samples"], "grad_evals_per_launch": evals_per_launch}
        if nuts:
            common = {"kernel": kname, "kernel_ms_per_step": prof["avg_ms"],
                      "launches_per_step": prof.get("sampled_of", prof["samples"]),
                      "timed_launches": prof["samples"], "leapfrog_steps_per_step": evals_per_launch}
        if flops is not None and hmc.hmc_uses_tensor_cores(s.ctx):
            # 3xTF32: algorithmic flops (2 D^2 per gradient evaluation) against
            # the dense TF32 peak / 3 (three tf32 products per float32 product)
            achieved = flops * evals_per_launch / kernel_s / 1e12
            peak = pk["bf16_tflops"] * TF32_PER_BF16 / 3.0
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "peak_source": f"{src} bf16 {pk['bf16_tflops']:.0f} TFLOP/s x (1.1/2.25 nominal tf32:bf16) / 3",
                    **common}
        elif nuts:
            # warp per chain: a launch cannot end before its longest chain has
            # built its leaves one after another.  Bound: that critical path
            # at the per-leaf latency of one chain running alone (measured
            # here on the same target, dim and final step size)
            t_leaf = nuts_leaf_latency(p, final_eps)
            achieved = crit_per_step / kernel_s
            peak = 1.0 / t_leaf
            roof = {"bound": "latency", "achieved": achieved, "peak": peak,
                    "unit": "critical-path leaves/s", "frac": achieved / peak, "traffic": None,
                    "peak_source": f"measured: one chain alone, {t_leaf * 1e9:.0f} ns per leaf",
                    "critical_path_leaves_per_step": crit_per_step,
                    "leapfrog_steps_per_critical_leaf": evals_per_launch / crit_per_step, **common}
        elif flops is not None:
            # SIMT float32 products: FP32-pipe roofline from unit counts and clock
            achieved = flops * evals_per_launch / kernel_s / 1e12
            sm_max = pk.get("sm_max_mhz", 2070.0)
            peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                    **common}
        else:
            # fused elementwise transition: x and g read and written once per chain row
            bytes_per_launch = 4.0 * 4 * C * D
            achieved = bytes_per_launch / kernel_s / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "traffic": None,
                    "peak_source": src, **common}

    e2e = None
    if not args.no_e2e and streaming:
        # host state in, moments / ESS / traces out, through pinned buffers
        xh = torch.as_tensor(p.x0).pin_memory()
        outs = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (x, mean, m2, ess_d, eps, acc)]
        n_e2e = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            x.copy_(xh, non_blocking=True)
            hmc.hmc_sample_chain_streaming_ess(s.ctx, x, B, K, args.streaming, mean, m2, ess_d, eps, acc)
            for o, t in zip(outs, (x, mean, m2, ess_d, eps, acc)):
                o.copy_(t, non_blocking=True)
            torch.cuda.synchronize()
        el = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": world * evals_per_step / el, "unit": "grad-evals/s",
               "h2d_bytes_per_step": C * D * 4,
               "d2h_bytes_per_step": sum(o.numel() * o.element_size() for o in outs),
               "ms_per_step": 1000.0 * el}
    elif not args.no_e2e:
        xh = torch.empty((C, D), dtype=torch.float32, pin_memory=True)
        sh = torch.empty((K, C, D), dtype=torch.float32, pin_memory=True)
        eh = torch.empty(K, dtype=torch.float32, pin_memory=True)
        ah = torch.empty((K, C), dtype=torch.uint8, pin_memory=True)
        x0h = torch.as_tensor(p.x0)
        xh.copy_(x0h)
        hmc.hmc_sample_chain_host(s.ctx, xh, B, K, sh, eh, ah)   # warm the staging buffers
        n_e2e = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            xh.copy_(x0h)
            hmc.hmc_sample_chain_host(s.ctx, xh, B, K, sh, eh, ah)
        el = (time.perf_counter() - t0) / n_e2e
        if world > 1:
            t = torch.tensor([el], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * evals_per_step / el, "unit": "grad-evals/s",
               "h2d_bytes_per_step": C * D * 4,
               "d2h_bytes_per_step": (K * C * D + C * D) * 4 + K * 4 + K * C,
               "ms_per_step": 1000.0 * el}

    # The comparison target: the plain path (one kernel launch per operation
    # per leapfrog step, SIMT products) on the same workload and GPU, with
    # the same seed, L and adaptation -- statistically the same chains.
    vs = None
    if (not args.no_plain_baseline and not args.plain and not streaming and args.replicas == 1
            and proposal == hmc.HMC_PROPOSAL_LEAPFROG and p.kind in ("corr_gauss", "logreg")):
        vs = plain_baseline(p, stream, x, x0, samples, eps, acc, value / world, min_ess_per_s / world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(p, args.cpu_seconds, args.proposal)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        line = {
            "metric": "leapfrog grad-evals/s", "value": value, "unit": "grad-evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": vs, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "impl": "plain" if args.plain else "fused",
                       "chains": C, "dim": D,
                       "l2": ("each step first writes a 256 MB buffer (> 129 MB L2)" if streaming else
                              f"each step writes its {K * C * D * 4 / 1e9:.1f} GB kept-sample buffer "
                              "(> 129 MB L2), which flushes L2 between steps"),
                       "min_ess_estimator": "batch means (device)" if streaming else "BDA3 / Geyer (host, after the run)",
                       "parallelism": f"replicas x{world}",
                       "transitions_per_launch": args.max_transitions_per_launch or "all"},
            "min_ess_per_s": min_ess_per_s, "min_ess": min_ess,
            "final_step_size": final_eps, "accept_rate": accept_rate,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk,
        }
        if nuts_info:
            line["nuts_lockstep"] = nuts_info
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
