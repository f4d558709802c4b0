"""Continuous-batching sampling server.

Requests (posterior + sampling schedule) arrive over time.  A request is
admitted as soon as a slot is free and its device memory fits the HBM budget;
its chain state stays resident on the device for the whole job, its
transitions are enqueued on the slot's own CUDA stream, so the work of every
admitted job overlaps on the GPU, and a finished job frees its slot and memory
for the next one.  All sampling work runs in libhmc's kernels; this loop only
admits, polls and copies results to the host.  Because every random draw is
keyed by (seed, chain, transition) and every job owns its state and step-size
adaptation, a job's result is the same whether it runs alone or in the mix.

The host work of a job -- creating its context, capturing and instantiating
its chain's CUDA graph (tens of milliseconds for a long logistic-regression
chain: two dozen launches per transition), and destroying it afterwards --
runs on a pool of admission threads (the library's calls release the
interpreter lock; each context captures on its own stream in thread-local
mode), so that the loop keeps admitting and polling meanwhile.
"""
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np
import torch

from . import diagnostics, hmc
from .sampler import Sampler


def job_bytes(problem, keep_samples=True):
    """Device bytes a job holds while resident: the library context's
    workspace (hmc_create_device_bytes, for the configuration the job's
    Sampler builds), the target data the Sampler copies to the device, the
    chain state and the job's traces."""
    C, D, K = problem.num_chains, problem.dim, problem.num_results
    n_data = 0 if problem.X is None else int(problem.X.shape[0])
    target = hmc.hmc_target(hmc.TARGET_IDS[problem.kind], int(D), n_data, None, None, None)
    config = hmc.make_config(problem.num_leapfrog, problem.step_size, problem.seed, problem.adapt,
                             problem.target_accept, problem.num_burnin if problem.adapt else 0,
                             hmc.HMC_IMPL_FUSED, 0, True)
    b = hmc.hmc_create_device_bytes(target, C, config)
    if problem.P is not None:
        b += 4 * problem.P.size
    if problem.X is not None:
        b += 4 * problem.X.size + 4 * problem.y.size
    b += 4 * C * D                                   # chain state
    b += 4 * K + K * C                               # step-size and accept traces
    if keep_samples:
        b += 4 * K * C * D
    return int(b)


@dataclass
class Job:
    id: int
    arrival: float
    problem: object
    admitted: float = None
    finished: float = None
    result: dict = field(default_factory=dict)
    _sampler: object = None
    _x: object = None
    _samples: object = None
    _eps: object = None
    _acc: object = None
    _event: object = None
    _bytes: int = 0
    _slot: int = -1
    _future: object = None


class Server:
    def __init__(self, hbm_budget_bytes=150 * 2 ** 30, slots=16, keep_samples=True,
                 ess_dims=8, device="cuda", workers=4):
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.keep_samples = keep_samples
        self.ess_dims = ess_dims
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.active = []
        self.done = []
        self.backlog = 0
        # host time in the steps: admission and teardown on the worker
        # threads, results on the loop's thread
        self.host_s = {"admit": 0.0, "finish": 0.0, "teardown": 0.0}
        self._lock = threading.Lock()
        self.workers = workers
        self._pool = None

    def _time(self, key, t0):
        with self._lock:
            self.host_s[key] += time.perf_counter() - t0

    # -- admission ---------------------------------------------------------
    def fits(self, job):
        return bool(self.free_slots) and self.used + job_bytes(job.problem, self.keep_samples) <= self.budget

    def admit(self, job, now):
        """Reserve a slot and the job's bytes; its context and chain start on
        an admission thread (or here, with workers=0)."""
        p = job.problem
        slot = self.free_slots.pop(0)
        job._slot = slot
        job._bytes = job_bytes(p, self.keep_samples)
        self.used += job._bytes
        job.admitted = now
        if self._pool is not None:
            job._future = self._pool.submit(self._start, job)
        else:
            self._start(job)
        self.active.append(job)

    def _start(self, job):
        h0 = time.perf_counter()
        p = job.problem
        stream = self.streams[job._slot]
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            job._sampler = Sampler(p, stream=stream, use_graph=True)
            x = torch.empty((p.num_chains, p.dim), dtype=torch.float32, device="cuda")
            x.copy_(torch.from_numpy(p.x0).pin_memory(), non_blocking=True)
            job._x = x
            K = p.num_results
            job._samples = torch.empty((K, p.num_chains, p.dim), device="cuda") if self.keep_samples else None
            job._eps = torch.empty(K, device="cuda")
            job._acc = torch.empty((K, p.num_chains), dtype=torch.uint8, device="cuda")
            hmc.hmc_sample_chain(job._sampler.ctx, x, p.num_burnin, K, job._samples, job._eps, job._acc)
            ev = torch.cuda.Event()
            ev.record(stream)
            job._event = ev
        self._time("admit", h0)

    # -- completion ----------------------------------------------------------
    def poll(self, now_fn):
        still = []
        for job in self.active:
            if job._future is not None:
                if not job._future.done():
                    still.append(job)
                    continue
                job._future.result()           # an admission error surfaces here
                job._future = None
            if job._event.query():
                self.finish(job, now_fn())
            else:
                still.append(job)
        self.active = still

    def finish(self, job, now):
        h0 = time.perf_counter()
        p = job.problem
        stream = self.streams[job._slot]
        with torch.cuda.stream(stream):
            res = {"x": job._x.cpu().numpy(), "step_size": job._eps.cpu().numpy(),
                   "accept_rate": float(job._acc.float().mean().item()) if p.num_results else None}
            if job._samples is not None and p.num_results >= 4 and p.num_chains >= 2:
                # the cheap batch-means figure (one batch per chain): the FFT
                # estimator's plans and launches cost more than the job itself
                res["min_ess"] = float(diagnostics.ess_batch_means(job._samples, max_dims=self.ess_dims).min())
                res["mean"] = job._samples.mean(dim=(0, 1)).cpu().numpy()
            torch.cuda.current_stream().synchronize()
        job.finished = now
        job.result = res
        sampler = job._sampler
        job._sampler = job._x = job._samples = job._eps = job._acc = None
        if self._pool is not None:
            self._pool.submit(self._teardown, sampler)
        else:
            self._teardown(sampler)
        self.used -= job._bytes
        self.free_slots.append(job._slot)
        self.done.append(job)
        self._time("finish", h0)

    def _teardown(self, sampler):
        # the context's graph and stream-ordered memory go on its own stream
        h0 = time.perf_counter()
        sampler.close()
        self._time("teardown", h0)

    # -- the loop ------------------------------------------------------------
    def run(self, requests, time_scale=1.0, max_wall=None):
        """Serve (arrival_time, problem) requests; arrival times are divided
        by `time_scale` (to compress a long stream).  Returns the jobs."""
        jobs = [Job(i, t / time_scale, p) for i, (t, p) in enumerate(requests)]
        pending = list(jobs)
        self._pool = ThreadPoolExecutor(max_workers=self.workers) if self.workers > 0 else None
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or self.active:
            t = now()
            if max_wall is not None and t > max_wall:
                break
            while pending and pending[0].arrival <= t and self.fits(pending[0]):
                self.admit(pending.pop(0), now())
            if pending and pending[0].arrival <= t and not self.active and not self.fits(pending[0]):
                raise RuntimeError(f"request {pending[0].id} needs more than the HBM budget")
            self.poll(now)
            time.sleep(0.0005)
        self.wall = now()
        self.backlog = len(pending) + len(self.active)
        if self._pool is not None:
            # teardowns still queued finish here; a run stopped by max_wall
            # leaves its active jobs' contexts to the process's exit
            self._pool.shutdown(wait=True)
            self._pool = None
        return jobs


def summarize(jobs, wall):
    """Served against offered load and the completed requests' latencies.

    grad_evals_per_s: leapfrog gradient evaluations of the completed
    requests over the wall time; offered_grad_evals_per_s: those of every
    request over the arrival span.  ess_per_s: the completed requests'
    min-ESS (each request's smallest over its dimensions) summed, over the
    wall time -- effective draws the server delivered per second;
    job_min_ess_per_s_p50: the median over completed requests of that
    request's min-ESS over its own time in the system."""
    done = [j for j in jobs if j.finished is not None]
    lat = np.array([j.finished - j.arrival for j in done]) if done else np.array([np.nan])
    work = lambda j: j.problem.num_chains * j.problem.num_leapfrog * (j.problem.num_burnin + j.problem.num_results)
    evals = sum(work(j) for j in done)
    offered = sum(work(j) for j in jobs)
    ess = [j.result.get("min_ess") for j in done if j.result.get("min_ess") is not None]
    per_job = [j.result["min_ess"] / (j.finished - j.arrival) for j in done
               if j.result.get("min_ess") is not None and j.finished > j.arrival]
    span = max(j.arrival for j in jobs) if jobs else 0.0
    return {"requests": len(jobs), "completed": len(done), "wall_s": wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "grad_evals_per_s": evals / wall if wall else None,
            "offered_grad_evals_per_s": offered / span if span else None,
            "completed_work_fraction": evals / offered if offered else None,
            "ess_per_s": (sum(ess) / wall) if ess and wall else None,
            "job_min_ess_per_s_p50": float(np.median(per_job)) if per_job else None}
