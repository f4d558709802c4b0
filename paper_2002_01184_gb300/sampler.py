"""Convenience layer over the binding: holds a workload's target data on the
device and one libhmc context.  All sampling work runs in libhmc's kernels."""
import torch

from . import hmc


class Sampler:
    """One posterior (a ``workloads.Problem``) bound to a libhmc context."""

    def __init__(self, problem, impl=hmc.HMC_IMPL_FUSED, num_chains=None, chain_offset=0,
                 step_size=None, adapt=None, stream=None, device="cuda", use_graph=True,
                 max_transitions_per_launch=0, proposal=hmc.HMC_PROPOSAL_LEAPFROG):
        self.problem = problem
        self.C = int(num_chains or problem.num_chains)
        self.D = int(problem.dim)
        self.device = torch.device(device)
        dev = lambda a: None if a is None else torch.as_tensor(a).to(self.device).contiguous()
        self.P, self.X, self.y = dev(problem.P), dev(problem.X), dev(problem.y)
        self.target = hmc.make_target(problem.kind, self.D, self.P, self.X, self.y)
        adapt = problem.adapt if adapt is None else adapt
        self.config = hmc.make_config(
            problem.num_leapfrog, problem.step_size if step_size is None else step_size,
            problem.seed, adapt, problem.target_accept,
            problem.num_burnin if adapt else 0, impl, chain_offset, use_graph,
            max_transitions_per_launch, proposal)
        self.stream = stream
        self.ctx = hmc.hmc_create(self.target, self.C, self.config, stream)

    def bootstrap(self, x):
        hmc.hmc_bootstrap(self.ctx, x)

    def step(self, x, t):
        return hmc.hmc_step(self.ctx, x, t)

    def results(self, r):
        """Copy the device kernel results of the last step into new tensors."""
        torch.cuda.current_stream().synchronize()
        return {
            "target_log_prob": device_view(r.target_log_prob, (self.C,), "<f4").clone(),
            "grad": device_view(r.grad, (self.C, self.D), "<f4").clone(),
            "is_accepted": device_view(r.is_accepted, (self.C,), "|u1").clone(),
            "log_accept_ratio": device_view(r.log_accept_ratio, (self.C,), "<f4").clone(),
            "step_size": device_view(r.step_size, (1,), "<f4").clone(),
        }

    def sample_chain(self, x, num_burnin, num_results, keep_samples=True):
        K = int(num_results)
        samples = torch.empty((K, self.C, self.D), dtype=torch.float32, device=self.device) \
            if keep_samples else None
        eps = torch.empty(K, dtype=torch.float32, device=self.device)
        acc = torch.empty((K, self.C), dtype=torch.uint8, device=self.device)
        hmc.hmc_sample_chain(self.ctx, x, num_burnin, K, samples, eps, acc)
        return samples, eps, acc

    def adaptation(self):
        return hmc.hmc_read_adaptation(self.ctx)

    def close(self):
        if self.ctx:
            hmc.hmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr, shape, typestr):
    """Zero-copy torch view of library-owned device memory (valid until the
    next call on the context)."""
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")
