"""ctypes binding of libhmc (include/hmc.h): the same names, argument
marshalling only.  Every step of the sampler runs in the library's CUDA
kernels; importing this module raises if ``libhmc.so`` has not been built.

Device buffers are passed as torch CUDA tensors (float32 / uint8, contiguous)
or raw integer addresses; host buffers for ``hmc_sample_chain_host`` as numpy
arrays or CPU tensors.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhmc.so")

HMC_OK, HMC_E_INVALID, HMC_E_OOM, HMC_E_CUDA, HMC_E_TIMEOUT, HMC_E_UNSUPPORTED = range(6)
STATUS_NAMES = ["HMC_OK", "HMC_E_INVALID", "HMC_E_OOM", "HMC_E_CUDA", "HMC_E_TIMEOUT",
                "HMC_E_UNSUPPORTED"]
HMC_T_STD_NORMAL, HMC_T_CORR_GAUSS, HMC_T_LOGREG, HMC_T_FUNNEL = range(4)
TARGET_IDS = {"std_normal": 0, "corr_gauss": 1, "logreg": 2, "funnel": 3}
HMC_IMPL_FUSED, HMC_IMPL_PLAIN, HMC_IMPL_FUSED_SINGLE_CTA, HMC_IMPL_FUSED_TENSOR, HMC_IMPL_FUSED_SIMT = range(5)
HMC_PROPOSAL_LEAPFROG, HMC_PROPOSAL_RANDOM_WALK, HMC_PROPOSAL_NUTS = 0, 1, 2


class hmc_target(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("dim", ctypes.c_int32), ("n_data", ctypes.c_int64),
                ("P", ctypes.c_void_p), ("X", ctypes.c_void_p), ("y", ctypes.c_void_p)]


class hmc_config(ctypes.Structure):
    _fields_ = [("num_leapfrog", ctypes.c_int32), ("step_size", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("adapt", ctypes.c_int32),
                ("target_accept", ctypes.c_float), ("num_adapt_steps", ctypes.c_int64),
                ("impl", ctypes.c_int32), ("chain_offset", ctypes.c_int64),
                ("use_graph", ctypes.c_int32), ("max_transitions_per_launch", ctypes.c_int32),
                ("proposal", ctypes.c_int32)]


class hmc_proposal(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("target_log_prob", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("log_accept_ratio", ctypes.c_void_p)]


class hmc_kernel_results(ctypes.Structure):
    _fields_ = [("target_log_prob", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("is_accepted", ctypes.c_void_p), ("log_accept_ratio", ctypes.c_void_p),
                ("step_size", ctypes.c_void_p)]


class HMCError(RuntimeError):
    def __init__(self, status, message):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhmc.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    sigs = {
        "hmc_create": [ctypes.POINTER(hmc_target), ctypes.c_int64, ctypes.POINTER(hmc_config), P,
                       ctypes.POINTER(P)],
        "hmc_bootstrap": [P, P],
        "hmc_step": [P, P, ctypes.c_uint64, ctypes.POINTER(hmc_kernel_results)],
        "hmc_propose": [P, P, ctypes.c_uint64, ctypes.POINTER(hmc_proposal)],
        "hmc_nuts_leapfrog_count": [P, ctypes.POINTER(ctypes.c_uint64)],
        "hmc_nuts_leaf_iterations": [P, ctypes.POINTER(ctypes.c_uint64)],
        "hmc_mh_select": [P, P, ctypes.c_uint64, ctypes.POINTER(hmc_kernel_results)],
        "hmc_sample_chain": [P, P, ctypes.c_int64, ctypes.c_int64, P, P, P],
        "hmc_sample_chain_host": [P, P, ctypes.c_int64, ctypes.c_int64, P, P, P],
        "hmc_read_adaptation": [P, ctypes.POINTER(ctypes.c_double)],
        "hmc_sample_chain_range": [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P],
        "hmc_state_bytes": [P, ctypes.POINTER(ctypes.c_uint64)],
        "hmc_create_device_bytes": [ctypes.POINTER(hmc_target), ctypes.c_int64, ctypes.POINTER(hmc_config),
                                    ctypes.POINTER(ctypes.c_uint64)],
        "hmc_context_device_bytes": [P, ctypes.POINTER(ctypes.c_uint64)],
        "hmc_save_state": [P, P, ctypes.c_uint64],
        "hmc_restore_state": [P, P, ctypes.c_uint64],
        "hmc_destroy": [P],
        "hmc_grad_workspace_bytes": [ctypes.POINTER(hmc_target), ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_uint64)],
        "hmc_target_log_prob_and_grad": [ctypes.POINTER(hmc_target), ctypes.c_int64, P, P, P, P,
                                         ctypes.c_uint64, P],
        "hmc_synchronize": [P],
        "hmc_remc_create": [ctypes.POINTER(hmc_target), ctypes.c_int64, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(hmc_config), P,
                            ctypes.POINTER(P)],
        "hmc_remc_swaps": [P, ctypes.POINTER(P)],
        "hmc_batch_create": [ctypes.c_int32, ctypes.POINTER(hmc_target), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(hmc_config), P, ctypes.POINTER(P)],
        "hmc_batch_sample_chain": [P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(P),
                                   ctypes.POINTER(P), ctypes.POINTER(P)],
        "hmc_batch_destroy": [P],
        "hmc_batch_synchronize": [P],
        "hmc_batch_create_autotuned": [ctypes.c_int32, ctypes.POINTER(hmc_target), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(hmc_config), P, ctypes.POINTER(P)],
        "hmc_batch_member_path": [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "hmc_sample_chain_streaming": [P, P, ctypes.c_int64, ctypes.c_int64, P, P, P, P],
        "hmc_sample_chain_streaming_ess": [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P,
                                           P, P, P],
        "hmc_dominant_kernel_info": [P, ctypes.c_char_p, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int64)],
        "hmc_target_vjp_workspace_bytes": [ctypes.POINTER(hmc_target), ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_uint64)],
        "hmc_target_vjp": [ctypes.POINTER(hmc_target), ctypes.c_int64, P, P, P, P, ctypes.c_uint64,
                           P],
        "hmc_target_log_prob_and_grad_noalloc": [ctypes.POINTER(hmc_target), ctypes.c_int64, P, P,
                                                 P, P],
        "hmc_profile_dominant_kernel": [P, ctypes.c_int32],
        "hmc_profile_read": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_uint64)],
        "hmc_philox4x32_10": [P, ctypes.c_int64, ctypes.c_uint64, P, P],
        "hmc_momentum": [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                         ctypes.c_int64, P, P],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hmc_last_error.argtypes = [P]
    lib.hmc_last_error.restype = ctypes.c_char_p
    lib.hmc_uses_tensor_cores.argtypes = [P]
    lib.hmc_uses_tensor_cores.restype = ctypes.c_int32
    lib.hmc_batch_last_error.argtypes = [P]
    lib.hmc_batch_last_error.restype = ctypes.c_char_p
    lib.hmc_batch_context.argtypes = [P, ctypes.c_int32]
    lib.hmc_batch_context.restype = P
    lib.hmc_debug_set_grid_barrier.argtypes = [ctypes.c_uint64, ctypes.c_int32]
    lib.hmc_debug_set_grid_barrier.restype = None
    lib.hmc_kernel_launch_count.argtypes = []
    lib.hmc_kernel_launch_count.restype = ctypes.c_uint64
    return lib


lib = _load()


def _ptr(t):
    """Address of a tensor / array / raw int (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("buffers passed to libhmc must be contiguous")
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers passed to libhmc must be contiguous")
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status, ctx=None):
    if status != HMC_OK:
        msg = lib.hmc_last_error(ctx)
        raise HMCError(status, msg.decode() if msg else "")


def make_target(kind, dim, P=None, X=None, y=None):
    """hmc_target for a family name or id; P, X, y are device tensors (kept
    alive by the caller)."""
    tid = TARGET_IDS[kind] if isinstance(kind, str) else int(kind)
    n = 0 if X is None else int(X.shape[0])
    return hmc_target(tid, int(dim), n, _ptr(P), _ptr(X), _ptr(y))


def make_config(num_leapfrog, step_size, seed=0, adapt=False, target_accept=0.65,
                num_adapt_steps=0, impl=HMC_IMPL_FUSED, chain_offset=0, use_graph=True,
                max_transitions_per_launch=0, proposal=HMC_PROPOSAL_LEAPFROG):
    return hmc_config(int(num_leapfrog), float(step_size), int(seed) & 0xFFFFFFFFFFFFFFFF,
                      int(bool(adapt)), float(target_accept), int(num_adapt_steps), int(impl),
                      int(chain_offset), int(bool(use_graph)), int(max_transitions_per_launch),
                      int(proposal))


def hmc_create(target, num_chains, config, stream=None):
    ctx = ctypes.c_void_p()
    _check(lib.hmc_create(ctypes.byref(target), int(num_chains), ctypes.byref(config),
                          _stream(stream), ctypes.byref(ctx)))
    return ctx.value


def hmc_bootstrap(ctx, x0):
    _check(lib.hmc_bootstrap(ctx, _ptr(x0)), ctx)


def hmc_step(ctx, x_inout, t):
    out = hmc_kernel_results()
    _check(lib.hmc_step(ctx, _ptr(x_inout), int(t), ctypes.byref(out)), ctx)
    return out


def hmc_nuts_leapfrog_count(ctx):
    out = ctypes.c_uint64()
    _check(lib.hmc_nuts_leapfrog_count(ctx, ctypes.byref(out)), ctx)
    return int(out.value)


def hmc_nuts_leaf_iterations(ctx):
    out = ctypes.c_uint64()
    _check(lib.hmc_nuts_leaf_iterations(ctx, ctypes.byref(out)), ctx)
    return int(out.value)


def hmc_propose(ctx, x, t):
    out = hmc_proposal()
    _check(lib.hmc_propose(ctx, _ptr(x), int(t), ctypes.byref(out)), ctx)
    return out


def hmc_mh_select(ctx, x_inout, t):
    out = hmc_kernel_results()
    _check(lib.hmc_mh_select(ctx, _ptr(x_inout), int(t), ctypes.byref(out)), ctx)
    return out


def hmc_sample_chain(ctx, x_inout, num_burnin, num_results, samples_out=None,
                     trace_step_size=None, trace_accept=None):
    _check(lib.hmc_sample_chain(ctx, _ptr(x_inout), int(num_burnin), int(num_results),
                                _ptr(samples_out), _ptr(trace_step_size), _ptr(trace_accept)), ctx)


def hmc_sample_chain_range(ctx, x_inout, num_burnin, t_begin, t_end, samples_out=None,
                           trace_step_size=None, trace_accept=None):
    _check(lib.hmc_sample_chain_range(ctx, _ptr(x_inout), int(num_burnin), int(t_begin), int(t_end),
                                      _ptr(samples_out), _ptr(trace_step_size), _ptr(trace_accept)), ctx)


def hmc_create_device_bytes(target, num_chains, config):
    n = ctypes.c_uint64()
    _check(lib.hmc_create_device_bytes(ctypes.byref(target), int(num_chains), ctypes.byref(config),
                                       ctypes.byref(n)))
    return int(n.value)


def hmc_context_device_bytes(ctx):
    n = ctypes.c_uint64()
    _check(lib.hmc_context_device_bytes(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def hmc_state_bytes(ctx):
    n = ctypes.c_uint64()
    _check(lib.hmc_state_bytes(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def hmc_save_state(ctx):
    """The context's resumable state as bytes (kernel results + adaptation)."""
    buf = ctypes.create_string_buffer(hmc_state_bytes(ctx))
    _check(lib.hmc_save_state(ctx, buf, len(buf)), ctx)
    return buf.raw


def hmc_restore_state(ctx, state):
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(lib.hmc_restore_state(ctx, buf, len(state)), ctx)


def hmc_debug_set_grid_barrier(wait_limit_ns=500_000_000, unreachable_generation=0):
    lib.hmc_debug_set_grid_barrier(int(wait_limit_ns), int(unreachable_generation))


def hmc_sample_chain_host(ctx, x_inout, num_burnin, num_results, samples_out=None,
                          trace_step_size=None, trace_accept=None):
    _check(lib.hmc_sample_chain_host(ctx, _ptr(x_inout), int(num_burnin), int(num_results),
                                     _ptr(samples_out), _ptr(trace_step_size),
                                     _ptr(trace_accept)), ctx)


def hmc_read_adaptation(ctx):
    out = (ctypes.c_double * 5)()
    _check(lib.hmc_read_adaptation(ctx, out), ctx)
    return {"step_size": out[0], "log_eps_bar": out[1], "h_bar": out[2], "m": int(out[3]),
            "last_stat": out[4]}


def hmc_destroy(ctx):
    _check(lib.hmc_destroy(ctx))


def hmc_last_error(ctx=None):
    return lib.hmc_last_error(ctx).decode()


def hmc_grad_workspace_bytes(target, num_chains):
    b = ctypes.c_uint64()
    _check(lib.hmc_grad_workspace_bytes(ctypes.byref(target), int(num_chains), ctypes.byref(b)))
    return int(b.value)


def hmc_target_log_prob_and_grad(target, num_chains, x, lp, grad, workspace=None,
                                 workspace_bytes=0, stream=None):
    _check(lib.hmc_target_log_prob_and_grad(ctypes.byref(target), int(num_chains), _ptr(x),
                                            _ptr(lp), _ptr(grad), _ptr(workspace),
                                            int(workspace_bytes), _stream(stream)))


def hmc_kernel_launch_count():
    return int(lib.hmc_kernel_launch_count())


def hmc_philox4x32_10(counters, n, seed, out, stream=None):
    _check(lib.hmc_philox4x32_10(_ptr(counters), int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out),
                                 _stream(stream)))


def hmc_momentum(seed, t, num_chains, dim, chain_offset, out, stream=None):
    _check(lib.hmc_momentum(int(seed) & 0xFFFFFFFFFFFFFFFF, int(t), int(num_chains), int(dim),
                            int(chain_offset), _ptr(out), _stream(stream)))


def hmc_profile_dominant_kernel(ctx, sample_every):
    _check(lib.hmc_profile_dominant_kernel(ctx, int(sample_every)), ctx)


def hmc_profile_read(ctx):
    ms, n, launches = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.hmc_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(launches)), ctx)
    return {"avg_ms": ms.value, "samples": int(n.value), "launches": int(launches.value)}


def hmc_synchronize(ctx):
    _check(lib.hmc_synchronize(ctx), ctx)


def hmc_uses_tensor_cores(ctx):
    return bool(lib.hmc_uses_tensor_cores(ctx))


def hmc_target_log_prob_and_grad_noalloc(target, num_chains, x, lp, grad, stream=None):
    """Gradient for callers that cannot allocate: scratch comes from a fixed
    64 MiB array inside the library (see include/hmc.h)."""
    _check(lib.hmc_target_log_prob_and_grad_noalloc(ctypes.byref(target), int(num_chains), _ptr(x),
                                                    _ptr(lp), _ptr(grad), _stream(stream)))


def hmc_target_vjp_workspace_bytes(target, num_chains):
    b = ctypes.c_uint64()
    _check(lib.hmc_target_vjp_workspace_bytes(ctypes.byref(target), int(num_chains), ctypes.byref(b)))
    return int(b.value)


def hmc_target_vjp(target, num_chains, x, w, dx, workspace, workspace_bytes, stream=None):
    _check(lib.hmc_target_vjp(ctypes.byref(target), int(num_chains), _ptr(x), _ptr(w), _ptr(dx),
                              _ptr(workspace), int(workspace_bytes), _stream(stream)))


def hmc_dominant_kernel_info(ctx):
    buf = ctypes.create_string_buffer(128)
    per = ctypes.c_int64()
    _check(lib.hmc_dominant_kernel_info(ctx, buf, 128, ctypes.byref(per)), ctx)
    return buf.value.decode(), int(per.value)


def hmc_sample_chain_streaming(ctx, x_inout, num_burnin, num_results, mean_out, m2_out,
                               trace_step_size=None, trace_accept=None):
    _check(lib.hmc_sample_chain_streaming(ctx, _ptr(x_inout), int(num_burnin), int(num_results),
                                          _ptr(mean_out), _ptr(m2_out), _ptr(trace_step_size),
                                          _ptr(trace_accept)), ctx)


def hmc_sample_chain_streaming_ess(ctx, x_inout, num_burnin, num_results, batch_size, mean_out,
                                   m2_out, ess_out, trace_step_size=None, trace_accept=None):
    _check(lib.hmc_sample_chain_streaming_ess(ctx, _ptr(x_inout), int(num_burnin), int(num_results),
                                              int(batch_size), _ptr(mean_out), _ptr(m2_out),
                                              _ptr(ess_out), _ptr(trace_step_size),
                                              _ptr(trace_accept)), ctx)


def _check_batch(status, batch):
    if status != HMC_OK:
        msg = lib.hmc_batch_last_error(batch) if batch else lib.hmc_last_error(None)
        raise HMCError(status, msg.decode() if msg else "")


def hmc_batch_create(targets, num_chains, configs, stream=None):
    n = len(targets)
    T = (hmc_target * n)(*targets)
    Cs = (ctypes.c_int64 * n)(*[int(c) for c in num_chains])
    G = (hmc_config * n)(*configs)
    out = ctypes.c_void_p()
    _check_batch(lib.hmc_batch_create(n, T, Cs, G, _stream(stream), ctypes.byref(out)), None)
    return out.value


def hmc_batch_create_autotuned(targets, num_chains, configs, stream=None):
    n = len(targets)
    T = (hmc_target * n)(*targets)
    Cs = (ctypes.c_int64 * n)(*[int(c) for c in num_chains])
    G = (hmc_config * n)(*configs)
    out = ctypes.c_void_p()
    _check_batch(lib.hmc_batch_create_autotuned(n, T, Cs, G, _stream(stream), ctypes.byref(out)), None)
    return out.value


def hmc_batch_member_path(batch, i):
    """(path, ms_grouped, ms_tensor) of posterior i: path 0 grouped launch,
    1 own context on tensor cores (autotuned), 2 own context (untuned rule)."""
    path = ctypes.c_int32()
    mg, mt = ctypes.c_double(), ctypes.c_double()
    _check_batch(lib.hmc_batch_member_path(batch, int(i), ctypes.byref(path), ctypes.byref(mg),
                                           ctypes.byref(mt)), batch)
    return int(path.value), float(mg.value), float(mt.value)


def hmc_batch_sample_chain(batch, xs, num_burnin, num_results, samples=None, trace_step_size=None,
                           trace_accept=None):
    n = len(xs)
    arr = lambda seq: (ctypes.c_void_p * n)(*[_ptr(v) for v in seq]) if seq is not None else None
    B = (ctypes.c_int64 * n)(*[int(v) for v in num_burnin])
    K = (ctypes.c_int64 * n)(*[int(v) for v in num_results])
    _check_batch(lib.hmc_batch_sample_chain(batch, arr(xs), B, K, arr(samples), arr(trace_step_size),
                                            arr(trace_accept)), batch)


def hmc_batch_context(batch, i):
    return lib.hmc_batch_context(batch, int(i))


def hmc_batch_destroy(batch):
    _check_batch(lib.hmc_batch_destroy(batch), None)


def hmc_remc_create(target, num_chains, betas, config, stream=None):
    n = len(betas)
    arr = (ctypes.c_float * n)(*[float(b) for b in betas])
    ctx = ctypes.c_void_p()
    _check(lib.hmc_remc_create(ctypes.byref(target), int(num_chains), n, arr, ctypes.byref(config),
                               _stream(stream), ctypes.byref(ctx)))
    return ctx.value


def hmc_remc_swaps(ctx):
    p = ctypes.c_void_p()
    _check(lib.hmc_remc_swaps(ctx, ctypes.byref(p)), ctx)
    return p.value


def hmc_batch_synchronize(batch):
    _check_batch(lib.hmc_batch_synchronize(batch), batch)
